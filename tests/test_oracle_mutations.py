"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in the oracle, on the
CPU, through pytest's monkeypatch (undone when the case ends).  It then checks that a named
pin fails on it.  The original oracle passes every one of these pins in their own test files.
"""
import importlib

import numpy as np
import pytest

import oracle
import test_oracle_grid as pins_grid
import test_oracle_place as pins_place
import test_oracle_table as pins_table

table_mod = importlib.import_module("oracle.table")
grid_mod = importlib.import_module("oracle.grid")
place_mod = importlib.import_module("oracle.place")


def test_conjugated_w_screen_fails_the_direct_fourier_image(monkeypatch):
    # the screen of 1/g_w with the wrong sign: w-projection then doubles the w-term
    screen = table_mod.exact_screen
    monkeypatch.setattr(table_mod, "exact_screen", lambda w, l, m: np.conj(screen(w, l, m)))
    with pytest.raises(AssertionError):
        pins_grid.test_end_to_end_against_direct_fourier(17, 60.0)


def test_transposed_kernel_fails_the_closed_form(monkeypatch):
    # kernel rows and columns swapped (u <-> v, eq. "choose" read the other way)
    trim = table_mod._trim
    monkeypatch.setattr(table_mod, "_trim", lambda C, beta, S: trim(C.T, beta, S))
    with pytest.raises(AssertionError):
        pins_table.test_closed_form_paraxial_gaussian()


def test_dropped_take_conjugate_fails_the_direct_fourier_image(monkeypatch):
    # records with w < 0 are moved to (-u, -v, -w) but their visibilities are not conjugated
    def weighted_no_conj(pl, vis, weight, flag, cross_swap=False):
        P = np.asarray(vis).shape[-1]
        v = np.asarray(vis, dtype=np.complex128).reshape(-1, P)
        wf = np.asarray(weight, np.float64).reshape(-1, P) * (1.0 - np.asarray(flag, np.float64).reshape(-1, P))
        return wf * v

    monkeypatch.setattr(grid_mod, "weighted_vis", weighted_no_conj)
    with pytest.raises(AssertionError):
        pins_grid.test_end_to_end_against_direct_fourier(17, 60.0)


def test_cell_split_with_upward_ties_fails_the_exact_rationals(monkeypatch):
    # sub-cell offsets in [-beta/2, beta/2) instead of (-beta/2, beta/2]
    def cell_ties_up(q, beta):
        qi = q.astype(np.int64)
        xc = (2 * qi + beta) // (2 * beta)
        return xc, qi - beta * xc

    monkeypatch.setattr(place_mod, "_cell", cell_ties_up)
    with pytest.raises(AssertionError):
        pins_place.test_exact_cell_and_suboffset(8)


def test_compression_without_kernel_pointer_fails_invariance(monkeypatch):
    # eq. "ci" compared on the footprint alone: records with another sub-cell offset merge
    def classify_footprint_only(pl):
        rows, C = pl.rows, pl.C
        gd = pl.griddable.reshape(rows, C)
        x0, y0 = pl.x0.reshape(rows, C), pl.y0.reshape(rows, C)
        c = np.zeros((rows, C), dtype=bool)
        c[1:] = gd[1:] & gd[:-1] & (x0[1:] == x0[:-1]) & (y0[1:] == y0[:-1])
        return (gd & ~c).reshape(-1), c.reshape(-1)

    monkeypatch.setattr(oracle, "classify", classify_footprint_only)
    with pytest.raises(AssertionError):
        pins_grid.test_compression_invariance_on_tracks()


def test_normaliser_without_zeta_fails_the_unit_point_source(monkeypatch):
    # eq. "normalizer" with the kernel sums zeta dropped
    def normaliser_no_zeta(pl, table, weight, flag, interleave=False, cross_swap=False):
        P = np.asarray(weight).shape[-1]
        wf = np.asarray(weight, np.float64).reshape(-1, P) * (1.0 - np.asarray(flag, np.float64).reshape(-1, P))
        out = np.zeros((pl.C, P))
        np.add.at(out, pl.chan, wf * pl.griddable[:, None])
        return out

    monkeypatch.setattr(oracle, "normaliser", normaliser_no_zeta)
    with pytest.raises(AssertionError):
        pins_grid.test_point_source_peak_is_one()
