"""FP64 CPU oracle for w-projection convolutional gridding with compression.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
and reference legs may import, call, link or execute anything in this package.  The
product (paper_1403_4209_gb300) never imports it, and it never imports the product:
the two share no code, headers, tables or constant generators.  Both consume the
seeded inputs of the separate `synth` module.

Every function is the plain definition the thesis gives, or (for the table build) the
steps of its Algorithm "convgen" in order, in FP64:

  pswf.psi0           prolate spheroidal taper (Sec. 2.3.3), via scipy.special.pro_ang1
  table.build_table   Algorithm "convgen" + outputs C-1/C-2/C-3 (Sec. 4.2.2, 4.2.3)
  place.place         record placement, w-plane, take-conjugate (Sec. 4.2.2 eqs.
                      "choose"/"sat", Sec. 4.3.3 position tuple, eq. "conj")
  place.classify      griddable / compression indicators (Sec. 4.3.2-4.3.4, eq. "ci")
  grid.grid_plain     eq. "gridding" summed record by record, no compression
  grid.grid_compressed  compression (eqs. "compress1", "conjugatetake") then gridding
  grid.normaliser     eq. "normalizer"
  grid.stats          the four statistics of Sec. 4.3.4
  grid.degrid         adjoint of the gridding map (not in the thesis)
  correct.grid_correct  Algorithm "finalizer" steps 1-4 (Sec. 4.7)
  dft.dirty_image     direct Fourier inversion including the w-term (Sec. 1.4 / 2.2.1)
  model.forward / model.adjoint / model.chi2_grad
                      sky -> visibility forward model from degridding, its adjoint and the
                      chi^2 gradient (not in the thesis)

Parity pins (tests/test_oracle_*.py) tie each of these to something other than itself:
closed forms, brute force, invariants and worked counts from the thesis.  Kernel values
for the exact (non-paraxial) w-screen are pinned by direct 2-D Fourier sums: on whole tables
for small patches, and on sampled values of the w-projection workload's 256^2-patch table
up to its w_max.  Tables on larger patches (the 8192^2 workload's 512^2) are not sampled;
they run the same steps.  The thesis prints no kernel values.
"""
from .cloops import lib  # noqa: F401  (compiles oracle.c on first use)
from .pswf import psi0
from .table import Table, build_table, delta_table
from .place import place, classify, Placement
from .grid import grid_plain, grid_compressed, compress, normaliser, stats, degrid, weighted_vis
from .correct import grid_correct, grid_correct_stokes, taper_1d
from .dft import dirty_image
from . import model, weighting, wstack

__all__ = [
    "psi0", "Table", "build_table", "delta_table", "place", "classify", "Placement",
    "grid_plain", "grid_compressed", "compress", "normaliser", "stats", "degrid",
    "weighted_vis", "grid_correct", "taper_1d", "dirty_image",
]
