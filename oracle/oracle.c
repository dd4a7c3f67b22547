/*
 * oracle.c -- plain, slow FP64 loops for the w-projection gridding path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference leg may load this library.  It shares no code with the
 * CUDA path.  Built with -O2 -ffp-contract=off so every FP64 operation is rounded
 * exactly as written.
 *
 * Conventions (thesis Sec. 4.2.2 and 4.3.3):
 *   grid   : complex double, [C][N][N][P] (pixel (y,x) holds P polarisations),
 *            pixel (0,0) has the most negative u,v; u=v=0 at index N/2.
 *   table  : complex double samples of the oversampled w-kernels, one S x S row-major
 *            sub-kernel per (plane, sub-offset); z is the index of a sub-kernel's
 *            first sample (the "Convolution Data Pointer" of Sec. 4.3.3).
 *   record : one (row, channel) pair with P polarisations.
 */
#include <stdint.h>
#include <string.h>

/* Eq. "gridding" (Sec. 4.3.2): grid_p(x0+j, y0+i) += q_p * K[z + i*S + j]
 * for every listed record; q already holds eps*(1-f)*(psi-conjugated) vis. */
void or_grid(int64_t n, const int32_t* chan, const int32_t* x0, const int32_t* y0,
             const int64_t* z, const int32_t* S, const double* q, int32_t P, int32_t N,
             const double* table, double* grid)
{
    for (int64_t r = 0; r < n; ++r) {
        const int32_t s = S[r];
        const double* k = table + 2 * z[r];
        double* g0 = grid + 2 * ((int64_t)chan[r] * N * N * P);
        for (int32_t i = 0; i < s; ++i) {
            for (int32_t j = 0; j < s; ++j) {
                const double kr = k[2 * (i * s + j)];
                const double ki = k[2 * (i * s + j) + 1];
                const int64_t pix = ((int64_t)(y0[r] + i) * N + (x0[r] + j)) * P;
                for (int32_t p = 0; p < P; ++p) {
                    const double qr = q[2 * (r * P + p)];
                    const double qi = q[2 * (r * P + p) + 1];
                    g0[2 * (pix + p)] += qr * kr - qi * ki;
                    g0[2 * (pix + p) + 1] += qr * ki + qi * kr;
                }
            }
        }
    }
}

/* Adjoint of or_grid's C-linear core: m_{r,p} = sum_{i,j} conj(K[z+i*S+j]) * grid_p(x0+j, y0+i). */
void or_degrid(int64_t n, const int32_t* chan, const int32_t* x0, const int32_t* y0,
               const int64_t* z, const int32_t* S, int32_t P, int32_t N,
               const double* table, const double* grid, double* m)
{
    for (int64_t r = 0; r < n; ++r) {
        const int32_t s = S[r];
        const double* k = table + 2 * z[r];
        const double* g0 = grid + 2 * ((int64_t)chan[r] * N * N * P);
        for (int32_t p = 0; p < P; ++p) {
            double ar = 0.0, ai = 0.0;
            for (int32_t i = 0; i < s; ++i) {
                for (int32_t j = 0; j < s; ++j) {
                    const double kr = k[2 * (i * s + j)];
                    const double ki = k[2 * (i * s + j) + 1];
                    const int64_t pix = ((int64_t)(y0[r] + i) * N + (x0[r] + j)) * P + p;
                    const double gr = g0[2 * pix], gi = g0[2 * pix + 1];
                    ar += kr * gr + ki * gi;   /* conj(k) * g */
                    ai += kr * gi - ki * gr;
                }
            }
            m[2 * (r * P + p)] = ar;
            m[2 * (r * P + p) + 1] = ai;
        }
    }
}

/*
 * Compression (Sec. 4.3.3 "Compression", eq. "ci"; Algorithms "compressindex" and the
 * "Compress and Weigh Visibilities" operator, eqs. "compress1"/"conjugatetake").
 *
 * cross_swap (full-Stokes gridding): a conjugated quad-pol record also swaps its cross hands,
 * since conj(V_XY(u)) is V_YX(-u); the thesis conjugates each polarisation in place, which is
 * exact for the parallel hands and for U = (XY + YX)/2 but flips the sign of V's contribution.
 *
 * Records are visited per channel in row order (row = baseline-major, time-minor), or,
 * with channel interleaving (the thesis's multi-frequency synthesis onto one grid, Sec. 5.4
 * batch 1), as one sequence in natural record order i = row*C + chan.  Record i is
 * compressed into its predecessor (same channel, previous row; interleaved: record i-1)
 * when both are griddable and they share the footprint origin (x0,y0) and the kernel
 * pointer z.  A record that is griddable and not compressed starts a new gridded
 * entry.  For each gridded entry the weighted, flagged, psi-conjugated visibilities
 * of the whole run are summed.
 *
 * Inputs are per record i = row*C + chan.  Outputs:
 *   g[i], c[i]          gridding / compression indicators (uint8)
 *   head_of[i]          index (into the output list) of the entry a record feeds, or -1
 *   list_rec[e]         record index of entry e (the "Gridding Index" g^d)
 *   list_last[e]        last record of the run (the "Last Compressed Entry Index")
 *   gamma[e][P][2]      summed visibilities
 * Entries are ordered channel-major, then row (interleaved: by record).  Returns the number
 * of entries.
 */
int64_t or_compress(int64_t rows, int32_t C, int32_t P, int32_t interleave, int32_t cross_swap,
                    const uint8_t* griddable,
                    const int32_t* x0, const int32_t* y0, const int64_t* z, const int8_t* psi,
                    const float* vis /* [rows][C][P][2] */, const float* weight, const uint8_t* flag,
                    uint8_t* g, uint8_t* c, int64_t* head_of, int64_t* list_rec, int64_t* list_last,
                    double* gamma)
{
    int64_t ne = 0;
    const int32_t n_seq = interleave ? 1 : C;              /* sequences: channels, or one */
    const int64_t len = interleave ? rows * C : rows;       /* records per sequence */
    for (int32_t ch = 0; ch < n_seq; ++ch) {
        int64_t cur = -1;
        for (int64_t s = 0; s < len; ++s) {
            const int64_t i = interleave ? s : s * C + ch;
            const int64_t ip = interleave ? i - 1 : i - C;  /* predecessor in the sequence */
            g[i] = 0;
            c[i] = 0;
            head_of[i] = -1;
            if (!griddable[i]) { cur = -1; continue; }
            int comp = 0;
            if (s > 0 && griddable[ip] && x0[i] == x0[ip] && y0[i] == y0[ip] && z[i] == z[ip])
                comp = 1;
            if (comp) {
                c[i] = 1;
            } else {
                g[i] = 1;
                cur = ne++;
                list_rec[cur] = i;
                for (int32_t p = 0; p < P; ++p) {
                    gamma[2 * (cur * P + p)] = 0.0;
                    gamma[2 * (cur * P + p) + 1] = 0.0;
                }
            }
            head_of[i] = cur;
            list_last[cur] = i;
            for (int32_t p = 0; p < P; ++p) {
                /* with cross_swap, a conjugated quad-pol record feeds pol 1 from pol 2 and pol 2
                   from pol 1: the conjugate of one cross hand is the other at -u */
                const int32_t ps = (cross_swap && psi[i] < 0 && P == 4 && (p == 1 || p == 2)) ? 3 - p : p;
                const int64_t e = i * P + ps;
                const double wf = (1.0 - (double)flag[e]) * (double)weight[e];
                gamma[2 * (cur * P + p)] += wf * (double)vis[2 * e];
                gamma[2 * (cur * P + p) + 1] += (double)psi[i] * wf * (double)vis[2 * e + 1];
            }
        }
    }
    return ne;
}
