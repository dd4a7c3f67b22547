/*
 * wgrid.h -- C ABI of the GB300 w-projection gridder/degridder with compression.
 *
 * Operation: convolutional gridding with w-projection (thesis Sec. 2.1-2.2, eqs.
 * "convgrid", "C_W") as restated for the WImager algorithm (Sec. 4.3.2, eq. "gridding"),
 * with the thesis's compression of consecutive records (Sec. 4.3.3, eq. "compression"),
 * the convolution-function generator (Sec. 4.2, Algorithm "convgen") and the image
 * finaliser (Sec. 4.7, Algorithm "finalizer").  Degridding, the exact adjoint of
 * gridding, is not in the thesis.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: WG_OK (0) or a negative WG_E_* code.  No C++
 *     exception crosses this boundary.  wg_last_error() returns a thread-local message
 *     describing the most recent failure on the calling thread.
 *   - Pointers documented "device" must point to CUDA device memory of the current device;
 *     they are owned by the caller and must stay valid until the stream work that uses
 *     them has completed.  Opaque handles (wg_grid, wg_table, wg_worklist) are owned by the
 *     library and released by the matching *_destroy function.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Every
 *     call that takes a stream only enqueues work on it and returns without synchronising,
 *     except where a comment says "synchronises".
 *   - Record layout: a record is one (row, channel) pair with n_pol polarisations.  Rows are
 *     expected grouped by baseline and sorted by time (Sec. 4.3: compression and the
 *     gridder's register accumulation rely on it; any order is still correct).
 *   - Grid layout: complex64 (float re, float im) [n_chan][N][N][n_pol]; pixel (y, x) holds
 *     n_pol polarisations; (0,0) is the most negative (u, v); u = v = 0 at index N/2
 *     (Sec. 4.3.3).  One grid per channel (Sec. 4.1: channels are imaged independently).
 *   - Coordinates decide placement in FP64 exactly as stated at vis_compress(); the
 *     accumulation is FP32.
 */
#ifndef WGRID_H
#define WGRID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define WG_OK 0
#define WG_E_INVALID_ARG (-1) /* null pointer, bad enum, inconsistent sizes            */
#define WG_E_SHAPE (-2)       /* grid / table / input dimensions do not match          */
#define WG_E_OOB_SUPPORT (-3) /* support larger than the grid or the implementation    */
#define WG_E_CUDA (-4)        /* a CUDA runtime or cuFFT call failed                   */
#define WG_E_OOM (-5)         /* device allocation failed                              */
#define WG_E_CAPACITY (-6)    /* input larger than the worklist was created for        */

/* kernel-table storage read by the gridder (the complex float32 table is always kept too,
 * for degridding and inspection) */
#define WG_F32 0  /* complex float32, 8 bytes per sample                            */
#define WG_BF16 1 /* complex bfloat16, 4 bytes per sample (round to nearest even)    */
#define WG_F16 2  /* complex float16, 4 bytes per sample (round to nearest even)     */

/* visibility element types (wg_vis_in.vis_dtype) */
#define WG_VIS_COMPLEX64 0   /* float re, float im                                      */
#define WG_VIS_COMPLEX_HALF 1 /* float16 re, float16 im; value = vis_scale[chan] x (re, im) */

/* grid flags (wg_grid_desc.flags) */
#define WG_GRID_COMPENSATED 1 /* flushes recover each atomic add's rounding error     */
                              /* (TwoSum) into an error grid folded back after every  */
                              /* grid_vis: an FP32 grid with compensated summation    */

/* support modes of conv_table_build */
#define WG_SUPPORT_THRESHOLD 0  /* outermost sample with |C| > threshold (Sec. 4.2.3) */
#define WG_TABLE_WSTACK 256      /* OR-ed into support_mode: w-stacking table (Sec. 2.2.2,  */
                                 /* eq. "stacking"): every plane holds the w = 0 kernel,   */
                                 /* the planes and their w_k are the w-projection ones     */
#define WG_SUPPORT_PRESCRIBED 1 /* trim or zero-pad to given supports ("normal" mode,
                                   Sec. 4.2.1), one odd support per w-plane          */

/* degrid_vis modes */
#define WG_DEGRID_PREDICT 0 /* model visibilities: psi-conjugated kernel sums          */
#define WG_DEGRID_ADJOINT 1 /* exact adjoint of the vis -> grid map (also eps (1-f))   */

/* vis_compress flags (bit set) */
#define WG_PREP_COMPRESS 1   /* compress consecutive records (Sec. 4.3.3)                */
#define WG_PREP_UNWEIGHTED 2 /* gamma and N_p use weight 1 and ignore per-pol flags; the */
                             /* griddable records are unchanged (all-flagged ones stay   */
                             /* excluded): gridding is then the adjoint of PREDICT-mode  */
                             /* degridding                                               */
#define WG_PREP_CROSS_SWAP 8 /* full-Stokes gridding (n_pol = 4): a take-conjugate record */
                             /* (psi = -1) also swaps its cross hands, pol 1 <-> pol 2,  */
                             /* since conj(V_XY(u)) = V_YX(-u); the thesis conjugates in */
                             /* place (eq. "conjugatetake"), exact for the parallel      */
                             /* hands and U but not for V.  N_p and degridding follow.   */
#define WG_PREP_WSTACK 16    /* w-stacking (Sec. 2.2.2, eq. "stacking"; needs a table    */
                             /* built with WG_TABLE_WSTACK): record (r, c) in plane k    */
                             /* grids onto grid channel c * K + k of a grid with n_chan  */
                             /* x K channels; N_p of channel c is kept in grid channel   */
                             /* c * K (the other planes' N_p stay 0); not combined with  */
                             /* WG_PREP_INTERLEAVE                                       */
#define WG_PREP_INTERLEAVE 4 /* channel interleaving (Sec. 5.4, batch 1): the records of */
                             /* all channels, in natural order row * n_chan + chan, grid */
                             /* onto a one-channel grid (multi-frequency synthesis), and */
                             /* a record compresses into the previous record in that     */
                             /* order; the work list is created with the vis channels    */
#define WG_PREP_APPEND 32    /* batching (Sec. 5.4: many channels in one gridder launch): */
                             /* the batch's entries are added after those of the earlier */
                             /* appended batches (since worklist_clear) and grid onto    */
                             /* grid channels chan0 .. chan0 + n_chan - 1; its N_p terms */
                             /* and statistics go into the grid at this call, and one    */
                             /* grid_vis then grids every appended batch.  Not combined  */
                             /* with WG_PREP_INTERLEAVE or WG_PREP_WSTACK                */

/* grid_correct modes */
#define WG_IMAGE_PER_POL 0 /* output float [n_chan][n_pol][N][N]                      */
#define WG_IMAGE_STOKES_I 1 /* output float [n_chan][N][N]: mean of pols 0 and P-1     */
#define WG_IMAGE_STOKES_LINEAR 4   /* float [n_chan][S][N][N], feeds XX XY YX YY: S = 4:    */
                                   /* I = (XX+YY)/2, Q = (XX-YY)/2, U = (XY+YX)/2,          */
                                   /* V = -j(XY-YX)/2; n_pol 2 (XX YY): I, Q; n_pol 1: I    */
#define WG_IMAGE_WSTACK 6   /* w-stacking finaliser: float [n_chan / K][P][N][N]; for each */
                            /* input channel c, sum over planes k of the inverse FFT of   */
                            /* grid channel c*K + k times exp(+j2pi w_k (n-1)) (zero where */
                            /* l^2 + m^2 >= 1), real part, / N_p, / taper, / sinc        */
#define WG_IMAGE_STOKES_CIRCULAR 5 /* feeds RR RL LR LL: I = (RR+LL)/2, Q = (RL+LR)/2,      */
                                   /* U = -j(RL-LR)/2, V = (RR-LL)/2; n_pol 2 (RR LL): I, V */
                                   /* (Algorithm "finalizer" step 2; each polarisation's   */
                                   /* complex image divided by its own N_p, real part kept) */
#define WG_IMAGE_PER_POL_RAW 2 /* as PER_POL without the division by N_p               */
#define WG_IMAGE_TRANSPOSE 3 /* reads image_out (float [n_chan][n_pol][N][N]) and      */
                             /* OVERWRITES the grid with the exact transpose of mode 2:  */
                             /* grid = (-1)^(x+y) FFT((-1)^(mx+my) img / (taper sinc)),  */
                             /* the sky-to-grid half of the forward model               */

/* Thread-local description of the last failure on this thread ("" if none). */
const char* wg_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far (all devices).
 * Library FFT kernels (cuFFT) are not counted.  A measurement aid; not in the thesis. */
uint64_t wg_launch_count(void);

/* Allocation-failure fake for host-side failure tests (the thesis has no counterpart).
 * after >= 0 arms it: the device allocations of grid_create and worklist_create succeed
 * `after` more times, then the next one and every later one fail as an out-of-memory
 * cudaMalloc would, without calling the CUDA runtime, so the failing call returns WG_E_OOM
 * after freeing what it had allocated.  after < 0 disarms it (the default).  Process-wide;
 * meant for tests, not for use alongside other work.  Always returns WG_OK. */
int wg_debug_fail_allocations(int64_t after);

/* ---- grid (output O-1 and O-2 of Sec. 4.3.2) --------------------------------------- */
typedef struct wg_grid wg_grid;

typedef struct wg_grid_desc {
    int32_t n;      /* grid side N, even, 8 <= N <= 32768                                */
    int32_t n_pol;  /* polarisations per pixel: 1, 2 or 4                                */
    int32_t n_chan; /* channels (independent grids), >= 1                                */
    int32_t flags;  /* 0 or WG_GRID_COMPENSATED (allocates an error grid of the same size)  */
    double du;      /* cell size Delta u = Delta v in wavelengths, > 0                    */
    void* data;     /* optional caller-owned device buffer of n_chan*N*N*n_pol complex64 */
                    /* (8-byte aligned); NULL: the library allocates and owns it          */
} wg_grid_desc;

/* Creates a grid and its FP64 normaliser accumulators N_p [n_chan][n_pol] (eq.
 * "normalizer"), both zeroed.  Synchronises the device.  Errors: INVALID_ARG, OOM, CUDA. */
int grid_create(const wg_grid_desc* desc, wg_grid** out);
/* Frees the grid's library-owned device memory (O-1 and O-2 of Sec. 4.3.2; never a caller's
 * external buffer) and the handle.  NULL is accepted.  Synchronises the device (cudaFree).  Returns WG_OK. */
int grid_destroy(wg_grid* grid);
/* Zeroes the grid O-1, the normaliser O-2 (Sec. 4.3.2) and the statistics counters on
 * `stream`.  Errors: INVALID_ARG, CUDA. */
int grid_zero(wg_grid* grid, void* stream);
/* Device pointers of the grid data O-1 (complex64, layout above) and of N_p, O-2 (double
 * [n_chan][n_pol]; Sec. 4.3.2), owned by the grid.  Either output may be NULL.
 * Errors: INVALID_ARG. */
int grid_device_ptrs(const wg_grid* grid, void** data, double** normaliser);

/* ---- convolution functions (inputs C-1, C-2, C-3 of Sec. 4.2.2) -------------------- */
typedef struct wg_table wg_table;

typedef struct wg_table_desc {
    int32_t n_wplanes;     /* K >= 1; plane k has w_k = w_max (k/(K-1))^2 (sqrt-w spacing) */
    int32_t oversample;    /* beta, 1 <= beta <= 64                                       */
    int32_t taper_support; /* S0: the prolate spheroidal taper has bandwidth c = pi S0 / 2 */
    int32_t n_k;           /* image-plane patch side N_k (even, >= 8); 0 = max(64, next    */
                           /* power of two >= 2 * largest support) or 256 (threshold mode) */
    int32_t support_mode;  /* WG_SUPPORT_THRESHOLD or WG_SUPPORT_PRESCRIBED, | WG_TABLE_WSTACK*/
    int32_t store_dtype;   /* WG_F32, WG_BF16 or WG_F16: samples the gridder reads        */
    double w_max;          /* largest |w| in wavelengths (> 0 if K > 1)                    */
    double du;             /* cell size in wavelengths; must equal the grid's              */
    double threshold;      /* support threshold on |C| (thesis: 1e-3)                      */
    const int32_t* supports; /* host [K] odd supports for WG_SUPPORT_PRESCRIBED, else NULL */
} wg_table_desc;

/* Algorithm "convgen" on the GPU: per plane, sample taper(l) taper(m) exp(+j2pi w (n-1))
 * on an N_k x N_k patch covering the field of view, zero-pad to beta N_k, FFT (cuFFT,
 * FP64), normalise by C_0(0,0), find or apply the support, trim into beta^2 sub-kernels
 * of S x S row-major samples ordered (dv, du) (C-1), plane supports and offsets (C-2),
 * and zeta = sum of the real parts of each sub-kernel (C-3, FP64).
 * Synchronises `stream` (supports are read back, as in the thesis).
 * Errors: INVALID_ARG (even or non-positive support, beta or K out of range),
 *         OOB_SUPPORT (support > 1023), OOM, CUDA. */
int conv_table_build(const wg_table_desc* desc, wg_table** out, void* stream);

/* Builds a table from caller-provided host data in the same layout as C-1/C-2/C-3 (Sec.
 * 4.2.2), for kernels made elsewhere:
 * data = complex double [sum_k beta^2 S_k^2] (interleaved re, im), supports [K] (odd),
 * zeta [K beta^2].  Stored as complex float32.  Synchronises the device. */
int conv_table_import(int32_t n_wplanes, int32_t oversample, double w_max, double du,
                      int32_t taper_support, const int32_t* supports, const double* data,
                      const double* zeta, wg_table** out);
/* Frees the table's device memory (C-1 .. C-3 of Sec. 4.2.2 and their reduced-precision copy)
 * and the handle.  NULL is accepted.  Synchronises the device (cudaFree).  Returns WG_OK. */
int table_destroy(wg_table* table);

/* Sets the storage the gridder reads (WG_F32, WG_BF16, WG_F16), converting the float32 samples
 * with round-to-nearest-even (a precision variant; the thesis stores float32).  Synchronises the device.  Errors: INVALID_ARG, OOM, CUDA. */
int table_set_store(wg_table* table, int32_t store_dtype);

typedef struct wg_table_info {
    int32_t n_wplanes, oversample, taper_support, max_support;
    int64_t n_samples;        /* total complex samples in C-1                         */
    double w_max, du;
    const void* data;         /* device complex float32 [n_samples]                   */
    const double* zeta;       /* device double [K beta^2]                              */
    const int32_t* supports;  /* device int32 [K]                                      */
    const int32_t* offsets;   /* device int32 [K] first sample of each plane           */
    int32_t store_dtype;      /* storage read by the gridder                           */
    int32_t reserved;
    const void* data_lp;      /* device complex bf16/f16 [n_samples], or NULL for WG_F32 */
} wg_table_info;
/* Sizes and device pointers (owned by the table) of C-1 .. C-3 (Sec. 4.2.2).
 * Errors: INVALID_ARG. */
int table_info(const wg_table* table, wg_table_info* info);
/* Copies C-1 (complex float32, interleaved), C-3 and C-2 (Sec. 4.2.2) to caller-owned host
 * buffers sized from table_info; any pointer may be NULL.  Synchronises the device.
 * Errors: INVALID_ARG, CUDA. */
int table_copy_to_host(const wg_table* table, float* data, double* zeta, int32_t* supports,
                       int32_t* offsets);

/* ---- visibility input (inputs I-1 .. I-5 of Sec. 4.3.2) ----------------------------- */
typedef struct wg_vis_in {
    int64_t n_rows;         /* rows (baseline-major, time-minor)                          */
    int32_t n_chan;         /* must equal the grid's                                       */
    int32_t n_pol;          /* must equal the grid's                                       */
    const double* uvw;      /* device [n_rows][3] baseline in metres (I-1)                */
    const double* freq_hz;  /* device [n_chan] channel frequencies (I-2: lambda^-1 = f/c) */
    const void* vis;        /* device [n_rows][n_chan][n_pol] visibilities (I-5), type per */
                            /* vis_dtype (4-byte aligned for half, 8-byte for complex64)   */
    const float* weight;    /* device [n_rows][n_chan][n_pol] natural weights (I-3)       */
    const uint8_t* flag;    /* device [n_rows][n_chan][n_pol], 1 = flagged (I-4)          */
    int32_t vis_dtype;      /* WG_VIS_COMPLEX64 (vis is complex64) or WG_VIS_COMPLEX_HALF */
    int32_t chan0;          /* with WG_PREP_APPEND: the grid channel of the batch's first  */
                            /* channel (chan0 + n_chan <= the grid's channels); else 0     */
    const float* vis_scale; /* device [n_chan] scales for WG_VIS_COMPLEX_HALF, else NULL  */
} wg_vis_in;

/* ---- work list: the preparation phase's outputs (Sec. 4.3.4) ----------------------- */
typedef struct wg_worklist wg_worklist;

/* Allocates device buffers for up to max_records = n_rows * n_chan records: about
 * 41 + 16 n_pol bytes per record (placement, entries, weighted visibilities, runs and the
 * degridder's per-entry sums).  Errors: INVALID_ARG, OOM. */
int worklist_create(int64_t max_records, int32_t n_chan, int32_t n_pol, wg_worklist** out);
/* As worklist_create, with room for max_entries gridded entries over the batches appended with
 * WG_PREP_APPEND (Sec. 5.4, batching) and max_records records per batch: 17 bytes per record
 * (placement and class) plus 24 + 8 n_pol bytes per entry (entry, weighted visibilities, run).
 * It has no degridding accumulator, so degrid_vis rejects it.  max_entries <= 2^31 - 1.
 * Entries past max_entries are not written and are counted in wg_stats.dropped.
 * Errors: INVALID_ARG, OOM. */
int worklist_create2(int64_t max_records, int64_t max_entries, int32_t n_chan, int32_t n_pol,
                     wg_worklist** out);
/* Empties the work list for a new sequence of WG_PREP_APPEND batches (Sec. 5.4, batching):
 * no entries, statistics zero.  Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
int worklist_clear(wg_worklist* wl, void* stream);
/* Frees the work list's device buffers (the preparation outputs of Sec. 4.3.4) and the handle.  NULL is accepted.  Synchronises the
 * device (cudaFree).  Returns WG_OK. */
int worklist_destroy(wg_worklist* wl);

typedef struct wg_stats {
    int64_t records;         /* records presented                                         */
    int64_t griddable;       /* records with g + c = 1                                    */
    int64_t gridded;         /* sum g (Sec. 4.3.4)                                        */
    int64_t compressed;      /* sum c                                                     */
    int64_t updates;         /* sum g S^2 * n_pol: grid-point updates done by the gridder */
    int64_t updates_saved;   /* sum c S^2 * n_pol: updates saved by compression           */
    int64_t tasks;           /* gridder work items                                        */
    int64_t dropped;         /* entries rejected by device-side bounds checks (always 0;  */
                             /* nonzero means an internal error, the entries were skipped)*/
} wg_stats;

/* Preparation phase (Sec. 4.3.4) for one batch, on `stream`:
 *   A1 placement, per record (row r, channel c), FP64, each operation rounded once:
 *      lam_inv = f_c / 299792458;  sc = lam_inv * (beta / du)
 *      tu = u' sc, tv = v' sc, w = w' lam_inv;  if w' < 0: negate all three, psi = -1
 *      q = ceil(t - 0.5);  x_c = ceil((q - beta/2) / beta) (integer);  frac = q - beta x_c
 *      x = N/2 + x_c;  k = the nearest plane in sqrt(w) (Sec. 2.2.1), decided without a
 *      square root: k = the number of m in 1..K-1 with w >= b_m, where b_m = w_max t_m^2 and
 *      t_m = (m - 1/2)/(K-1) (each product rounded once), so ties go to the upper plane and
 *      w >= b_K is beyond the last plane (k = 0 if K = 1)
 *      footprint origin (x - (S_k-1)/2, y - (S_k-1)/2); kernel pointer
 *      z = offset_k + ((frac_v - lo) beta + (frac_u - lo)) S_k^2, lo = -((beta-1)/2)
 *      griddable: k <= K-1, footprint inside the grid, some polarisation unflagged;
 *   A2 compression (if flags & WG_PREP_COMPRESS): record (r, c) is compressed into (r-1, c)
 *      (with WG_PREP_INTERLEAVE: into the previous record r * n_chan + c - 1) when both are
 *      griddable with equal footprint origin and z (eq. "ci");
 *   A3 compaction of gridded records into channel-major lists (interleaved: one list in record
 *      order), segmented into tasks;
 *   A4 gamma = sum over each run of eps (1-f) psi-conj(vis) (eqs. "compress1",
 *      "conjugatetake"), FP32 (eps (1-f) = 1 with WG_PREP_UNWEIGHTED);
 *   A5 the normaliser terms (eps (1-f) zeta, summed per run) and statistics, added into the
 *      grid's N_p and counters when grid_vis runs.
 * `grid` supplies N and du; `table` the planes, supports and zeta.  The work list keeps
 * the results until the next call on it.
 * With WG_PREP_INTERLEAVE the grid must have one channel (SHAPE otherwise) and the work list's
 * runs hold record indices instead of rows.
 * Errors: INVALID_ARG, SHAPE (n_chan/n_pol/du mismatch), CAPACITY (also when n_chan x
 * (16 n_pol + 1) bytes exceed the 227 KB preparation tile, e.g. more than 3575 channels at
 * n_pol = 4), CUDA. */
int vis_compress(const wg_grid* grid, const wg_table* table, const wg_vis_in* in,
                 int32_t flags, wg_worklist* wl, void* stream);

/* Copies the work list's statistics (Sec. 4.3.4) to *out.  Synchronises `stream`. */
int worklist_stats(const wg_worklist* wl, wg_stats* out, void* stream);

/* Device views (owned by the work list) of the gridded-record list of Algorithms "index" and
 * "compressindex" (Sec. 4.3.3), for inspection and tests.  entries: int32 [n][4] with
 * {x0 | y0 << 16, (-x0 mod S) | (-y0 mod S) << 16, z, k | chan << 16}; gamma: complex64
 * [n][n_pol]; runs: int32 [n][2] first and last row of each gridded run (first and last
 * record when interleaved); rec_class: uint8
 * per input record, bit0 = g, bit1 = c, bit2 = griddable, bit3 = take-conjugate (w' < 0).  *n_entries is read from the
 * device (synchronises `stream`). */
int worklist_view(const wg_worklist* wl, const int32_t** entries, const void** gamma,
                  const int32_t** runs, const uint8_t** rec_class, int64_t* n_entries,
                  void* stream);

/* A6: adds every gridded record's gamma_p * C_k[i][j] to grid pixel (y0+i, x0+j) (eq.
 * "gridding"), FP32 accumulation, and adds the batch's normaliser terms and statistics
 * into the grid.  Persistent kernel over the work list's tasks.  A work list holding
 * WG_PREP_APPEND batches is gridded in one launch over every appended batch (planned here if
 * entries were appended since the last plan); their normaliser terms and statistics were
 * added by vis_compress, and the grid must have the channels they name.  Errors: SHAPE, CUDA. */
int grid_vis(wg_grid* grid, const wg_table* table, const wg_worklist* wl, void* stream);

/* ---- gridder plan (not in the thesis: GPU work decomposition) ----------------------
 * grid_vis cuts the work list's gridded entries into segments of seg_len consecutive entries
 * and each segment's footprint (of its largest support S) into ceil(S^2 / slots) tasks; a
 * warp runs one task at a time with R points per lane.  By default R = ceil(S^2 / (32 x
 * tasks)) per support; with WG_PLAN_FIXED_R, R = slots / 32 for every support (no per-point
 * checks; the last task of a small support then has idle points).  FIXED_R takes effect for
 * slots 128 and 256 on FP32 tables without compensation; elsewhere the per-support R runs.
 * vis_compress plans with the work list's current plan (initially WG_PLAN_SEG_LEN_DEFAULT,
 * WG_PLAN_SLOTS_DEFAULT, no flags).  The plan changes only the order of the FP32 additions,
 * not what is added. */
#define WG_PLAN_SEG_LEN_MIN 32
#define WG_PLAN_SEG_LEN_MAX 256
#define WG_PLAN_SEG_LEN_DEFAULT 128
#define WG_PLAN_SLOTS_MIN 64
#define WG_PLAN_SLOTS_MAX 256
#define WG_PLAN_SLOTS_DEFAULT 256
#define WG_PLAN_FIXED_R 1

typedef struct wg_plan {
    int32_t seg_len;        /* gridded entries per segment: a multiple of 32 in [MIN, MAX] */
    int32_t slots;          /* footprint points per task: a multiple of 32 in [MIN, MAX]   */
    int32_t flags;          /* 0 or WG_PLAN_FIXED_R                                          */
    int32_t reserved;       /* 0                                                              */
} wg_plan;

/* Sets the work list's plan and re-plans the batch last prepared on it (no repeat of the
 * preparation).  `table` must be the one given to vis_compress.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, CUDA. */
int worklist_plan(wg_worklist* wl, const wg_table* table, const wg_plan* plan, void* stream);

/* The work list's current plan (not in the thesis).  Errors: INVALID_ARG. */
int worklist_get_plan(const wg_worklist* wl, wg_plan* plan);

/* Autotuner (not in the thesis; it picks the GPU work decomposition of the gridding phase,
 * Sec. 4.3.3).  Times grid_vis on the batch prepared on `wl` under each of the n_candidates plans (NULL or
 * 0: seg_len {64, 128, 256} x slots {128, 256} x flags {0, WG_PLAN_FIXED_R}), `repeats`
 * timed launches each after one warm-up launch (CUDA events on `stream`), keeps the fastest
 * plan in `wl` and copies it to *best (may be NULL), writes its mean milliseconds per launch
 * to *best_ms (may be NULL), and then zeroes the grid (grid_zero: data, normaliser and
 * statistics).  Synchronises `stream`; not to be captured in a CUDA graph.
 * Errors: INVALID_ARG, SHAPE, CUDA. */
int grid_autotune(wg_grid* grid, const wg_table* table, wg_worklist* wl, const wg_plan* candidates,
                  int32_t n_candidates, int32_t repeats, wg_plan* best, float* best_ms, void* stream);

/* ---- uniform and robust weighting ------------------------------------------------------
 * The thesis names the weighting schemes (Sec. 2.1, "Deconvolution and weighting schemes")
 * and grids with natural weights only; these follow the published definitions. */
#define WG_WEIGHT_UNIFORM 1  /* eps' = eps / W(cell)                                       */
#define WG_WEIGHT_ROBUST 2   /* eps' = eps / (1 + W(cell) f^2), Briggs robustness R         */

/* Writes new weights for the batch: W_p(cell) is the sum of eps_p (1 - f_p) over the griddable
 * records (placed as vis_compress places them) in each grid cell (x, y) and polarisation, per
 * grid channel (one grid with WG_PREP_INTERLEAVE in flags, the only flag read); uniform:
 * eps'_p = eps_p / W_p (0 where W_p = 0); robust: eps'_p = eps_p / (1 + W_p f_p^2) with
 * f_p^2 = (5 10^-robust)^2 sum eps_p (1 - f_p) / sum_cells W_p^2.  Records that are not
 * griddable keep eps.  weight_out: device float [n_rows][n_chan][n_pol], may alias in->weight.
 * Allocates and frees a float density grid of (grid channels) x N^2 x n_pol on `stream`
 * (stream-ordered).  Errors: INVALID_ARG, SHAPE, OOM, CUDA. */
int vis_weight(const wg_grid* grid, const wg_table* table, const wg_vis_in* in, int32_t scheme,
               double robust, int32_t flags, float* weight_out, void* stream);

/* A7 (not in the thesis): for every input record, m_p = sum_ij conj(C_k[i][j]) grid_p(y0+i,
 * x0+j), conjugated back where psi = -1; WG_DEGRID_ADJOINT also multiplies by eps (1-f).
 * Runs the gridder's tasks under the work list's plan (worklist_plan / grid_autotune): the
 * sums are taken once per gridded entry into the work list's FP32 accumulator, then written
 * to every record of the entry's run.
 * After a vis_compress with WG_PREP_CROSS_SWAP, pols 1 and 2 of a psi = -1 record come from
 * grid pols 2 and 1.  Records that are not griddable get 0.  `in` and `wl` must be the batch given to the
 * last vis_compress on `wl`, which must not hold WG_PREP_APPEND batches (INVALID_ARG).
 * vis_out: device complex64 [n_rows][n_chan][n_pol], overwritten.  Errors: INVALID_ARG, SHAPE,
 * CUDA. */
int degrid_vis(const wg_grid* grid, const wg_table* table, const wg_vis_in* in,
               const wg_worklist* wl, int32_t mode, void* vis_out, void* stream);

/* A9, Algorithm "finalizer": inverse FFT per polarisation (cuFFT, FP32, centred so that
 * image pixel N/2 is l = 0), real part, divide by N_p, by the taper psi_0(c, 2 du l)
 * psi_0(c, 2 du m) and by sinc(pi l du / beta) sinc(pi m du / beta), l = (k - N/2)/(N du).
 * The Stokes modes keep each polarisation's complex image, divide it by its own N_p and
 * combine (step 2); for n_pol = 4 they are exact for V only after a vis_compress with
 * WG_PREP_CROSS_SWAP.  image_out: device float, layout per `mode`.  The grid is not modified, except by
 * WG_IMAGE_TRANSPOSE, which reads image_out and writes the grid (see the mode list).
 * Errors: INVALID_ARG, SHAPE, CUDA. */
int grid_correct(wg_grid* grid, const wg_table* table, int32_t mode, float* image_out,
                 void* stream);

/* ---- allocation-free gridding of small batches ---------------------------------------
 * The thesis has no counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: code recording into a CUDA graph (an allocation breaks the capture), processes
 * whose device memory belongs to another allocator or to a fixed budget, and real-time
 * loops that must stay out of the driver's allocator.  It does what vis_compress followed by
 * grid_vis does, without a work list: its scratch is a fixed 6 MB array inside the library,
 * which every GPU that loads the library holds until the process exits.
 *   - At most WG_NOALLOC_MAX_RECORDS records (n_rows * n_chan) and WG_NOALLOC_MAX_CHAN
 *     channels per call; larger batches return WG_E_CAPACITY (split them into calls).
 *   - The first call on each device looks up the scratch's device address for that device
 *     (with it current) and caches it: make the first call before any stream capture.
 *   - Every call reuses the same scratch and clears what must start at zero itself; calls
 *     whose GPU work overlaps (several streams or host threads at once) race on it, so
 *     serialise them.
 *   - The caller passes the output grid and normaliser as device pointers (layouts as for
 *     grid_create); both are accumulated into.  `table` comes from conv_table_build or
 *     conv_table_import.  Nothing is allocated or freed: no cudaMalloc, no cudaFree.
 *   - Visibilities are complex64 (8-byte aligned) or complex half with scales (4-byte
 *     aligned), as for vis_compress; `compress` is 0 or WG_PREP_COMPRESS.
 * Errors: INVALID_ARG, SHAPE, OOB_SUPPORT, CAPACITY, CUDA. */
#define WG_NOALLOC_MAX_RECORDS 65536
#define WG_NOALLOC_MAX_CHAN 64

typedef struct wg_grid_view {
    int32_t n, n_pol, n_chan, reserved; /* as wg_grid_desc                                */
    double du;                          /* cell size in wavelengths, positive and finite */
    void* data;                         /* device complex64 [n_chan][N][N][n_pol], 16-B aligned */
    double* normaliser;                 /* device double [n_chan][n_pol]                  */
    int64_t* dropped;                   /* optional (NULL: not reported) device int64,    */
                                        /* 8-B aligned: overwritten, stream-ordered, with */
                                        /* the call's count of entries rejected by the    */
                                        /* device-side bounds checks (wg_stats.dropped:   */
                                        /* always 0 unless an internal error occurred)    */
} wg_grid_view;

int grid_vis_noalloc(const wg_grid_view* grid, const wg_table* table, const wg_vis_in* in,
                     int32_t compress, void* stream);

/* ---- roofline ceilings (measurement; not in the thesis) ------------------------------
 * Gridding does 8 flops per update (one complex multiply-add, Sec. 5.4.4) and fetches one
 * 8-byte kernel sample per footprint point and record, shared by the n_pol polarisations, so
 * its ceilings are the FP32 FMA rate and the bandwidth of 8-byte read-only loads.  Each kind
 * times one launch of a microbenchmark kernel over every SM (8 blocks of 256 threads per SM),
 * after a warm-up launch, with CUDA events on the legacy default stream of the current device:
 *   FP32_FMA2: FLOP/s of independent packed FMAs (fma.rn.f32x2, 4 flops each);
 *   FP32_FMA:  FLOP/s of independent scalar FMAs (2 flops each);
 *   FETCH_L1:  bytes/s of warp-wide 8-byte __ldg loads of 256 contiguous bytes at warp-uniform
 *              pseudo-random positions in a 64 KB buffer (L1-resident);
 *   FETCH_L2:  the same in a 32 MB buffer (L2-resident, L1 hit rate about 0);
 *   SHARED:    bytes/s of warp-wide 8-byte shared-memory loads of 256 contiguous bytes.
 * Synchronous: allocates and frees its scratch (at most 32 MB), returns after the timing.
 * value: host double.  Errors: INVALID_ARG, OOM, CUDA. */
#define WG_CEIL_FP32_FMA2 1
#define WG_CEIL_FP32_FMA 2
#define WG_CEIL_FETCH_L1 3
#define WG_CEIL_FETCH_L2 4
#define WG_CEIL_SHARED 5
int ceiling_measure(int32_t kind, double* value);

#ifdef __cplusplus
}
#endif
#endif /* WGRID_H */
