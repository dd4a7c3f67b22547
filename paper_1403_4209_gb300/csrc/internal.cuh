// Internal declarations of the wgrid library (handles, error reporting, kernel launchers).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "wgrid.h"

namespace wg {

// ---- errors -------------------------------------------------------------------------
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();   // empties this thread's wg_last_error() message
#define WG_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)
#define WG_LAUNCHED(what)                                       \
    do {                                                        \
        ::wg::count_launch();                                   \
        cudaError_t e_ = cudaGetLastError();                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);      \
    } while (0)

extern std::atomic<uint64_t> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int num_sms();

// ---- compile-time limits --------------------------------------------------------------
constexpr int kMaxSupport = 1023;     // largest odd support
constexpr int kMaxBeta = 64;
constexpr int kTileRecords = 2048;    // records per preparation tile (rows x channels)
constexpr int kSegLenMin = 32;        // gridded entries per gridder segment: range and default
constexpr int kSegLenMax = 256;
constexpr int kSegLenDefault = 128;
constexpr int kSlotsMin = 64;         // footprint points per gridder task: range and default
constexpr int kSlotsMax = 256;        // (32 lanes x kRMax)
constexpr int kSlotsDefault = 256;
static_assert(kSegLenMin == WG_PLAN_SEG_LEN_MIN && kSegLenMax == WG_PLAN_SEG_LEN_MAX &&
                  kSegLenDefault == WG_PLAN_SEG_LEN_DEFAULT && kSlotsMin == WG_PLAN_SLOTS_MIN &&
                  kSlotsMax == WG_PLAN_SLOTS_MAX && kSlotsDefault == WG_PLAN_SLOTS_DEFAULT,
              "plan limits differ from the header's");
constexpr int kRMax = 8;              // points per lane
constexpr int kNormSlots = 256;       // privatised normaliser accumulators

// ---- handles --------------------------------------------------------------------------
struct Grid {
    int n = 0, n_pol = 0, n_chan = 0;
    double du = 0;
    float2* data = nullptr;
    bool owns = false;
    bool comp = false;                    // compensated flushes (WG_GRID_COMPENSATED)
    float2* err = nullptr;                // [n_chan][N][N][P] rounding errors of the flushes
    double* norm = nullptr;               // [n_chan][n_pol]
    unsigned long long* counters = nullptr;  // [8] accumulated statistics
    // grid_correct resources
    float2* scratch = nullptr;            // [G][N][N][P], G = scratch_chans
    int scratch_chans = 0;
    double* corr = nullptr;               // [N] taper x sinc
    float* icorr = nullptr;               // [N] 1 / (taper x sinc)
    float* inv_norm = nullptr;            // [n_chan][n_pol] 1 / N_p (0 where N_p = 0)
    int corr_s0 = -1, corr_beta = -1;
    cufftHandle plan = 0;
    cufftHandle plan_c = 0;               // batch of scratch_chans contiguous N x N planes
    bool plan_c_ok = false;
    bool plan_ok = false;
};

struct Table {
    int K = 0, beta = 0, s0 = 0, max_support = 0;
    double w_max = 0, du = 0;
    int64_t n_samples = 0;
    float2* data = nullptr;               // C-1, complex float32
    int store = WG_F32;                   // samples the gridder reads
    void* data_lp = nullptr;              // C-1 as complex bf16 / f16 (store != WG_F32)
    double* zeta = nullptr;               // C-3 [K beta^2]
    int* supports_d = nullptr;            // C-2 supports [K]
    int* offsets_d = nullptr;             // C-2 offsets [K]
    double* wbounds_d = nullptr;          // [K] squared sqrt(w) midpoints between planes
    float* wbounds_f = nullptr;           // [K] the same rounded to float
    float* zeta_f = nullptr;              // C-3 in FP32 (normaliser terms)
    std::vector<int> supports, offsets;   // host copies
    std::vector<double> pswf;             // Legendre coefficients of psi_0 (even degrees)
    bool stacking = false;                // every plane holds the w = 0 kernel (w-stacking)
    std::vector<double> w_planes;         // w_k of each plane, wavelengths
};

struct WorkList {
    int64_t cap = 0;                      // records of one batch
    int64_t ecap = 0;                     // gridded entries (over the appended batches)
    int C = 0, P = 0;
    int64_t tile_cap = 0;                 // tiles x C counters
    int64_t seg_cap = 0;
    int seg_len = kSegLenDefault;         // gridder plan: entries per segment
    int slots = kSlotsDefault;            // gridder plan: footprint points per task
    bool fixed_r = false;                 // gridder plan: R = slots / 32 for every support
    bool interleave = false;              // last batch: channels interleaved onto one grid
    bool cross_swap = false;              // last batch: take-conjugate records swap cross hands
    int wstack_k = 1;                     // last batch: w-stacking planes (1: no stacking)
    bool append = false;                  // holds batches added with WG_PREP_APPEND
    int chan_hi = 0;                      // appended batches: one past their highest grid channel
    bool plan_stale = false;              // entries were appended since the last plan
    // per record (rinfo: placement, written for gridded records and each tile's first row)
    int4* rinfo = nullptr;
    uint8_t* rclass = nullptr;
    // per (tile, chan)
    int* tile_cnt = nullptr;
    float2* carry_q = nullptr;            // [tile_cap][P] run parts carried into a tile
    int* carry_last = nullptr;            // [tile_cap] their last row (record), or -1
    // per gridded entry (channel-major)
    int4* entries = nullptr;
    float2* gamma = nullptr;
    int2* runs = nullptr;
    float2* dacc = nullptr;               // [cap][P] degridding sums per entry (not in no-alloc views)
    // segments
    int* seg_nblk = nullptr;
    int* seg_off = nullptr;               // [seg_cap + 1]
    // scalars and small arrays (device)
    long long* scal = nullptr;            // [0] n_entries [1] n_tasks [2] n_seg [3] overflow
    int* chan_base = nullptr;             // [C + 1]
    double* norm_priv = nullptr;          // [kNormSlots][C][P]
    double* norm_batch = nullptr;         // [C][P]
    unsigned long long* stat_priv = nullptr;  // [kNormSlots][8]
    unsigned long long* stats = nullptr;  // [8] (summed over appended batches)
    unsigned long long* stats_batch = nullptr;  // [8] the last batch's
    unsigned int* task_counter = nullptr;
    // last batch
    int64_t rows = 0;
    int rpb = 0;
    int64_t n_tiles = 0;
    int N = 0;
};

// statistics slots
enum { ST_RECORDS = 0, ST_GRIDDABLE, ST_GRIDDED, ST_COMPRESSED, ST_UPD, ST_UPD_SAVED, ST_TASKS, ST_N };

// rinfo.w bit layout
constexpr int kBitG = 12, kBitC = 13, kBitNeg = 14, kBitGd = 15;

// ---- launchers (defined in the .cu files) ---------------------------------------------
struct PlaceParams {
    int N, beta, K, lo, compress, unweighted, interleave, cross_swap, wstack, C, P;
    double w_max, beta_over_du;
    const int* supports;
    const int* offsets;
    const double* wbounds;
    const float* wbounds_f;               // wbounds rounded to float (monotone prefilter)
    const float* zeta_f;
    int qlim;                             // beta (N/2 + 2): |q| beyond it is off the grid
    int beta_log2;                        // log2(beta), or -1 when beta is not a power of two
    int flag_vec;                         // the flag array is aligned to n_pol bytes
    float kscale_f;                       // (K - 1) / sqrt(w_max): estimate of the nearest plane
    int chan0;                            // grid channel of the batch's channel 0 (WG_PREP_APPEND)
};

int launch_prep(const Table& t, const Grid& g, const wg_vis_in& in, int flags, WorkList& wl,
                cudaStream_t s);
int launch_grid(Grid& g, const Table& t, const WorkList& wl, cudaStream_t s);
// adds the last batch's normaliser and statistics into grid channels chan0 .. chan0 + C - 1
int launch_accumulate(const Grid& g, const WorkList& wl, int chan0, cudaStream_t s);
int launch_plan(const Table& t, WorkList& wl, cudaStream_t s);
int launch_weight(const Table& t, const Grid& g, const wg_vis_in& in, int scheme, double robust, int flags,
                  float* out, cudaStream_t s);
int launch_degrid(const Grid& g, const Table& t, const wg_vis_in& in, const WorkList& wl, int mode,
                  float2* out, cudaStream_t s);
int launch_correct(Grid& g, const Table& t, int mode, float* image, cudaStream_t s);
int build_table(const wg_table_desc& d, Table& t, cudaStream_t s);
int import_table(int K, int beta, double w_max, double du, int s0, const int* supports,
                 const double* data, const double* zeta, Table& t);
int free_table(Table& t);
int set_table_store(Table& t, int store);

// psi_0(c, x) from its even Legendre coefficients a[0..n): sum_m a_m P_2m(x), by the
// three-term Legendre recurrence.
__device__ __forceinline__ double pswf_eval_dev(const double* a, int n, double x)
{
    double pm1 = 1.0, p = x, s = a[0];
    const int deg = 2 * n - 2;
    for (int j = 1; j < deg; ++j) {
        const double pn = ((2.0 * j + 1) * x * p - j * pm1) / (j + 1);
        pm1 = p;
        p = pn;
        if ((j + 1) % 2 == 0) s += a[(j + 1) / 2] * p;
    }
    return s;
}

// (a / d, a mod d) for 0 <= a < 2^22 and 1 <= d < 2^12, inv_d = 1.0f / d: the truncated float
// quotient is within one of the integer quotient, and one correction step each way makes it
// exact (a few instructions against about twenty for an integer division by a runtime divisor)
__device__ __forceinline__ int2 divmod_small(int a, int d, float inv_d)
{
    int q = __float2int_rz((float)a * inv_d);
    int m = a - q * d;
    if (m < 0) { --q; m += d; }
    if (m >= d) { ++q; m -= d; }
    return make_int2(q, m);
}

// Exclusive scan of a[0..n) in place by the whole block (every thread calls it; blockDim a
// multiple of 32, at most 1024), a[n] = the total; warp_tot is shared scratch of 32 ints.
// Each thread sums a contiguous chunk, the chunk sums are scanned with warp shuffles and
// the warp totals by the first warp, then each thread writes its chunk's prefixes.
__device__ __forceinline__ void block_exclusive_scan(int* a, int n, int* warp_tot)
{
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int ipt = (n + T - 1) / T;
    const int b0 = min(n, t * ipt), b1 = min(n, b0 + ipt);
    int s = 0;
    for (int i = b0; i < b1; ++i) s += a[i];
    int inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int nw = T >> 5;
        int v = (lane < nw) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < nw) warp_tot[lane] = v;   // inclusive
    }
    __syncthreads();
    int run = inc - s + (wid > 0 ? warp_tot[wid - 1] : 0);
    for (int i = b0; i < b1; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    __syncthreads();
    if (t == T - 1) a[n] = run;
    __syncthreads();
}

// prolate spheroidal psi_0(c, x) as even Legendre coefficients (host eigen-solver)
std::vector<double> pswf_coefficients(double c);
double pswf_eval_host(const std::vector<double>& coef, double x);

}  // namespace wg

// opaque C-ABI handles
struct wg_grid { wg::Grid g; };
struct wg_table { wg::Table t; };
struct wg_worklist { wg::WorkList w; };
