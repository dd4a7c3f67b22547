// Gridding phase (thesis Sec. 4.3.3 "The gridding phase", eq. "gridding"), GB300 design.
//
// Work unit ("task") = one segment of kSegLen consecutive gridded entries x one block of up to
// kSlotsPerBlock footprint points.  A warp takes tasks from a global counter (persistent
// kernel, dynamic load balance).  Each lane owns R <= kRMax fixed residue classes
// (x mod S, y mod S) of the footprint, the ownership Romein's algorithm uses (Sec. 2.5): for
// every record exactly one grid pixel of each owned class lies inside the S x S footprint, so
// lanes never touch the same pixel and can accumulate in registers while the pixel stays the
// same; when it moves, the lane flushes its accumulators to the grid with one vector FP32
// atomic per pixel (all polarisations of a pixel are contiguous).  Records are staged per warp
// in shared memory, 32 at a time; kernel samples are read through the read-only cache.  A
// change of support or channel inside a segment flushes and re-maps the lane's classes.
#include "internal.cuh"

namespace wg {

namespace {

template <int P>
__device__ __forceinline__ void flush_pixel(float2* __restrict__ gch, int pix, float2 (&a)[P])
{
    float2* d = gch + (size_t)pix * P;
    if constexpr (P == 1) {
        atomicAdd(d, a[0]);
    } else if constexpr (P == 2) {
        atomicAdd(reinterpret_cast<float4*>(d), make_float4(a[0].x, a[0].y, a[1].x, a[1].y));
    } else {
        atomicAdd(reinterpret_cast<float4*>(d), make_float4(a[0].x, a[0].y, a[1].x, a[1].y));
        atomicAdd(reinterpret_cast<float4*>(d + 2), make_float4(a[2].x, a[2].y, a[3].x, a[3].y));
    }
#pragma unroll
    for (int p = 0; p < P; ++p) a[p] = make_float2(0.f, 0.f);
}

}  // namespace

template <int P>
__global__ void __launch_bounds__(256, 2) k_grid(const int4* __restrict__ entries, const float2* __restrict__ gamma,
                                                 const int* __restrict__ seg_off, const long long* __restrict__ scal,
                                                 const int* __restrict__ supports, const float2* __restrict__ table,
                                                 float2* __restrict__ grid, int N, int K, int C, int64_t n_samples,
                                                 unsigned int* __restrict__ counter, long long* __restrict__ dropped)
{
    constexpr int W = 8;
    __shared__ int4 s_e[W][32];
    __shared__ float2 s_g[W][32 * P];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long n_entries = scal[0], n_tasks = scal[1], n_seg = scal[2];
    const size_t chan_stride = (size_t)N * N * P;

    for (;;) {
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(counter, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((long long)t >= n_tasks) break;
        int lo = 0, hi = (int)n_seg;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&seg_off[mid]) <= (int)t) lo = mid; else hi = mid;
        }
        const int blk = (int)t - __ldg(&seg_off[lo]);
        const int e0 = lo * kSegLen;
        const int e1 = (int)min((long long)e0 + kSegLen, n_entries);

        int curS = -1, curCh = -1;
        bool active = false;
        unsigned valid = 0;
        int pu[kRMax], pv[kRMax], cur[kRMax];
        float2 acc[kRMax][P];
#pragma unroll
        for (int r = 0; r < kRMax; ++r) {
            cur[r] = -1;
            pu[r] = pv[r] = 0;
#pragma unroll
            for (int p = 0; p < P; ++p) acc[r][p] = make_float2(0.f, 0.f);
        }
        float2* gch = grid;

        for (int base = e0; base < e1; base += 32) {
            const int n = min(32, e1 - base);
            __syncwarp();
            if (lane < n) {
                s_e[wid][lane] = entries[base + lane];
#pragma unroll
                for (int p = 0; p < P; ++p) s_g[wid][lane * P + p] = gamma[(size_t)(base + lane) * P + p];
            }
            __syncwarp();
            for (int j = 0; j < n; ++j) {
                const int4 E = s_e[wid][j];
                const int k = E.w & 0xFFF, ch = (E.w >> 16) & 0xFFFF;
                if (k >= K || ch >= C) {          // device-side bounds check (never taken)
                    if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(dropped), 1ull);
                    continue;
                }
                const int S = __ldg(&supports[k]);
                {
                    const int x0c = E.x & 0xFFFF, y0c = (E.x >> 16) & 0xFFFF;
                    if (x0c + S > N || y0c + S > N || E.z < 0 || (int64_t)E.z + (int64_t)S * S > n_samples) {
                        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(dropped), 1ull);
                        continue;
                    }
                }
                if (S != curS || ch != curCh) {
#pragma unroll
                    for (int r = 0; r < kRMax; ++r)
                        if (cur[r] >= 0) {
                            flush_pixel<P>(gch, cur[r], acc[r]);
                            cur[r] = -1;
                        }
                    curS = S;
                    curCh = ch;
                    gch = grid + (size_t)ch * chan_stride;
                    const int s2 = S * S;
                    const int nb = (s2 + kSlotsPerBlock - 1) / kSlotsPerBlock;
                    active = blk < nb;
                    const int R = (s2 + 32 * nb - 1) / (32 * nb);
                    const int sbase = blk * 32 * R;
                    valid = 0;
#pragma unroll
                    for (int r = 0; r < kRMax; ++r) {
                        const int sl = sbase + r * 32 + lane;
                        if (r < R && sl < s2) {
                            valid |= 1u << r;
                            pv[r] = sl / S;
                            pu[r] = sl - pv[r] * S;
                        }
                    }
                }
                if (!active) continue;
                const int x0 = E.x & 0xFFFF, y0 = (E.x >> 16) & 0xFFFF;
                const int cu = E.y & 0xFFFF, cv = (E.y >> 16) & 0xFFFF;
                const int z = E.z;
                float2 gm[P];
#pragma unroll
                for (int p = 0; p < P; ++p) gm[p] = s_g[wid][j * P + p];
#pragma unroll
                for (int r = 0; r < kRMax; ++r) {
                    if (valid & (1u << r)) {
                        int du = pu[r] + cu;
                        du -= (du >= S) ? S : 0;
                        int dv = pv[r] + cv;
                        dv -= (dv >= S) ? S : 0;
                        const int pix = (y0 + dv) * N + x0 + du;
                        const float2 kv = __ldg(&table[z + dv * S + du]);
                        if (pix != cur[r]) {
                            if (cur[r] >= 0) flush_pixel<P>(gch, cur[r], acc[r]);
                            cur[r] = pix;
                        }
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            acc[r][p].x = fmaf(gm[p].x, kv.x, fmaf(-gm[p].y, kv.y, acc[r][p].x));
                            acc[r][p].y = fmaf(gm[p].x, kv.y, fmaf(gm[p].y, kv.x, acc[r][p].y));
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kRMax; ++r)
            if (cur[r] >= 0) flush_pixel<P>(gch, cur[r], acc[r]);
    }
}

// adds the batch normaliser and statistics into the grid's accumulators
__global__ void k_accumulate(double* __restrict__ gnorm, const double* __restrict__ bnorm, int n,
                             unsigned long long* __restrict__ gcnt, const unsigned long long* __restrict__ bcnt)
{
    const int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (i < n) gnorm[i] += bnorm[i];
    if (i < ST_N) gcnt[i] += bcnt[i];
}

template <int P>
static int grid_impl(Grid& g, const Table& t, const WorkList& wl, cudaStream_t s)
{
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_grid<P>, 256, 0) != cudaSuccess ||
            blocks_per_sm < 1)
            blocks_per_sm = 1;
    }
    WG_CUDA(cudaMemsetAsync(wl.task_counter, 0, sizeof(unsigned int), s));
    k_grid<P><<<num_sms() * blocks_per_sm, 256, 0, s>>>(wl.entries, wl.gamma, wl.seg_off, wl.scal, t.supports_d,
                                                         t.data, g.data, g.n, t.K, g.n_chan, t.n_samples,
                                                         wl.task_counter, wl.scal + 3);
    WG_LAUNCHED("k_grid");
    const int n = g.n_chan * g.n_pol;
    const int m = std::max(n, (int)ST_N);
    k_accumulate<<<(m + 255) / 256, 256, 0, s>>>(g.norm, wl.norm_batch, n, g.counters, wl.stats);
    WG_LAUNCHED("k_accumulate");
    return WG_OK;
}

int launch_grid(Grid& g, const Table& t, const WorkList& wl, cudaStream_t s)
{
    switch (g.n_pol) {
        case 1: return grid_impl<1>(g, t, wl, s);
        case 2: return grid_impl<2>(g, t, wl, s);
        case 4: return grid_impl<4>(g, t, wl, s);
        default: return fail(WG_E_INVALID_ARG, "n_pol must be 1, 2 or 4");
    }
}

}  // namespace wg
