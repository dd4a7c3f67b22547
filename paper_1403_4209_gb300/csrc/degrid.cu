// Degridding: the adjoint of the gridding map (not in the thesis).
//
// For a gridded entry (footprint origin (x0, y0), kernel pointer z, channel c) the kernel sum
//   m_p = sum_{i,j} conj(C[z + i S + j]) grid_c,p(y0 + i, x0 + j)
// is a gather: one warp per entry (chunks of consecutive entries per warp), lanes striding over
// the S x S footprint, a shuffle reduction.  Compression (Sec. 4.3.3) carries over: every record compressed into the entry
// has the same footprint and kernel samples, so m is computed once per run and written to each
// record of the run, conjugated back where psi = -1 (w' < 0), and for the adjoint mode scaled
// by eps (1 - f) (the vis -> grid map's R-linear outer factor).
#include "internal.cuh"

namespace wg {

typedef unsigned long long f32x2;     // a packed FP32 pair (Blackwell f32x2 arithmetic)

__device__ __forceinline__ f32x2 pack2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float2 unpack2(f32x2 v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// the P polarisations of one pixel as packed pairs
template <int P>
__device__ __forceinline__ void load_pixel(const float2* __restrict__ g, f32x2 (&v)[P])
{
    if constexpr (P == 1) {
        v[0] = __ldg(reinterpret_cast<const f32x2*>(g));
    } else {
#pragma unroll
        for (int h = 0; h < P; h += 2) {
            const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(g + h));
            v[h] = a.x;
            v[h + 1] = a.y;
        }
    }
}

constexpr int kDegridChunk = 4;     // consecutive entries a warp takes from the counter at a time

// A warp takes chunks of consecutive entries from a global counter, so that the overlapping
// footprints of consecutive entries of a track are read by the same SM (L1 reuse).  Per entry
// the lanes stride over the S x S footprint and accumulate conj(k) g as the packed pairs
// A = (kx, kx) (gx, gy) and B = (ky, ky) (gx, gy): conj(k) g = (A.x + B.y, A.y - B.x).
template <int P>
__global__ void __launch_bounds__(256, 4) k_degrid(const int4* __restrict__ entries, const int2* __restrict__ runs,
                                                const long long* __restrict__ scal, const int* __restrict__ supports,
                                                const float2* __restrict__ table, const float2* __restrict__ grid,
                                                int N, int C, int kst, const double* __restrict__ uvw,
                                                const float* __restrict__ weight, const uint8_t* __restrict__ flag,
                                                int adjoint, float2* __restrict__ out, int K, int64_t n_samples,
                                                int64_t rows, int interleave, int cross_swap,
                                                unsigned int* __restrict__ counter,
                                                long long* __restrict__ dropped)
{
    const long long n = scal[0];
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned int chunk = 0;
        if (lane == 0) chunk = atomicAdd(counter, 1u);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const long long c0 = (long long)chunk * kDegridChunk;
        if (c0 >= n) break;
        const long long c1 = min(n, c0 + kDegridChunk);
        for (long long e = c0; e < c1; ++e) {
            const int4 E = entries[e];
            const int k = E.w & 0xFFF, gchan = (E.w >> 16) & 0xFFFF;
            const int ch = gchan / kst;                  // input channel (w-stacking: kst planes each)
            if (k >= K || ch >= C) {                 // device-side bounds checks (never taken)
                if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(dropped), 1ull);
                continue;
            }
            const int S = __ldg(&supports[k]);
            const int x0 = E.x & 0xFFFF, y0 = (E.x >> 16) & 0xFFFF, z = E.z;
            const int2 run = runs[e];
            if (x0 + S > N || y0 + S > N || z < 0 || (int64_t)z + (int64_t)S * S > n_samples || run.x < 0 ||
                run.y < run.x || (int64_t)run.y >= (interleave ? rows * C : rows)) {
                if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(dropped), 1ull);
                continue;
            }
            const float2* gch = grid + (size_t)gchan * N * N * P;   // channel 0 when interleaved
            f32x2 A[P], B[P];
#pragma unroll
            for (int p = 0; p < P; ++p) A[p] = B[p] = 0ull;
            const int s2 = S * S;
            int i = lane / S, j = lane - (lane / S) * S;
            const int di = 32 / S, dj = 32 - di * S;
            for (int s = lane; s < s2; s += 32) {
                const float2 kv = __ldg(&table[z + s]);
                const f32x2 kxx = pack2(kv.x, kv.x), kyy = pack2(kv.y, kv.y);
                f32x2 gv[P];
                load_pixel<P>(gch + ((size_t)(y0 + i) * N + x0 + j) * P, gv);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    A[p] = fma2(kxx, gv[p], A[p]);
                    B[p] = fma2(kyy, gv[p], B[p]);
                }
                j += dj;
                i += di;
                if (j >= S) {
                    j -= S;
                    ++i;
                }
            }
            float2 acc[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float2 a = unpack2(A[p]), b = unpack2(B[p]);
                acc[p] = make_float2(a.x + b.y, a.y - b.x);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    acc[p].x += __shfl_xor_sync(0xffffffffu, acc[p].x, o);
                    acc[p].y += __shfl_xor_sync(0xffffffffu, acc[p].y, o);
                }
            }
            // the run's records: rows run.x..run.y of channel ch, or records run.x..run.y
            for (int r = run.x + lane; r <= run.y; r += 32) {
                const int64_t rec = interleave ? (int64_t)r : (int64_t)r * C + ch;
                const int64_t row = interleave ? (int64_t)r / C : (int64_t)r;
                const bool neg = uvw[3 * row + 2] < 0.0;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    // with cross-hand swapping, output pol 1 of a take-conjugate record comes from
                    // grid pol 2 and pol 2 from pol 1 (the adjoint of the swap is the swap)
                    float2 a = acc[p];
                    if constexpr (P == 4) {
                        if (cross_swap && neg && p == 1) a = acc[2];
                        if (cross_swap && neg && p == 2) a = acc[1];
                    }
                    float2 v = neg ? make_float2(a.x, -a.y) : a;
                    if (adjoint) {
                        const float wf = weight[rec * P + p] * (1.0f - (float)flag[rec * P + p]);
                        v.x *= wf;
                        v.y *= wf;
                    }
                    out[rec * P + p] = v;
                }
            }
        }
    }
}

template <int P>
static int degrid_impl(const Grid& g, const Table& t, const wg_vis_in& in, const WorkList& wl, int mode, float2* out,
                       cudaStream_t s)
{
    WG_CUDA(cudaMemsetAsync(out, 0, sizeof(float2) * (size_t)in.n_rows * in.n_chan * P, s));
    WG_CUDA(cudaMemsetAsync(wl.task_counter + 1, 0, sizeof(unsigned int), s));
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_degrid<P>, 256, 0) != cudaSuccess ||
         blocks_per_sm < 1))
        blocks_per_sm = 1;
    const int blocks = num_sms() * blocks_per_sm;
    k_degrid<P><<<blocks, 256, 0, s>>>(wl.entries, wl.runs, wl.scal, t.supports_d, t.data, g.data, g.n, in.n_chan,
                                       wl.wstack_k,
                                       in.uvw, in.weight, in.flag, mode == WG_DEGRID_ADJOINT ? 1 : 0, out, t.K,
                                       t.n_samples, in.n_rows, wl.interleave ? 1 : 0, wl.cross_swap ? 1 : 0,
                                       wl.task_counter + 1,
                                       wl.scal + 3);
    WG_LAUNCHED("k_degrid");
    return WG_OK;
}

int launch_degrid(const Grid& g, const Table& t, const wg_vis_in& in, const WorkList& wl, int mode, float2* out,
                  cudaStream_t s)
{
    switch (g.n_pol) {
        case 1: return degrid_impl<1>(g, t, in, wl, mode, out, s);
        case 2: return degrid_impl<2>(g, t, in, wl, mode, out, s);
        case 4: return degrid_impl<4>(g, t, in, wl, mode, out, s);
        default: return fail(WG_E_INVALID_ARG, "n_pol must be 1, 2 or 4");
    }
}

}  // namespace wg
