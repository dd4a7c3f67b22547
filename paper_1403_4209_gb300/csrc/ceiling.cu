// Ceilings of the gridder's roofline, measured on the device (not in the thesis).  Gridding
// does one complex multiply-add (8 flops) per update and fetches one 8-byte kernel sample per
// footprint point and record, shared by the P polarisations (Sec. 5.4.4 counts the flops), so
// its rate is bounded by the FP32 FMA pipe and by the bandwidth of 8-byte read-only loads.
// These kernels measure both with the gridder's instruction forms: packed fma.rn.f32x2 (and
// scalar FFMA for comparison), and warp-wide 8-byte __ldg loads of 256 contiguous bytes at
// warp-uniform pseudo-random positions in a buffer that stays in L1 (64 KB) or only in L2
// (32 MB), plus 8-byte shared-memory loads.
#include "internal.cuh"

namespace wg {

namespace {

typedef unsigned long long f32x2;

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

constexpr int kThreads = 256;
constexpr int kChains = 8;          // independent accumulators per thread
constexpr int kLoads = 8;           // independent loads in flight per thread

// 4 kChains packed FMAs (4 flops each) per thread and iteration
__global__ void __launch_bounds__(kThreads) k_ceil_fma2(int iters, float seed, float* __restrict__ sink)
{
    f32x2 acc[kChains];
    const float x = seed + 1e-7f * (float)threadIdx.x;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = pack2(x + (float)i, x - (float)i);
    const f32x2 a = pack2(0.9999999f, 0.9999999f), b = pack2(1e-7f, 1e-7f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) acc[i] = fma2(acc[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        const float2 v = unpack2(acc[i]);
        s += v.x + v.y;
    }
    if (s == 1234.5f) sink[0] = s;     // keeps the chains live; practically never true
}

// the same work as scalar FFMAs (2 kChains chains)
__global__ void __launch_bounds__(kThreads) k_ceil_fma(int iters, float seed, float* __restrict__ sink)
{
    float acc[2 * kChains];
    const float x = seed + 1e-7f * (float)threadIdx.x;
#pragma unroll
    for (int i = 0; i < 2 * kChains; ++i) acc[i] = x + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < 2 * kChains; ++i) acc[i] = fmaf(acc[i], 0.9999999f, 1e-7f);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * kChains; ++i) s += acc[i];
    if (s == 1234.5f) sink[0] = s;
}

// each warp reads 32 consecutive 8-byte words (256 B) at a warp-uniform position drawn from a
// linear congruential sequence; n_chunks (a power of two) 256-byte chunks in the buffer
__global__ void __launch_bounds__(kThreads) k_ceil_fetch(const f32x2* __restrict__ buf, unsigned n_chunks, int iters,
                                                         float* __restrict__ sink)
{
    const unsigned lane = threadIdx.x & 31;
    unsigned h = ((blockIdx.x * kThreads + threadIdx.x) >> 5) * 2654435761u + 12345u;
    float sx = 0.f, sy = 0.f;
    for (int it = 0; it < iters; ++it) {
        f32x2 v[kLoads];
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            h = h * 1664525u + 1013904223u;
            const unsigned chunk = (h >> 7) & (n_chunks - 1);
            v[u] = __ldg(buf + (size_t)chunk * 32 + lane);
        }
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const float2 f = unpack2(v[u]);
            sx += f.x;
            sy += f.y;
        }
    }
    if (sx + sy == 1234.5f) sink[0] = sx;
}

constexpr int kSmemWords = 2048;    // 16 KB of 8-byte words per block

__global__ void __launch_bounds__(kThreads) k_ceil_shared(int iters, float* __restrict__ sink)
{
    __shared__ f32x2 sm[kSmemWords];
    for (int i = threadIdx.x; i < kSmemWords; i += kThreads) sm[i] = pack2((float)i, -(float)i);
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned pos = warp * 256u;
    float sx = 0.f, sy = 0.f;
    for (int it = 0; it < iters; ++it) {
        f32x2 v[kLoads];
#pragma unroll
        for (int u = 0; u < kLoads; ++u) v[u] = sm[((pos + 32u * u) & (kSmemWords - 32u)) + lane];
        pos += 32u * kLoads + 96u;     // stays a multiple of 32: each warp reads whole 256-byte rows
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const float2 f = unpack2(v[u]);
            sx += f.x;
            sy += f.y;
        }
    }
    if (sx + sy == 1234.5f) sink[0] = sx;
}

}  // namespace

}  // namespace wg

using namespace wg;

extern "C" int ceiling_measure(int32_t kind, double* value)
{
    if (!value) return fail(WG_E_INVALID_ARG, "ceiling_measure: null argument");
    *value = 0.0;
    if (kind < WG_CEIL_FP32_FMA2 || kind > WG_CEIL_SHARED) return fail(WG_E_INVALID_ARG, "unknown ceiling %d", kind);
    const int blocks = num_sms() * 8;
    const double threads = (double)blocks * kThreads;
    float* sink = nullptr;
    f32x2* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = WG_OK;
    auto run = [&]() -> int {
        WG_CUDA(cudaMalloc(&sink, sizeof(float)));
        WG_CUDA(cudaEventCreate(&e0));
        WG_CUDA(cudaEventCreate(&e1));
        unsigned n_chunks = 0;
        if (kind == WG_CEIL_FETCH_L1 || kind == WG_CEIL_FETCH_L2) {
            n_chunks = kind == WG_CEIL_FETCH_L1 ? 256u : 131072u;          // 64 KB or 32 MB
            WG_CUDA(cudaMalloc(&buf, (size_t)n_chunks * 256));
            WG_CUDA(cudaMemset(buf, 0, (size_t)n_chunks * 256));
        }
        double per_iter = 0.0;   // flops or bytes per thread and iteration
        int iters = 0;
        auto launch = [&](int it) -> int {
            switch (kind) {
                case WG_CEIL_FP32_FMA2: k_ceil_fma2<<<blocks, kThreads>>>(it, 1.0f, sink); break;
                case WG_CEIL_FP32_FMA: k_ceil_fma<<<blocks, kThreads>>>(it, 1.0f, sink); break;
                case WG_CEIL_FETCH_L1:
                case WG_CEIL_FETCH_L2: k_ceil_fetch<<<blocks, kThreads>>>(buf, n_chunks, it, sink); break;
                default: k_ceil_shared<<<blocks, kThreads>>>(it, sink); break;
            }
            WG_LAUNCHED("k_ceil");
            return WG_OK;
        };
        switch (kind) {
            case WG_CEIL_FP32_FMA2: per_iter = 4.0 * kChains * 4.0; iters = 20000; break;
            case WG_CEIL_FP32_FMA: per_iter = 4.0 * 2 * kChains * 2.0; iters = 20000; break;
            default: per_iter = 8.0 * kLoads; iters = 8000; break;
        }
        int r = launch(iters / 10);     // warm-up
        if (r != WG_OK) return r;
        WG_CUDA(cudaEventRecord(e0));
        r = launch(iters);
        if (r != WG_OK) return r;
        WG_CUDA(cudaEventRecord(e1));
        WG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        WG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms <= 0.f) return fail(WG_E_CUDA, "ceiling_measure: empty timing");
        *value = threads * iters * per_iter / (ms * 1e-3);
        return WG_OK;
    };
    rc = run();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    return rc;
}
