// Gridding phase (thesis Sec. 4.3.3 "The gridding phase", eq. "gridding"), GB300 design.
//
// Work unit ("task") = one segment of seg_len consecutive gridded entries x one block of up to
// `slots` footprint points (both chosen by the work list's plan; see grid_autotune).  A warp takes tasks from a global counter (persistent
// kernel, dynamic load balance).  Each lane owns R <= kRMax fixed residue classes
// (x mod S, y mod S) of the footprint, the ownership of Romein's algorithm (Sec. 2.5): for
// every record exactly one grid pixel of each owned class lies inside the S x S footprint, so
// lanes never touch the same pixel and accumulate in registers while the pixel stays the
// same; when it moves, the lane flushes its accumulators with one vector FP32 atomic per pixel
// (all polarisations of a pixel are contiguous).
//
// Fast path: consecutive gridded entries of a track usually keep the same footprint origin and
// differ only in the sub-kernel z (about 85% of them, weighted by S^2, in the benchmark
// workload).  Then each point's kernel offset toff = dv S + du and pixel are unchanged: the lane
// only loads C[z + toff] and does 4P FMAs.  When the footprint moves, the lane recomputes
// its offsets with the modular wrap and flushes the pixels that changed.  The segment's entries
// and weighted visibilities are staged in shared memory once per task (cp.async).  R (points per
// lane) is chosen per run of records with the same support and channel, or fixed per launch.
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace wg {

namespace {

constexpr int kWarps = 4;           // warps per block

// One staged record: its entry (w replaced by the key) and weighted visibilities, 16-byte
// aligned for cp.async (P = 1 pads to 32 bytes).
template <int P>
struct StagedRec {
    int4 e;
    float2 g[P == 1 ? 2 : P];
};

// Per-warp shared memory: the residue-class arrays, then seg_len staged records, all at fixed
// offsets from the warp's base.
template <int P>
struct WarpSmem {
    short (*pu)[32];         // [kRMax][32] each lane's owned residue classes: x mod S
    short (*pv)[32];         // [kRMax][32] and y mod S
    int (*cur)[32];          // [kRMax][32] each lane's current pixels (read when the footprint moves)
    StagedRec<P>* rec;       // [seg_len]
    static constexpr size_t kFixed = 2 * kRMax * 32 * sizeof(short) + kRMax * 32 * sizeof(int);
    __device__ explicit WarpSmem(unsigned char* base)
        : pu(reinterpret_cast<short (*)[32]>(base)),
          pv(reinterpret_cast<short (*)[32]>(base) + kRMax),
          cur(reinterpret_cast<int (*)[32]>(base + 2 * kRMax * 32 * sizeof(short))),
          rec(reinterpret_cast<StagedRec<P>*>(base + kFixed)) {}
    static constexpr size_t bytes(int seg_len) { return kFixed + (size_t)seg_len * sizeof(StagedRec<P>); }
};

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }

template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Packed FP32 pairs (Blackwell f32x2 arithmetic): one instruction does two FP32 FMAs.
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

// kernel-table samples: complex float32, bfloat16 or float16, widened to float at use
__device__ __forceinline__ float2 to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
__device__ __forceinline__ float2 to_f2(__half2 v) { return __half22float2(v); }

template <typename TS>
__device__ __forceinline__ TS load_sample(const TS* p)
{
    const unsigned u = __ldg(reinterpret_cast<const unsigned*>(p));
    TS v;
    memcpy(&v, &u, sizeof(v));
    return v;
}

// A float2 sample is loaded straight into a 64-bit register pair; narrower samples are widened
// and packed.
__device__ __forceinline__ f32x2 load_kv(const float2* p) { return __ldg(reinterpret_cast<const f32x2*>(p)); }
template <typename TS>
__device__ __forceinline__ TS load_kv(const TS* p) { return load_sample(p); }
// A point's sample offset: in bytes for FP32 samples, added to the sub-kernel's address as an
// unsigned 32-bit value (as a signed element index it measured about two integer instructions
// more per load); in elements for the 4-byte samples, where the element form measured faster.
template <typename TS>
constexpr int kOffScale = std::is_same<TS, float2>::value ? (int)sizeof(float2) : 1;
__device__ __forceinline__ f32x2 load_at(const float2* kz, int off)
{
    return load_kv(reinterpret_cast<const float2*>(reinterpret_cast<const char*>(kz) + (unsigned)off));
}
template <typename TS>
__device__ __forceinline__ TS load_at(const TS* kz, int off) { return load_kv(kz + off); }

template <typename TS>
struct KvReg { typedef TS type; };
template <>
struct KvReg<float2> { typedef f32x2 type; };
__device__ __forceinline__ f32x2 kv_x2(f32x2 v) { return v; }
template <typename TS>
__device__ __forceinline__ f32x2 kv_x2(TS v)
{
    const float2 f = to_f2(v);
    return pack2(f.x, f.y);
}

// Accumulators per point and polarisation.  P = 1 keeps two packed pairs, A = k (gx, gx) and
// B = k (gy, gy) summed over records, so that a loaded sample k = (kx, ky) feeds the packed FMAs
// as it is; the pixel's sum is (A.x - B.y, A.y + B.x).  P = 2, 4 keep one pair, summed as
// (gx, gy) (kx, kx) + (-gy, gx) (ky, ky): the two broadcasts of k per point serve P polarisations.
template <int P>
constexpr int acc_pairs() { return P == 1 ? 2 : 1; }

// exact rounding error of s = fl(a + b) (TwoSum, Knuth)
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    return __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

__device__ __forceinline__ float4 add_err4(float4 old, float4 v)
{
    return make_float4(two_sum_err(old.x, v.x, __fadd_rn(old.x, v.x)), two_sum_err(old.y, v.y, __fadd_rn(old.y, v.y)),
                       two_sum_err(old.z, v.z, __fadd_rn(old.z, v.z)), two_sum_err(old.w, v.w, __fadd_rn(old.w, v.w)));
}

// Adds a lane's accumulators to one pixel.  COMP: the atomic returns the previous value, from
// which the rounding error of the add is recovered exactly and added to the error grid.
template <int P, bool COMP>
__device__ __forceinline__ void flush_pixel(float2* __restrict__ gch, float2* __restrict__ ech, int pix,
                                            f32x2 (&acc)[P][acc_pairs<P>()])
{
    float2* d = gch + (size_t)pix * P;
    float2 a[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if constexpr (acc_pairs<P>() == 2) {
            const float2 u = unpack2(acc[p][0]), v = unpack2(acc[p][1]);
            a[p] = make_float2(u.x - v.y, u.y + v.x);
        } else {
            a[p] = unpack2(acc[p][0]);
        }
    }
    if constexpr (P == 1) {
        if constexpr (COMP) {
            const float2 o = atomicAdd(d, a[0]);
            const float2 e = make_float2(two_sum_err(o.x, a[0].x, __fadd_rn(o.x, a[0].x)),
                                         two_sum_err(o.y, a[0].y, __fadd_rn(o.y, a[0].y)));
            atomicAdd(ech + pix, e);
        } else {
            atomicAdd(d, a[0]);
        }
    } else {
#pragma unroll
        for (int h = 0; h < P; h += 2) {
            const float4 v = make_float4(a[h].x, a[h].y, a[h + 1].x, a[h + 1].y);
            if constexpr (COMP) {
                const float4 o = atomicAdd(reinterpret_cast<float4*>(d + h), v);
                atomicAdd(reinterpret_cast<float4*>(ech + (size_t)pix * P + h), add_err4(o, v));
            } else {
                atomicAdd(reinterpret_cast<float4*>(d + h), v);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int q = 0; q < acc_pairs<P>(); ++q) acc[p][q] = 0ull;
}

// After staging, an entry's w field holds its key: support << 16 | channel, or -1 for an
// entry rejected by the staging bounds checks.
__device__ __forceinline__ int entry_key(const int4& E) { return E.w; }

// Processes records [j, e1) while their (support, channel) key equals `key` with R <= kRMax
// points per lane (task block `blk` of the support's footprint); flushes its pixels and returns
// the first record not processed.  R is warp-uniform.  RT > 0 fixes R = RT at compile time (the
// point loops then run without per-point checks; points past S^2 in the last block load sample
// offset 0 and are never flushed); RT = 0 takes the runtime R and stops each loop at it.
// The samples of a record are loaded just before its FMAs: the other warps on the SM hide
// their latency (a register prefetch of the next record's samples measured slower).
template <int P, typename TS, bool COMP, int RT>
__device__ __forceinline__ int run_records(int j, int e1, int key, int S, int R, int blk, int N, int lane,
                                           WarpSmem<P>& sm, const TS* __restrict__ table,
                                           const int* __restrict__ supports, float2* __restrict__ gch,
                                           float2* __restrict__ ech)
{
    constexpr int KA = acc_pairs<P>();
    typedef typename KvReg<TS>::type KV;
    if constexpr (RT > 0) R = RT;
    f32x2 acc[kRMax][P][KA];
    int toff[kRMax];         // each point's sample offset in the sub-kernel (kOffScale units)
    unsigned valid = 0;
    const int s2 = S * S, sbase = blk * 32 * R;
    // slots run row-major over the residue classes, so the 32 lanes of a point-row read
    // consecutive samples (a layout of 4 x 8 class blocks per point-row, which wraps fewer
    // point-rows per footprint move, spread each load over more cache lines and measured slower)
    const float inv_s = 1.0f / (float)S;
#pragma unroll
    for (int r = 0; r < kRMax; ++r) {
        const int sl = sbase + r * 32 + lane;
        sm.cur[r][lane] = -1;
        toff[r] = 0;
        if (r < R) {
            // a slot past S^2 follows class (0, 0): its sample offset stays inside the
            // sub-kernel, and it is never flushed
            int pu = 0, pv = 0;
            if (sl < s2) {
                valid |= 1u << r;
                const int2 vu = divmod_small(sl, S, inv_s);
                pv = vu.x;
                pu = vu.y;
            }
            sm.pu[r][lane] = (short)pu;
            sm.pv[r][lane] = (short)pv;
        }
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int q = 0; q < KA; ++q) acc[r][p][q] = 0ull;
    }
    int fp = -1;             // footprint origin (x0 | y0 << 16) the offsets refer to
    for (; j < e1; ++j) {
        const int4 E = sm.rec[j].e;
        if (entry_key(E) != key) break;
        if (E.x != fp) {     // the footprint moved: new offsets, flush the pixels that change
            const int x0 = E.x & 0xFFFF, y0 = (E.x >> 16) & 0xFFFF;
            const int cu = E.y & 0xFFFF, cv = (E.y >> 16) & 0xFFFF;
            const int dx = x0 - (fp & 0xFFFF), dy = y0 - (fp >> 16);
            if (fp >= 0 && ((dy == 0 && (dx == 1 || dx == -1)) || (dx == 0 && (dy == 1 || dy == -1)))) {
                // A one-cell move (almost every move of a track).  Every point's offset shifts by
                // the move; only the column (or row) of classes that left the footprint wraps to
                // its other side, and only its points change pixel.  That class is the new
                // origin's residue, one less for a move towards +x (+y).
                const bool along_x = dy == 0;
                const int d = along_x ? dx : dy;
                const int cn = along_x ? cu : cv;                  // (-origin) mod S
                const int m = cn ? S - cn : 0;                     // origin mod S
                const int c = d > 0 ? (m ? m - 1 : S - 1) : m;     // the class that wraps
                const int step = along_x ? 1 : S;                  // samples per cell of the move
                const int shift = d * step * kOffScale<TS>;
                const int wrap = d * S * step * kOffScale<TS>;
                const int pstep = along_x ? d * S : d * S * N;     // pixel step of a wrapped point
                short (*cls)[32] = along_x ? sm.pu : sm.pv;
#pragma unroll
                for (int r = 0; r < kRMax; ++r) {
                    if (r < R) {
                        const bool w = cls[r][lane] == c;
                        toff[r] += w ? wrap - shift : -shift;
                        if (w && (valid & (1u << r))) {
                            const int cur = sm.cur[r][lane];
                            flush_pixel<P, COMP>(gch, ech, cur, acc[r]);
                            sm.cur[r][lane] = cur + pstep;
                        }
                    }
                }
            } else {
                // the first record of the run, or a jump: place every point from its class
#pragma unroll
                for (int r = 0; r < kRMax; ++r) {
                    if (r < R) {
                        int du = sm.pu[r][lane] + cu;
                        du -= (du >= S) ? S : 0;
                        int dv = sm.pv[r][lane] + cv;
                        dv -= (dv >= S) ? S : 0;
                        toff[r] = (dv * S + du) * kOffScale<TS>;
                        if (valid & (1u << r)) {
                            const int pix = (y0 + dv) * N + x0 + du;
                            const int cur = sm.cur[r][lane];
                            if (pix != cur) {
                                if (cur >= 0) flush_pixel<P, COMP>(gch, ech, cur, acc[r]);
                                sm.cur[r][lane] = pix;
                            }
                        }
                    }
                }
            }
            fp = E.x;
        }
        KV kv[kRMax];
        const TS* kz = table + E.z;
#pragma unroll
        for (int r = 0; r < kRMax; ++r) {
            if (RT == 0 && r >= R) break;
            if (r < R) kv[r] = load_at(kz, toff[r]);   // invalid points read offset 0, never flushed
        }
        if constexpr (KA == 2) {
            // A += k (gx, gx), B += k (gy, gy)
            f32x2 gxx[P], gyy[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float2 gm = sm.rec[j].g[p];
                gxx[p] = pack2(gm.x, gm.x);
                gyy[p] = pack2(gm.y, gm.y);
            }
#pragma unroll
            for (int r = 0; r < kRMax; ++r) {
                if (RT == 0 && r >= R) break;
                if (r < R) {
                    const f32x2 k = kv_x2(kv[r]);
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        acc[r][p][0] = fma2(k, gxx[p], acc[r][p][0]);
                        acc[r][p][1] = fma2(k, gyy[p], acc[r][p][1]);
                    }
                }
            }
        } else {
            // acc += gamma * kv as (gx, gy) (kx, kx) + (-gy, gx) (ky, ky), two packed FMAs per pol
            f32x2 g1[P], g2[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float2 gm = sm.rec[j].g[p];
                g1[p] = pack2(gm.x, gm.y);
                g2[p] = pack2(-gm.y, gm.x);
            }
#pragma unroll
            for (int r = 0; r < kRMax; ++r) {
                if (RT == 0 && r >= R) break;
                if (r < R) {
                    const float2 k = unpack2(kv_x2(kv[r]));
                    const f32x2 kxx = pack2(k.x, k.x), kyy = pack2(k.y, k.y);
#pragma unroll
                    for (int p = 0; p < P; ++p) acc[r][p][0] = fma2(g2[p], kyy, fma2(g1[p], kxx, acc[r][p][0]));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRMax; ++r) {
        if (r < R) {     // points past R hold no pixel
            const int cur = sm.cur[r][lane];
            if (cur >= 0) flush_pixel<P, COMP>(gch, ech, cur, acc[r]);
        }
    }
    return j;
}

}  // namespace

template <int P, typename TS, bool COMP, int RT>
// five blocks of 4 warps per SM at one polarisation (at most 102 registers), four otherwise
__global__ void __launch_bounds__(kWarps * 32, P == 1 ? 5 : 4) k_grid(const int4* __restrict__ entries,
                                                         const float2* __restrict__ gamma,
                                                         const int* __restrict__ seg_off,
                                                         const long long* __restrict__ scal,
                                                         const int* __restrict__ supports,
                                                         const TS* __restrict__ table,
                                                         float2* __restrict__ grid, float2* __restrict__ errgrid,
                                                         int N, int K, int C, int64_t n_samples, int seg_len,
                                                         int slots, unsigned int* __restrict__ counter,
                                                         long long* __restrict__ dropped)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem<P> sm(smem_raw + (size_t)wid * WarpSmem<P>::bytes(seg_len));
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
        const int e0 = lo * seg_len;
        const int n = (int)min((long long)seg_len, n_entries - e0);

        // stage the segment's entries and weighted visibilities
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            cp_async16(&sm.rec[i].e, entries + e0 + i);
            if constexpr (P == 1) {
                cp_async8(&sm.rec[i].g[0], gamma + (size_t)(e0 + i));
            } else {
#pragma unroll
                for (int p = 0; p < P; p += 2) cp_async16(&sm.rec[i].g[p], gamma + (size_t)(e0 + i) * P + p);
            }
        }
        cp_commit();
        cp_wait<0>();
        __syncwarp();
        // device-side bounds checks (never taken with a consistent work list)
        for (int i = lane; i < n; i += 32) {
            const int4 E = sm.rec[i].e;
            const int k = E.w & 0xFFF, ch = (E.w >> 16) & 0xFFFF;
            bool ok = E.w >= 0 && k < K && ch < C;
            if (ok) {
                const int S = __ldg(&supports[k]);
                const int x0 = E.x & 0xFFFF, y0 = (E.x >> 16) & 0xFFFF;
                const int cu = E.y & 0xFFFF, cv = (E.y >> 16) & 0xFFFF;
                ok = x0 + S <= N && y0 + S <= N && cu < S && cv < S && E.z >= 0 &&
                     (int64_t)E.z + (int64_t)S * S <= n_samples;
            }
            if (ok) {
                sm.rec[i].e.w = (__ldg(&supports[k]) << 16) | ch;
            } else {
                sm.rec[i].e.w = -1;
                if (blk == 0) atomicAdd(reinterpret_cast<unsigned long long*>(dropped), 1ull);
            }
        }
        __syncwarp();

        int j = 0;
        while (j < n) {
            const int key = entry_key(sm.rec[j].e);
            if (key < 0) {
                ++j;
                continue;
            }
            const int S = key >> 16, ch = key & 0xFFFF;
            float2* gch = grid + (size_t)ch * chan_stride;
            float2* ech = COMP ? errgrid + (size_t)ch * chan_stride : nullptr;
            const int s2 = S * S;
            const int nb = (s2 + slots - 1) / slots;
            const int R = RT > 0 ? RT : (s2 + 32 * nb - 1) / (32 * nb);
            if (blk >= nb) {     // this block has no points for this support: skip the run
                while (j < n && entry_key(sm.rec[j].e) == key) ++j;
                continue;
            }
            j = run_records<P, TS, COMP, RT>(j, n, key, S, R, blk, N, lane, sm, table, supports, gch, ech);
        }
    }
}

// adds the batch normaliser and statistics into the grid's accumulators; the batch's normaliser
// row c goes to grid channel c * stride (w-stacking keeps a channel's N_p in its plane 0)
__global__ void k_accumulate(double* __restrict__ gnorm, const double* __restrict__ bnorm, int n, int P, int stride,
                             unsigned long long* __restrict__ gcnt, const unsigned long long* __restrict__ bcnt)
{
    const int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (i < n) gnorm[(size_t)(i / P) * stride * P + i % P] += bnorm[i];
    if (i < ST_N) gcnt[i] += bcnt[i];
}

// grid += err; err = 0 (folds the compensated flushes' rounding errors back)
__global__ void k_fold(float4* __restrict__ grid, float4* __restrict__ err, int64_t n4)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    const float4 a = grid[i], e = err[i];
    grid[i] = make_float4(a.x + e.x, a.y + e.y, a.z + e.z, a.w + e.w);
    err[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int P, typename TS, bool COMP, int RT>
static int grid_launch(Grid& g, const Table& t, const WorkList& wl, const TS* table, cudaStream_t s)
{
    // occupancy per segment length (the shared-memory staging grows with it)
    static int blocks_per_sm[kSegLenMax / kSegLenMin + 1] = {0};
    const int smem = (int)(kWarps * WarpSmem<P>::bytes(wl.seg_len));
    int& bps = blocks_per_sm[wl.seg_len / kSegLenMin];
    if (bps == 0) {
        WG_CUDA(cudaFuncSetAttribute(k_grid<P, TS, COMP, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kWarps * WarpSmem<P>::bytes(kSegLenMax))));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_grid<P, TS, COMP, RT>, kWarps * 32, smem) !=
                cudaSuccess ||
            bps < 1)
            bps = 1;
    }
    k_grid<P, TS, COMP, RT><<<num_sms() * bps, kWarps * 32, smem, s>>>(
        wl.entries, wl.gamma, wl.seg_off, wl.scal, t.supports_d, table, g.data, g.err, g.n, t.K, g.n_chan,
        t.n_samples, wl.seg_len, wl.slots, wl.task_counter, wl.scal + 3);
    WG_LAUNCHED("k_grid");
    return WG_OK;
}

// Fixed-R kernels: R = 8 (slots = 256) for every table type, with or without compensation;
// R = 4 (slots = 128) for FP32 tables without compensation.  Other plans take the runtime-R
// kernel.
template <int P, bool COMP>
static int grid_dispatch(Grid& g, const Table& t, const WorkList& wl, cudaStream_t s)
{
    const bool r8 = wl.fixed_r && wl.slots == 256;
    switch (t.store) {
        case WG_BF16: {
            const auto* tb = static_cast<const __nv_bfloat162*>(t.data_lp);
            return r8 ? grid_launch<P, __nv_bfloat162, COMP, 8>(g, t, wl, tb, s)
                      : grid_launch<P, __nv_bfloat162, COMP, 0>(g, t, wl, tb, s);
        }
        case WG_F16: {
            const auto* th = static_cast<const __half2*>(t.data_lp);
            return r8 ? grid_launch<P, __half2, COMP, 8>(g, t, wl, th, s) : grid_launch<P, __half2, COMP, 0>(g, t, wl, th, s);
        }
        default:
            if (r8) return grid_launch<P, float2, COMP, 8>(g, t, wl, t.data, s);
            if constexpr (!COMP) {
                if (wl.fixed_r && wl.slots == 128) return grid_launch<P, float2, false, 4>(g, t, wl, t.data, s);
            }
            return grid_launch<P, float2, COMP, 0>(g, t, wl, t.data, s);
    }
}

template <int P>
static int grid_impl(Grid& g, const Table& t, const WorkList& wl, cudaStream_t s)
{
    WG_CUDA(cudaMemsetAsync(wl.task_counter, 0, sizeof(unsigned int), s));
    const int rc = g.comp ? grid_dispatch<P, true>(g, t, wl, s) : grid_dispatch<P, false>(g, t, wl, s);
    if (rc != WG_OK) return rc;
    if (g.comp) {
        const int64_t n4 = (int64_t)g.n_chan * g.n * g.n * P / 2;
        k_fold<<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(reinterpret_cast<float4*>(g.data),
                                                            reinterpret_cast<float4*>(g.err), n4);
        WG_LAUNCHED("k_fold");
    }
    if (wl.append) return WG_OK;     // appended batches added their N_p terms at vis_compress
    const int n = (g.n_chan / wl.wstack_k) * g.n_pol;     // normaliser rows of the batch
    const int m = std::max(n, (int)ST_N);
    k_accumulate<<<(m + 255) / 256, 256, 0, s>>>(g.norm, wl.norm_batch, n, g.n_pol, wl.wstack_k, g.counters, wl.stats);
    WG_LAUNCHED("k_accumulate");
    return WG_OK;
}

int launch_accumulate(const Grid& g, const WorkList& wl, int chan0, cudaStream_t s)
{
    const int n = wl.C * g.n_pol;
    const int m = std::max(n, (int)ST_N);
    k_accumulate<<<(m + 255) / 256, 256, 0, s>>>(g.norm + (size_t)chan0 * g.n_pol, wl.norm_batch, n, g.n_pol, 1,
                                                 g.counters, wl.stats_batch);
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
