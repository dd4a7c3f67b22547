// Degridding: the adjoint of the gridding map (not in the thesis).
//
// For a gridded entry (footprint origin (x0, y0), kernel pointer z, grid channel c) the kernel sum
//   m_p = sum_{i,j} conj(C[z + i S + j]) grid_c,p(y0 + i, x0 + j)
// takes two launches.
//
// k_degrid_sum runs the gridder's tasks (a segment of consecutive entries x one block of the
// footprint, as the work list's plan defines them) with the gridder's ownership: each lane owns
// R residue classes (x mod S, y mod S) of the footprint, so exactly one pixel of each class lies
// in every entry's footprint (Romein's argument, Sec. 2.5).  The lane keeps those pixels' values
// (all polarisations) in registers and reloads one only when the footprint moves and the class's
// pixel changes; for consecutive entries of a track that keep the footprint and differ only in
// the sub-kernel z it loads nothing but the kernel samples.  Per entry each lane sums its R
// points into 2P floats; these go through a shared-memory transpose (batches of 64 / (2P)
// entries), after which each lane holds two components of one entry summed over the warp and
// adds them to a per-entry FP32 accumulator with one vector atomic per footprint block.
//
// k_degrid_tile writes the records of each entry's run.  Compression (Sec. 4.3.3) carries over:
// every record compressed into an entry has its footprint and kernel samples, so m is computed
// once per entry and written to each record of the run, conjugated back where psi = -1 (w' < 0),
// with the cross hands swapped back under cross-hand swapping, and for the adjoint mode scaled
// by eps (1 - f) (the vis -> grid map's R-linear outer factor).  It works per preparation tile
// through shared memory so that the output is written row-major with coalesced stores.
#include "internal.cuh"

namespace wg {

namespace {

constexpr int kWarps = 4;           // warps per block of k_degrid_sum
constexpr int kTileCap = 4096;      // records per preparation tile: rpb x C <= max(kTileRecords, n_chan <= 4096)
static_assert(kTileRecords <= kTileCap, "a preparation tile must fit the degridder's output tile");

typedef unsigned long long f32x2;   // a packed FP32 pair (Blackwell f32x2 arithmetic)

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

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}

// the P polarisations of one pixel as packed pairs (gx, gy)
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

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The per-entry reduction buffers 64 / (2P) entries of 2P lane partials: slot b holds lane l's
// component c at b * (33 * 2P) + l * 2P + c (one 2P-float pad per slot, so that the 32 lanes'
// reads of two adjacent components of 32 / P different slots fall in distinct banks).
constexpr int kRedFloats = 64 * 33;      // per warp, any P

// Per-warp shared memory: the residue-class arrays, the reduction buffer, then the segment's
// staged entries.
struct WarpSmem {
    short (*pu)[32];         // [kRMax][32] each lane's owned residue classes: x mod S
    short (*pv)[32];         // [kRMax][32] and y mod S
    float* red;              // [kRedFloats]
    int4* rec;               // [seg_len] entries, w replaced by the key
    static constexpr size_t kFixed = 2 * kRMax * 32 * sizeof(short) + kRedFloats * sizeof(float);
    __device__ explicit WarpSmem(unsigned char* base)
        : pu(reinterpret_cast<short (*)[32]>(base)),
          pv(reinterpret_cast<short (*)[32]>(base) + kRMax),
          red(reinterpret_cast<float*>(base + 2 * kRMax * 32 * sizeof(short))),
          rec(reinterpret_cast<int4*>(base + kFixed)) {}
    static constexpr size_t bytes(int seg_len) { return kFixed + (size_t)seg_len * sizeof(int4); }
};

// Entries [j, e1) of the staged segment while their key (support, grid channel) equals `key`,
// footprint block `blk`, R points per lane (RT > 0 fixes R at compile time; points past S^2
// keep pixel value 0 and read sample offset 0).  Adds each entry's sums to acc[j][2P]; returns
// the first entry not processed.  Each lane stores its 2P partials of an entry in the reduction
// buffer; every 64 / (2P) entries (and at the end) each lane sums two adjacent components of one
// entry over the 32 lanes and adds them to acc with one vector atomic.
template <int P, int RT>
__device__ __forceinline__ int degrid_records(int j, int e1, int key, int S, int R, int blk, int N, int lane,
                                              WarpSmem& sm, const float2* __restrict__ table,
                                              const float2* __restrict__ gch, float* __restrict__ acc)
{
    constexpr int V = 2 * P, NB = 64 / V, SLOT = 33 * V;
    if constexpr (RT > 0) R = RT;
    int nbuf = 0, jb = j;     // entries buffered, and the first of them
    // lane l sums components c, c + 1 of buffered entry b over the 32 lanes
    auto drain = [&](int n) {
        __syncwarp();
        const int b = (2 * lane) / V, c = (2 * lane) % V;
        if (b < n) {
            const float* src = sm.red + b * SLOT + c;
            f32x2 t = 0ull;
#pragma unroll
            for (int l2 = 0; l2 < 32; ++l2) {
                // V = 8: lanes with bit 2 set stored their two 16-byte halves swapped
                const int cs = (V == 8 && (l2 & 4)) ? 4 : 0;
                t = add2(t, *reinterpret_cast<const f32x2*>(src + l2 * V + (c ^ cs) - c));
            }
            atomicAdd(reinterpret_cast<float2*>(acc + (size_t)(jb + b) * V + c), unpack2(t));
        }
        __syncwarp();
    };
    f32x2 pv[kRMax][P];
    int toff[kRMax], cur[kRMax];     // sample byte offset and pixel held of each owned class
    unsigned valid = 0;
    const int s2 = S * S, sbase = blk * 32 * R;
    const float inv_s = 1.0f / (float)S;
#pragma unroll
    for (int r = 0; r < kRMax; ++r) {
        const int sl = sbase + r * 32 + lane;
        cur[r] = -1;
        toff[r] = 0;
        if (r < R) {
            // a slot past S^2 follows class (0, 0): its sample offset stays inside the
            // sub-kernel, and its pixel value stays 0
            int pu = 0, pv_ = 0;
            if (sl < s2) {
                valid |= 1u << r;
                const int2 vu = divmod_small(sl, S, inv_s);
                pv_ = vu.x;
                pu = vu.y;
            }
            sm.pu[r][lane] = (short)pu;
            sm.pv[r][lane] = (short)pv_;
        }
#pragma unroll
        for (int p = 0; p < P; ++p) pv[r][p] = 0ull;
    }
    int fp = -1;             // footprint origin (x0 | y0 << 16) the offsets and pixels refer to
    for (; j < e1; ++j) {
        const int4 E = sm.rec[j];
        if (E.w != key) break;
        if (E.x != fp) {     // the footprint moved: new offsets, reload the pixels that change
            const int x0 = E.x & 0xFFFF, y0 = (E.x >> 16) & 0xFFFF;
            const int cu = E.y & 0xFFFF, cv = (E.y >> 16) & 0xFFFF;
            const int dx = x0 - (fp & 0xFFFF), dy = y0 - (fp >> 16);
            if (fp >= 0 && ((dy == 0 && (dx == 1 || dx == -1)) || (dx == 0 && (dy == 1 || dy == -1)))) {
                // a one-cell move: every offset shifts by the move, and only the class column
                // (or row) that left the footprint wraps and takes a new pixel (as in the gridder)
                const bool along_x = dy == 0;
                const int d = along_x ? dx : dy;
                const int cn = along_x ? cu : cv;                  // (-origin) mod S
                const int m = cn ? S - cn : 0;                     // origin mod S
                const int c = d > 0 ? (m ? m - 1 : S - 1) : m;     // the class that wraps
                const int step = along_x ? 1 : S;
                const int shift = d * step * (int)sizeof(float2);
                const int wrap = d * S * step * (int)sizeof(float2);
                const int pstep = along_x ? d * S : d * S * N;
                short (*cls)[32] = along_x ? sm.pu : sm.pv;
#pragma unroll
                for (int r = 0; r < kRMax; ++r) {
                    if (r < R) {
                        const bool w = cls[r][lane] == c;
                        toff[r] += w ? wrap - shift : -shift;
                        if (w && (valid & (1u << r))) {
                            cur[r] += pstep;
                            load_pixel<P>(gch + (size_t)cur[r] * P, pv[r]);
                        }
                    }
                }
            } else {
                // the first entry of the run, or a jump: place every point from its class
#pragma unroll
                for (int r = 0; r < kRMax; ++r) {
                    if (r < R) {
                        int du = sm.pu[r][lane] + cu;
                        du -= (du >= S) ? S : 0;
                        int dv = sm.pv[r][lane] + cv;
                        dv -= (dv >= S) ? S : 0;
                        toff[r] = (dv * S + du) * (int)sizeof(float2);
                        if (valid & (1u << r)) {
                            const int pix = (y0 + dv) * N + x0 + du;
                            if (pix != cur[r]) {
                                load_pixel<P>(gch + (size_t)pix * P, pv[r]);
                                cur[r] = pix;
                            }
                        }
                    }
                }
            }
            fp = E.x;
        }
        f32x2 kv[kRMax];
        const f32x2* kz = reinterpret_cast<const f32x2*>(table + E.z);
#pragma unroll
        for (int r = 0; r < kRMax; ++r) {
            if (RT == 0 && r >= R) break;
            // unsigned 32-bit byte offset: cheaper than a signed element index (see the gridder)
            if (r < R) kv[r] = __ldg(reinterpret_cast<const f32x2*>(reinterpret_cast<const char*>(kz) + (unsigned)toff[r]));
        }
        // A_p = sum kx (gx, gy), B_p = sum ky (gx, gy); conj(k) g = (A.x + B.y, A.y - B.x)
        f32x2 A[P], B[P];
#pragma unroll
        for (int p = 0; p < P; ++p) A[p] = B[p] = 0ull;
#pragma unroll
        for (int r = 0; r < kRMax; ++r) {
            if (RT == 0 && r >= R) break;
            if (r < R) {
                const float2 k = unpack2(kv[r]);
                const f32x2 kxx = pack2(k.x, k.x), kyy = pack2(k.y, k.y);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    A[p] = fma2(kxx, pv[r][p], A[p]);
                    B[p] = fma2(kyy, pv[r][p], B[p]);
                }
            }
        }
        float v[V];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float2 a = unpack2(A[p]), b = unpack2(B[p]);
            v[2 * p] = a.x + b.y;
            v[2 * p + 1] = a.y - b.x;
        }
        float* dst = sm.red + nbuf * SLOT + lane * V;
        if constexpr (V == 8) {
            // halves swapped for lanes with bit 2 set: the 8 lanes of a quarter-warp store to
            // distinct banks
            const int sw = (lane & 4) ? 4 : 0;
            *reinterpret_cast<float4*>(dst + sw) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(dst + (4 ^ sw)) = make_float4(v[4], v[5], v[6], v[7]);
        } else if constexpr (V == 4) {
            *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
        }
        if (++nbuf == NB) {
            drain(NB);
            nbuf = 0;
            jb = j + 1;
        }
    }
    if (nbuf) drain(nbuf);
    return j;
}

// An entry's placement is consistent with the table and the grid (the checks of the gridder's
// staging; never false for a work list written by vis_compress for this table and grid).
__device__ __forceinline__ bool entry_ok(const int4& E, const int* __restrict__ supports, int N, int K, int C,
                                         int64_t n_samples)
{
    const int k = E.w & 0xFFF, ch = (E.w >> 16) & 0xFFFF;
    if (E.w < 0 || k >= K || ch >= C) return false;
    const int S = __ldg(&supports[k]);
    const int x0 = E.x & 0xFFFF, y0 = (E.x >> 16) & 0xFFFF;
    const int cu = E.y & 0xFFFF, cv = (E.y >> 16) & 0xFFFF;
    return x0 + S <= N && y0 + S <= N && cu < S && cv < S && E.z >= 0 &&
           (int64_t)E.z + (int64_t)S * S <= n_samples;
}

}  // namespace

// acc[0 .. n_entries * 2P) = 0
__global__ void k_degrid_zero(float4* __restrict__ acc, const long long* __restrict__ scal, int P)
{
    const long long n4 = scal[0] * P / 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
        acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int P, int RT>
__global__ void __launch_bounds__(kWarps * 32, P == 1 ? 5 : 4) k_degrid_sum(const int4* __restrict__ entries,
                                                               const int* __restrict__ seg_off,
                                                               const long long* __restrict__ scal,
                                                               const int* __restrict__ supports,
                                                               const float2* __restrict__ table,
                                                               const float2* __restrict__ grid, int N, int K, int C,
                                                               int64_t n_samples, int seg_len, int slots,
                                                               unsigned int* __restrict__ counter,
                                                               float* __restrict__ acc, long long* __restrict__ dropped)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem sm(smem_raw + (size_t)wid * WarpSmem::bytes(seg_len));
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

        __syncwarp();
        for (int i = lane; i < n; i += 32) cp_async16(&sm.rec[i], entries + e0 + i);
        asm volatile("cp.async.commit_group;\n" ::);
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const int4 E = sm.rec[i];
            const bool ok = entry_ok(E, supports, N, K, C, n_samples);
            sm.rec[i].w = ok ? (__ldg(&supports[E.w & 0xFFF]) << 16) | ((E.w >> 16) & 0xFFFF) : -1;
            if (!ok && blk == 0) atomicAdd(reinterpret_cast<unsigned long long*>(dropped), 1ull);
        }
        __syncwarp();

        int j = 0;
        while (j < n) {
            const int key = sm.rec[j].w;
            if (key < 0) {
                ++j;
                continue;
            }
            const int S = key >> 16, ch = key & 0xFFFF;
            const int s2 = S * S;
            const int nb = (s2 + slots - 1) / slots;
            const int R = RT > 0 ? RT : (s2 + 32 * nb - 1) / (32 * nb);
            if (blk >= nb) {     // this block has no points for this support: skip the run
                while (j < n && sm.rec[j].w == key) ++j;
                continue;
            }
            j = degrid_records<P, RT>(j, n, key, S, R, blk, N, lane, sm, table, grid + (size_t)ch * chan_stride,
                                      acc + (size_t)e0 * 2 * P);
        }
    }
}

// One thread per entry writes the records of its run: rows run.x..run.y of input channel
// gchan / kst (w-stacking: kst planes per channel), or records run.x..run.y when interleaved.
// One block per preparation tile (rpb rows x all channels) writes the tile's output records
// row-major.  Phase 1 puts each entry's sums into the shared-memory tile at the records of its
// run that fall in the tile (the run before the tile's first head of a list can reach into
// it), phase 2 stores the tile with coalesced vector stores, conjugated back where psi = -1
// (the take-conjugate class bit), with the cross hands swapped back under cross-hand swapping,
// and for the adjoint mode scaled by eps (1 - f).  Records that are not griddable are in no run
// and keep the tile's zero.  Lists: one per input channel (rows), or one in natural record
// order when interleaved.
template <int P>
__global__ void __launch_bounds__(512) k_degrid_tile(const int2* __restrict__ runs, const float2* __restrict__ acc,
                                                     const int* __restrict__ tile_off, const int* __restrict__ chan_base,
                                                     const uint8_t* __restrict__ rclass, const float* __restrict__ weight,
                                                     const uint8_t* __restrict__ flag, int adjoint, int cross_swap,
                                                     int interleave, int64_t rows, int rpb, int C, int64_t n_tiles,
                                                     float2* __restrict__ out)
{
    extern __shared__ __align__(16) float2 s_out[];      // [rpb * C][P]
    const int64_t tile = blockIdx.x;
    const int64_t row0 = tile * rpb;
    const int nrows = (int)min((int64_t)rpb, rows - row0);
    const int nrec = nrows * C;
    for (int i = threadIdx.x; i < nrec * P; i += blockDim.x) s_out[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int nlist = interleave ? 1 : C;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // the tile in list units: rows of a channel, or records in natural order
    const int64_t lo = interleave ? row0 * C : row0, hi = interleave ? row0 * C + nrec : row0 + nrows;
    for (int l = threadIdx.x >> 5; l < nlist; l += nw) {
        const int base = chan_base[l];
        const int first = base + tile_off[tile * C + l];
        const int end = tile + 1 < n_tiles ? base + tile_off[(tile + 1) * C + l] : chan_base[l + 1];
        for (int e = first - 1 + lane; e < end; e += 32) {
            if (e < base) continue;
            const int2 run = runs[e];
            const int64_t a = max((int64_t)run.x, lo), b = min((int64_t)run.y + 1, hi);
            if (a >= b) continue;
            float2 m[P];
#pragma unroll
            for (int p = 0; p < P; ++p) m[p] = acc[(int64_t)e * P + p];
            for (int64_t r = a; r < b; ++r) {
                const int j = interleave ? (int)(r - lo) : (int)(r - row0) * C + l;
#pragma unroll
                for (int p = 0; p < P; ++p) s_out[j * P + p] = m[p];
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nrec; j += blockDim.x) {
        const int64_t rec = row0 * C + j;
        const bool neg = (rclass[rec] >> 3) & 1;
        float2 v[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            // with cross-hand swapping, output pol 1 of a take-conjugate record comes from grid
            // pol 2 and pol 2 from pol 1 (the adjoint of the swap is the swap)
            const int src = (P == 4 && cross_swap && neg && (p == 1 || p == 2)) ? 3 - p : p;
            const float2 a = s_out[j * P + src];
            v[p] = neg ? make_float2(a.x, -a.y) : a;
            if (adjoint) {
                const float wf = weight[rec * P + p] * (1.0f - (float)flag[rec * P + p]);
                v[p].x *= wf;
                v[p].y *= wf;
            }
        }
        float2* o = out + rec * P;
        if constexpr (P == 1) {
            o[0] = v[0];
        } else {
#pragma unroll
            for (int h = 0; h < P; h += 2)
                *reinterpret_cast<float4*>(o + h) = make_float4(v[h].x, v[h].y, v[h + 1].x, v[h + 1].y);
        }
    }
}

template <int P, int RT>
static int degrid_sum_launch(const Grid& g, const Table& t, const WorkList& wl, cudaStream_t s)
{
    static int blocks_per_sm[kSegLenMax / kSegLenMin + 1] = {0};
    const int smem = (int)(kWarps * WarpSmem::bytes(wl.seg_len));
    int& bps = blocks_per_sm[wl.seg_len / kSegLenMin];
    if (bps == 0) {
        WG_CUDA(cudaFuncSetAttribute(k_degrid_sum<P, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kWarps * WarpSmem::bytes(kSegLenMax))));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_degrid_sum<P, RT>, kWarps * 32, smem) !=
                cudaSuccess ||
            bps < 1)
            bps = 1;
    }
    k_degrid_sum<P, RT><<<num_sms() * bps, kWarps * 32, smem, s>>>(
        wl.entries, wl.seg_off, wl.scal, t.supports_d, t.data, g.data, g.n, t.K, g.n_chan, t.n_samples, wl.seg_len,
        wl.slots, wl.task_counter + 1, reinterpret_cast<float*>(wl.dacc), wl.scal + 3);
    WG_LAUNCHED("k_degrid_sum");
    return WG_OK;
}

template <int P>
static int degrid_impl(const Grid& g, const Table& t, const wg_vis_in& in, const WorkList& wl, int mode, float2* out,
                       cudaStream_t s)
{
    if (!wl.dacc) return fail(WG_E_INVALID_ARG, "degrid_vis: the work list has no degridding accumulator");
    WG_CUDA(cudaMemsetAsync(wl.task_counter + 1, 0, sizeof(unsigned int), s));
    const int zb = num_sms() * 4;
    k_degrid_zero<<<zb, 256, 0, s>>>(reinterpret_cast<float4*>(wl.dacc), wl.scal, P);
    WG_LAUNCHED("k_degrid_zero");
    int rc;
    if (wl.fixed_r && wl.slots == 256) rc = degrid_sum_launch<P, 8>(g, t, wl, s);
    else if (wl.fixed_r && wl.slots == 128) rc = degrid_sum_launch<P, 4>(g, t, wl, s);
    else rc = degrid_sum_launch<P, 0>(g, t, wl, s);
    if (rc != WG_OK) return rc;
    const int tile_smem = (int)(sizeof(float2) * (size_t)wl.rpb * in.n_chan * P);
    static bool attr_set[5] = {false, false, false, false, false};
    if (!attr_set[P]) {
        WG_CUDA(cudaFuncSetAttribute(k_degrid_tile<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(float2) * (size_t)kTileCap * P)));
        attr_set[P] = true;
    }
    if (tile_smem > (int)(sizeof(float2) * (size_t)kTileCap * P))
        return fail(WG_E_CAPACITY, "degrid_vis: %d records per preparation tile exceed %d", wl.rpb * in.n_chan, kTileCap);
    if (wl.n_tiles == 0) return WG_OK;     // no records
    k_degrid_tile<P><<<(unsigned)wl.n_tiles, 512, tile_smem, s>>>(
        wl.runs, wl.dacc, wl.tile_cnt, wl.chan_base, wl.rclass, in.weight, in.flag, mode == WG_DEGRID_ADJOINT ? 1 : 0,
        wl.cross_swap ? 1 : 0, wl.interleave ? 1 : 0, in.n_rows, wl.rpb, in.n_chan, wl.n_tiles, out);
    WG_LAUNCHED("k_degrid_tile");
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
