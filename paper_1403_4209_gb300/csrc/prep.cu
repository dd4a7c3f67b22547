// Preparation phase of the WImager algorithm (thesis Sec. 4.3.4) on the GPU.
//
// The input is tiled into blocks of whole rows x all channels (kTileRecords records), read in
// natural [row][chan][pol] order so every load is coalesced.
//   k_classify  (PreProcessUVW, Sec. 4.3.4): FP64 placement of each record (row, chan), its
//               griddability, the compression indicator c (eq. "ci": same footprint origin
//               and kernel pointer as the griddable predecessor (row-1, chan)), g = gd & !c,
//               and statistics; it counts each channel's gridded records in the tile (Index
//               Create and Filter, Algorithm "index").
//   k_scan_tiles / k_finalize: per-channel exclusive scan of the tile counts and the
//               channel bases, so gridded records land channel-major, row-ordered.
//   k_compact   (Compress Index Generate + Compress and Weigh Visibilities, Algorithm
//               "compressindex", eqs. "compress1"/"conjugatetake"): a block scan of g in
//               channel-major order lists the tile's gridded records and gives each its rank
//               in its channel's part of the tile; each gridded record
//               walks its run of compressed successors and sums eps (1-f) psi-conj(vis) (a run
//               crossing a tile end is finished by k_carry from the next tiles' carries); the
//               run's eps (1-f) times its sub-kernel's zeta gives the normaliser terms (eq.
//               "normalizer"), summed by k_norm_sum.
//   k_segments + k_seg_scan (Plan Create / Plan Analyse, Algorithm "plan"): gridded entries
//               are cut into segments of seg_len entries; each segment needs one gridder task
//               per block of `slots` footprint points of its largest support.  The plan can be
//               redone with other parameters (launch_plan) without repeating the preparation.
#include <cmath>
#include <cstdio>
#include <type_traits>

#include <cuda_fp16.h>

#include "internal.cuh"

namespace wg {

namespace {

// a mod S for 0 <= a < 2^20 and 1 <= S < 2^12: the float quotient a (1/S) is within one of the
// integer one, and one correction step each way makes the remainder exact
__device__ __forceinline__ int mod_small(int a, int S, float inv_s)
{
    const int q = __float2int_rz((float)a * inv_s);
    int r = a - q * S;
    r += (r < 0) ? S : 0;
    r -= (r >= S) ? S : 0;
    return r;
}

// ---- untiled bulk copies (TMA) from global into shared memory, completed on an mbarrier ----
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// arrives on the barrier and adds `bytes` to the transfer count its phase waits for
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared memory
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// waits until phase `parity` of the barrier completes, for at most limit_ns; false if it did not
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long limit_ns)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s: a copy that takes longer is an error
constexpr unsigned kBulkChunk = 16384;                        // bytes per bulk copy instruction
constexpr int kCompactThreads = 512;                          // threads of a k_compact block

// some polarisation of record rec unflagged; with `vec` (flag pointer aligned to P bytes) the P
// flag bytes are read in one load and tested for a zero byte
template <typename IDX>
__device__ __forceinline__ bool any_unflagged(const uint8_t* __restrict__ flag, IDX rec, int P, int vec)
{
    if (vec && P == 4) {
        const unsigned w = __ldg(reinterpret_cast<const unsigned*>(flag) + rec);
        return ((w - 0x01010101u) & ~w & 0x80808080u) != 0;     // a zero byte
    }
    if (vec && P == 2) {
        const unsigned short f = __ldg(reinterpret_cast<const unsigned short*>(flag) + rec);
        return (f & 0xFF) == 0 || (f >> 8) == 0;
    }
    bool any = false;
    for (int p = 0; p < P; ++p) any |= (__ldg(flag + rec * P + p) == 0);
    return any;
}

// floor(a / d) for d > 0; a shift when d = 2^sh (sh >= 1)
__device__ __forceinline__ int floor_div32(int a, int d, int sh)
{
    if (sh > 0 && (d == (1 << sh))) return a >> sh;
    int q = a / d;
    if ((a % d != 0) && (a < 0)) --q;
    return q;
}

struct Placed {
    int4 info;   // {x0 | y0 << 16, cu | cv << 16, z, k | neg << kBitNeg | gd << kBitGd}
    int S;
};

// One row's coordinates rounded to float, and its take-conjugate flag (w' < 0, decided on the
// FP64 value).
struct RowF {
    float u, v, wa;     // fl32(u'), fl32(v'), fl32(|w'|)
    int neg;
};

__device__ __forceinline__ RowF row_f(const double* __restrict__ uvw, int64_t row)
{
    const double up = uvw[3 * row], vp = uvw[3 * row + 1], wp = uvw[3 * row + 2];
    const unsigned long long bw = __double_as_longlong(wp);
    const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
    RowF r;
    r.u = __double2float_rn(up);
    r.v = __double2float_rn(vp);
    r.wa = __double2float_rn(__longlong_as_double(bw & kAbs));
    r.neg = (bw >> 63) && (bw & kAbs) != 0 && (bw & kAbs) <= kInf;
    return r;
}

// q = ceil(t - 1/2) from the float estimate tf of t = fl64(u' sc): decided when no integer lies
// within the estimate's error bound of tf - 1/2.  |tf - t| <= |t| (3 + tiny) 2^-24 (three float
// roundings), and tf - 1/2 adds |tf| 2^-24; the margin |tf| 2^-20 + 2^-40 covers both.
__device__ __forceinline__ bool ceil_half_f(float tf, int& q)
{
    if (!(fabsf(tf) < 16777216.0f)) return false;              // large, infinite or NaN
    const float d = __fsub_rn(tf, 0.5f);
    const float c = ceilf(d);
    const float e = fabsf(tf) * 9.5367431640625e-07f + 9.094947e-13f;   // 2^-20 |tf| + 2^-40
    if (!(__fsub_rn(c, d) > e) || !(__fsub_rn(d, __fsub_rn(c, 1.0f)) > e)) return false;
    q = (int)c;
    return true;
}

// Placement decisions (q_u, q_v, plane k), FP64, each operation rounded once (no contraction).
// Returns false when the record is not griddable by position or plane.
__device__ __forceinline__ bool place_exact(const double* __restrict__ uvw, int64_t row, double lam_inv, double sc,
                                            bool neg, const PlaceParams& pp, int& iqu, int& iqv, int& k)
{
    const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
    const double up = uvw[3 * row], vp = uvw[3 * row + 1], wp = uvw[3 * row + 2];
    // (-a) b = -(a b) exactly, so flipping the sign of the scale negates tu, tv and w exactly
    const double scs = neg ? -sc : sc;
    const double tu = __dmul_rn(up, scs), tv = __dmul_rn(vp, scs);
    const double w = __dmul_rn(__longlong_as_double(__double_as_longlong(wp) & kAbs), lam_inv);
    // a NaN position is not griddable (a NaN w fails the plane test below)
    if ((__double_as_longlong(tu) & kAbs) > kInf || (__double_as_longlong(tv) & kAbs) > kInf) return false;
    // q = ceil(t - 1/2), converted with rounding toward +infinity in one instruction; the
    // conversion saturates (beyond qlim: off the grid)
    iqu = __double2int_ru(__dsub_rn(tu, 0.5));
    iqv = __double2int_ru(__dsub_rn(tv, 0.5));
    k = 0;
    if (pp.K > 1) {
        // nearest plane in sqrt(w): k = number of b_1..b_{K-1} with b_m <= w, griddable if w < b_K.
        // Compared first in FP32: float rounding is monotone, so fl(b) < fl(w) implies b < w and
        // fl(b) > fl(w) implies b > w; only bounds with fl(b) == fl(w) are compared in FP64.
        const float wf = __double2float_rn(w);
        const float fbK = __ldg(&pp.wbounds_f[pp.K - 1]);
        if (wf == fbK) {
            if (!(w < __ldg(&pp.wbounds[pp.K - 1]))) return false;
        } else if (!(wf < fbK)) {
            return false;                                     // beyond the last plane (or NaN)
        }
        int lo = 0, hi = pp.K - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&pp.wbounds_f[mid - 1]) < wf) lo = mid; else hi = mid - 1;
        }
        k = lo;
        while (k < pp.K - 1 && __ldg(&pp.wbounds_f[k]) == wf && w >= __ldg(&pp.wbounds[k])) ++k;
    }
    return true;
}

// Placement of one record.  The cell (q_u, q_v) and the plane k are decided from float
// estimates when the estimate's error bound cannot cross a rounding or plane boundary, which
// gives the same decisions as the FP64 steps (place_exact) that every other record takes.
// (lam_inv and sc are the channels' FP64 scales, read only by the exact steps; rec indexes the
// flags from `flag`, a 32-bit record index within a tile or a 64-bit one)
template <typename IDX>
__device__ __forceinline__ Placed place(const double* __restrict__ uvw, int64_t row, const RowF& rf,
                                        const double* __restrict__ lam_inv, const double* __restrict__ sc, int ch,
                                        float lam_f, float sc_f, const uint8_t* __restrict__ flag, IDX rec, int P,
                                        const PlaceParams& pp)
{
    Placed o;
    o.info = make_int4(0, 0, 0, rf.neg ? (1 << kBitNeg) : 0);
    o.S = 0;
    const bool unflagged = any_unflagged(flag, rec, P, pp.flag_vec);   // issued early: its latency overlaps the placement
    int iqu, iqv, k = 0;
    bool fast = false;
    {
        const float scs = rf.neg ? -sc_f : sc_f;
        fast = ceil_half_f(__fmul_rn(rf.u, scs), iqu) && ceil_half_f(__fmul_rn(rf.v, scs), iqv);
        if (fast && pp.K > 1) {
            // w = fl64(|w'| lam_inv) estimated as fl32(fl32(|w'|) fl32(lam_inv)); b_m <= w is
            // decided when fl32(b_m) lies outside w_f +- 2^-20 w_f (covers the estimate's three
            // roundings and the rounding of b_m to float)
            const float wf = __fmul_rn(rf.wa, lam_f);
            const float e = wf * 9.5367431640625e-07f;
            const float lo_w = __fsub_rn(wf, e), hi_w = __fadd_rn(wf, e);
            const float fbK = __ldg(&pp.wbounds_f[pp.K - 1]);
            if (!(hi_w < fbK)) {
                fast = false;            // near or beyond the last bound, infinite or NaN: exact steps
            } else {
                // the nearest plane in sqrt(w) directly, floor((K-1) sqrt(w / w_max) + 1/2), then
                // both of its bounds checked with the margin: b_k <= w < b_{k+1} decided, or the
                // exact steps (an estimate off by one near a bound fails the check)
                // (an estimate only, so the one-instruction approximate square root serves)
                float sw;
                asm("sqrt.approx.f32 %0, %1;" : "=f"(sw) : "f"(wf));
                int kk = __float2int_rd(fmaf(pp.kscale_f, sw, 0.5f));
                kk = min(max(kk, 0), pp.K - 1);
                if ((kk == 0 || __ldg(&pp.wbounds_f[kk - 1]) < lo_w) && __ldg(&pp.wbounds_f[kk]) > hi_w)
                    k = kk;
                else
                    fast = false;
            }
        }
    }
    if (!fast && !place_exact(uvw, row, lam_inv[ch], sc[ch], rf.neg, pp, iqu, iqv, k)) return o;
    if (iqu >= pp.qlim || iqu <= -pp.qlim || iqv >= pp.qlim || iqv <= -pp.qlim) return o;   // off the grid
    const int b = pp.beta;
    const int xc = floor_div32(2 * iqu + b - 1, 2 * b, pp.beta_log2 + 1);
    const int yc = floor_div32(2 * iqv + b - 1, 2 * b, pp.beta_log2 + 1);
    const int fu = iqu - b * xc, fv = iqv - b * yc;
    const int S = __ldg(&pp.supports[k]);
    const int h = (S - 1) / 2;
    const int x0 = pp.N / 2 + xc - h, y0 = pp.N / 2 + yc - h;
    if (x0 < 0 || y0 < 0 || x0 + S - 1 > pp.N - 1 || y0 + S - 1 > pp.N - 1) return o;
    if (!unflagged) return o;
    const int sub = (fv - pp.lo) * pp.beta + (fu - pp.lo);
    o.info.x = x0 | (y0 << 16);
    o.info.y = S;                      // the support, for the statistics (entries take the footprint's residues here)
    o.info.z = __ldg(&pp.offsets[k]) + sub * S * S;
    o.info.w |= k | (1 << kBitGd);
    o.S = S;
    return o;
}

__device__ __forceinline__ int nblk_of(int S, int slots)
{
    const int s2 = S * S;
    return (s2 + slots - 1) / slots;
}

}  // namespace

__global__ void k_chan_scale(const double* __restrict__ freq, int C, double beta_over_du, double* lam_inv,
                             double* sc, float* lam_f, float* sc_f)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double li = __ddiv_rn(freq[c], 299792458.0);
    const double s = __dmul_rn(li, beta_over_du);
    lam_inv[c] = li;
    sc[c] = s;
    lam_f[c] = __double2float_rn(li);
    sc_f[c] = __double2float_rn(s);
}

template <int P>
__global__ void __launch_bounds__(512, 3) k_classify(const double* __restrict__ uvw, const double* __restrict__ lam_inv,
                                                  const double* __restrict__ sc, const float* __restrict__ lam_f,
                                                  const float* __restrict__ sc_f, const uint8_t* __restrict__ flag,
                                                  int64_t rows, int rpb, PlaceParams pp, int4* __restrict__ rinfo,
                                                  uint8_t* __restrict__ rclass, int* __restrict__ tile_cnt,
                                                  unsigned long long* __restrict__ stat_priv)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int C = pp.C;
    const float inv_c = __frcp_rn((float)C);
    const int64_t tile = blockIdx.x;
    const int64_t row0 = tile * rpb;
    const int nrows = (int)min((int64_t)rpb, rows - row0);
    const int nrec = nrows * C;
    const int cap = rpb * C;
    int4* s_info = reinterpret_cast<int4*>(smem);
    int* s_cnt = reinterpret_cast<int*>(s_info + cap);             // [C]: gridded records per channel
    RowF* s_row = reinterpret_cast<RowF*>(s_cnt + cap + 1);        // [rpb + 1]: rows row0-1 ..
    __shared__ unsigned long long s_stat[ST_N];

    if (threadIdx.x < ST_N) s_stat[threadIdx.x] = 0ull;
    for (int ch = threadIdx.x; ch < C; ch += blockDim.x) s_cnt[ch] = 0;

    // pass 0: each row's coordinates as floats, once for all its channels
    for (int rr = threadIdx.x - 1; rr < nrows; rr += blockDim.x)
        if (row0 + rr >= 0) s_row[rr + 1] = row_f(uvw, row0 + rr);
    __syncthreads();

    // the records of this thread are j = threadIdx.x + i blockDim.x; their (row in the tile,
    // channel) pairs are stepped from one to the next, and global arrays are indexed from the
    // tile's first record with 32-bit offsets
    const int2 q0 = divmod_small(threadIdx.x, C, inv_c);
    const int2 dq = divmod_small(blockDim.x, C, inv_c);
    const uint8_t* flag_t = flag + row0 * C * P;

    // pass 1: placement
    {
        int rr = q0.x, ch = q0.y;
        for (int j = threadIdx.x; j < nrec; j += blockDim.x) {
            s_info[j] = place(uvw, row0 + rr, s_row[rr + 1], lam_inv, sc, ch, lam_f[ch], sc_f[ch], flag_t, j, P, pp).info;
            rr += dq.x;
            ch += dq.y;
            if (ch >= C) {
                ch -= C;
                ++rr;
            }
        }
    }
    __syncthreads();

    // pass 2: compression indicator, g, statistics and the outputs; the gridded records of each
    // channel (interleaved: of the tile) are counted for the tile offsets, and k_compact gives
    // each its rank in the tile
    // per thread at most cap / blockDim records, so the counts fit 32 bits, and so do warp sums
    unsigned n_gd = 0, n_g = 0, n_c = 0, u_g = 0, u_c = 0;
    {
        int4* rinfo_t = rinfo + row0 * C;
        uint8_t* rclass_t = rclass + row0 * C;
        int rr = q0.x, ch = q0.y;
        for (int j = threadIdx.x; j < nrec; j += blockDim.x) {
            int4 info = s_info[j];
            const int gd = (info.w >> kBitGd) & 1;
            int c = 0;
            // the predecessor: the previous row of the channel, or with interleaving the previous
            // record in natural order (the last channel of the previous row for channel 0)
            if (pp.compress && gd && (row0 + rr > 0 || (pp.interleave && j > 0))) {
                int4 pinfo;
                if (!pp.interleave && rr > 0) {
                    pinfo = s_info[j - C];
                } else if (pp.interleave && j > 0) {
                    pinfo = s_info[j - 1];
                } else {                          // the first row of the tile: the row before it
                    const int pc = pp.interleave ? C - 1 : ch;
                    pinfo = place(uvw, row0 - 1, s_row[0], lam_inv, sc, pc, lam_f[pc], sc_f[pc], flag_t, pc - C, P,
                                  pp).info;
                }
                c = ((pinfo.w >> kBitGd) & 1) && pinfo.x == info.x && pinfo.z == info.z;
            }
            const int g = gd & (c ^ 1);
            const int gc = g | (c << 1) | (gd << 2) | (((info.w >> kBitNeg) & 1) << 3);
            info.w |= (g << kBitG) | (c << kBitC);
            // k_compact reads the placement of gridded records and of the tile's first row (whose
            // compressed records carry a run on from the previous tile): only those are written
            if (g || j < C) rinfo_t[j] = info;
            rclass_t[j] = (uint8_t)gc;
            if (g) atomicAdd(&s_cnt[pp.interleave ? 0 : ch], 1);
            if (gd) {
                const unsigned S = (unsigned)info.y;
                n_gd += 1;
                n_g += g;
                n_c += c;
                u_g += g ? S * S : 0u;
                u_c += c ? S * S : 0u;
            }
            rr += dq.x;
            ch += dq.y;
            if (ch >= C) {
                ch -= C;
                ++rr;
            }
        }
    }
    // block statistics
    {
        const unsigned v[5] = {n_gd, n_g, n_c, u_g, u_c};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const unsigned x = __reduce_add_sync(0xffffffffu, v[q]);
            if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_stat[q + 1], (unsigned long long)x);
        }
    }
    __syncthreads();

    for (int ch = threadIdx.x; ch < C; ch += blockDim.x)   // interleaved: one list, channel 0's
        tile_cnt[tile * C + ch] = pp.interleave ? (ch == 0 ? s_cnt[0] : 0) : s_cnt[ch];
    const int slot = (int)(tile % kNormSlots);
    if (threadIdx.x == 0) s_stat[ST_RECORDS] = (unsigned long long)nrec;
    __syncthreads();
    if (threadIdx.x < ST_TASKS && s_stat[threadIdx.x])
        atomicAdd(&stat_priv[slot * ST_N + threadIdx.x], s_stat[threadIdx.x]);
}

// per-channel exclusive scan of tile counts over tiles
__global__ void __launch_bounds__(1024) k_scan_tiles(int* __restrict__ tile_cnt, int64_t n_tiles, int C,
                                                     int* __restrict__ chan_total)
{
    __shared__ int warp_tot[32];
    __shared__ int carry_s;
    const int ch = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (int64_t base = 0; base < n_tiles; base += blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const int v = (t < n_tiles) ? tile_cnt[t * C + ch] : 0;
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int x = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            warp_tot[lane] = x;
        }
        __syncthreads();
        const int excl = carry + inc - v + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (t < n_tiles) tile_cnt[t * C + ch] = excl;
        if (threadIdx.x == blockDim.x - 1) carry_s = carry + warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
        carry = carry_s;
        __syncthreads();
    }
    if (threadIdx.x == 0) chan_total[ch] = carry;
}

__global__ void k_finalize(int* __restrict__ chan_base, int C, const unsigned long long* __restrict__ stat_priv,
                           unsigned long long* __restrict__ stats, unsigned long long* __restrict__ stats_batch,
                           long long* __restrict__ scal, long long cap, int append)
{
    if (threadIdx.x == 0) {
        // channel bases and the entry count, held to the work list's capacity (a count past it
        // is reported as dropped); an appended batch's entries follow those already listed
        long long run = append ? scal[0] : 0;
        bool over = false;
        for (int c = 0; c < C; ++c) {
            const int t = chan_base[c];
            chan_base[c] = (int)run;
            run += t;
            if (t < 0 || run > cap) {
                over = true;
                run = t < 0 ? run - t : cap;
            }
        }
        chan_base[C] = (int)run;
        scal[0] = run;
        if (over) atomicAdd(reinterpret_cast<unsigned long long*>(&scal[3]), 1ull);
    }
    for (int q = threadIdx.x; q < ST_TASKS; q += blockDim.x) {
        unsigned long long s = 0;
        for (int k = 0; k < kNormSlots; ++k) s += stat_priv[k * ST_N + q];
        stats_batch[q] = s;
        stats[q] = append ? stats[q] + s : s;
    }
}

// visibility element -> complex float (half-precision values carry a per-channel scale)
__device__ __forceinline__ float2 vis_value(const float2* __restrict__ v, int64_t i, float) { return v[i]; }
__device__ __forceinline__ float2 vis_value(const __half2* __restrict__ v, int64_t i, float scale)
{
    const float2 f = __half22float2(v[i]);
    return make_float2(scale * f.x, scale * f.y);
}

// The input polarisation that grid polarisation p of a record takes: with cross-hand swapping a
// take-conjugate quad-pol record feeds pol 1 from pol 2 and pol 2 from pol 1.
__device__ __forceinline__ int src_pol(int p, bool neg, int cross_swap)
{
    return (cross_swap && neg && (p == 1 || p == 2)) ? 3 - p : p;
}

// weighted value eps (1-f) psi-conj(vis) of polarisation p of record rec, and eps (1-f)
template <typename VT>
__device__ __forceinline__ float2 weighted(const VT* __restrict__ vis, const float* __restrict__ weight,
                                          const uint8_t* __restrict__ flag, int64_t i, float scale, bool neg,
                                          int unweighted, float& wf)
{
    wf = unweighted ? 1.0f : weight[i] * (1.0f - (float)flag[i]);
    const float2 v = vis_value(vis, i, scale);
    return make_float2(wf * v.x, (neg ? -1.f : 1.f) * (wf * v.y));
}

// The same for all P polarisations of record rec with vector loads (vis 16-byte, weight
// 4P-byte and flag P-byte aligned).
template <int P>
__device__ __forceinline__ void weighted_vec(const float2* __restrict__ vis, const float* __restrict__ weight,
                                             const uint8_t* __restrict__ flag, int64_t rec, float, bool neg,
                                             int unweighted, int cross_swap, float2 (&q)[P], float (&wf)[P])
{
    float2 v[P];
    if constexpr (P == 1) {
        v[0] = vis[rec];
    } else {
#pragma unroll
        for (int h = 0; h < P; h += 2) {
            const float4 a = *reinterpret_cast<const float4*>(vis + rec * P + h);
            v[h] = make_float2(a.x, a.y);
            v[h + 1] = make_float2(a.z, a.w);
        }
    }
    float w[P];
    unsigned f = 0;
    if constexpr (P == 4) {
        const float4 a = *reinterpret_cast<const float4*>(weight + rec * 4);
        w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
        f = *reinterpret_cast<const unsigned*>(flag + rec * 4);
    } else if constexpr (P == 2) {
        const float2 a = *reinterpret_cast<const float2*>(weight + rec * 2);
        w[0] = a.x; w[1] = a.y;
        f = *reinterpret_cast<const unsigned short*>(flag + rec * 2);
    } else {
        w[0] = weight[rec];
        f = flag[rec];
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int ps = src_pol(p, neg, cross_swap);
        wf[p] = unweighted ? 1.0f : w[ps] * (1.0f - (float)((f >> (8 * ps)) & 0xFF));
        q[p] = make_float2(wf[p] * v[ps].x, (neg ? -1.f : 1.f) * (wf[p] * v[ps].y));
    }
}

template <int P>
__device__ __forceinline__ void weighted_vec(const __half2* __restrict__ vis, const float* __restrict__ weight,
                                             const uint8_t* __restrict__ flag, int64_t rec, float scale, bool neg,
                                             int unweighted, int cross_swap, float2 (&q)[P], float (&wf)[P])
{
#pragma unroll
    for (int p = 0; p < P; ++p)
        q[p] = weighted(vis, weight, flag, rec * P + src_pol(p, neg, cross_swap), scale, neg, unweighted, wf[p]);
}

// the P values and weights of one record from record-major arrays (shared or global memory),
// with vector loads: qp 8P-byte and wp 4P-byte aligned (P = 1: 8 and 4 bytes)
template <int P>
__device__ __forceinline__ void load_rec(const float2* __restrict__ qp, const float* __restrict__ wp, float2 (&q)[P],
                                         float (&w)[P])
{
    if constexpr (P == 4) {
        const float4 a = *reinterpret_cast<const float4*>(qp);
        const float4 b = *reinterpret_cast<const float4*>(qp + 2);
        const float4 c = *reinterpret_cast<const float4*>(wp);
        q[0] = make_float2(a.x, a.y); q[1] = make_float2(a.z, a.w);
        q[2] = make_float2(b.x, b.y); q[3] = make_float2(b.z, b.w);
        w[0] = c.x; w[1] = c.y; w[2] = c.z; w[3] = c.w;
    } else if constexpr (P == 2) {
        const float4 a = *reinterpret_cast<const float4*>(qp);
        const float2 c = *reinterpret_cast<const float2*>(wp);
        q[0] = make_float2(a.x, a.y); q[1] = make_float2(a.z, a.w);
        w[0] = c.x; w[1] = c.y;
    } else {
        q[0] = qp[0];
        w[0] = wp[0];
    }
}

// loads the P weighted values and weights of record j from the shared staging arrays:
// polarisation-major [P][cap], or record-major [cap][P] (AOS, the bulk-copied layout)
template <int P, bool AOS>
__device__ __forceinline__ void stage_load(const float2* __restrict__ s_q, const float* __restrict__ s_w, int cap, int j,
                                           float2 (&q)[P], float (&w)[P])
{
    if constexpr (AOS) {
        load_rec<P>(s_q + (size_t)j * P, s_w + (size_t)j * P, q, w);
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            q[p] = s_q[(size_t)p * cap + j];
            w[p] = s_w[(size_t)p * cap + j];
        }
    }
}

template <int P>
__device__ __forceinline__ void stage_store_aos(float2* __restrict__ s_q, float* __restrict__ s_w, int j,
                                                const float2 (&q)[P], const float (&w)[P])
{
    if constexpr (P == 4) {
        *reinterpret_cast<float4*>(s_q + j * 4) = make_float4(q[0].x, q[0].y, q[1].x, q[1].y);
        *reinterpret_cast<float4*>(s_q + j * 4 + 2) = make_float4(q[2].x, q[2].y, q[3].x, q[3].y);
        *reinterpret_cast<float4*>(s_w + j * 4) = make_float4(w[0], w[1], w[2], w[3]);
    } else if constexpr (P == 2) {
        *reinterpret_cast<float4*>(s_q + j * 2) = make_float4(q[0].x, q[0].y, q[1].x, q[1].y);
        *reinterpret_cast<float2*>(s_w + j * 2) = make_float2(w[0], w[1]);
    } else {
        s_q[j] = q[0];
        s_w[j] = w[0];
    }
}

// the P flag bytes of record rec in one load (flag pointer aligned to P bytes)
template <int P>
__device__ __forceinline__ unsigned flags_of(const uint8_t* __restrict__ flag, int64_t rec)
{
    if constexpr (P == 4) return __ldg(reinterpret_cast<const unsigned*>(flag) + rec);
    else if constexpr (P == 2) return __ldg(reinterpret_cast<const unsigned short*>(flag) + rec);
    else return __ldg(flag + rec);
}

// Writes one run of a channel sequence (or of the interleaved sequence): for a head of the given
// rank among the tile's gridded records of its list, its entry,
// gamma and run (first and last row, or record when interleaved); for the compressed records a
// tile starts with (a carry: the end of a run begun in an earlier tile), their sum in
// carry[tile][sequence] for k_carry.  Adds zeta(sub-kernel) x sum eps (1-f) to the normaliser.
template <int P>
__device__ __forceinline__ void emit_run(const int4& info, bool is_carry, int rank, int64_t tile, int C, int ch,
                                         int gch, int64_t first, int64_t last, const float2 (&acc)[P], const float (&wsum)[P],
                                         const PlaceParams& pp, float* s_norm, const int* __restrict__ tile_off,
                                         const int* __restrict__ chan_base, int4* __restrict__ entries,
                                         float2* __restrict__ gamma, int2* __restrict__ runs, int64_t cap_entries,
                                         float2* __restrict__ carry_q, int* __restrict__ carry_last,
                                         long long* __restrict__ scal)
{
    const int k = info.w & 0xFFF;
    const int S = __ldg(&pp.supports[k]);
    const int sub = (info.z - __ldg(&pp.offsets[k])) / (S * S);
    const float zeta = __ldg(&pp.zeta_f[k * pp.beta * pp.beta + sub]);
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (wsum[p] != 0.f) atomicAdd(&s_norm[gch * P + p], zeta * wsum[p]);
    if (is_carry) {
        const int64_t c = tile * C + gch;
#pragma unroll
        for (int p = 0; p < P; ++p) carry_q[c * P + p] = acc[p];
        carry_last[c] = (int)last;
        return;
    }
    const int dst = chan_base[gch] + tile_off[tile * C + gch] + rank;
    if (dst < 0 || (int64_t)dst >= cap_entries) {   // cannot happen with a consistent scan
        atomicAdd(reinterpret_cast<unsigned long long*>(&scal[3]), 1ull);
        return;
    }
    const int ech = pp.wstack ? ch * pp.K + k : gch + pp.chan0;   // the grid channel
    // (-x0) mod S and (-y0) mod S: the residue classes of the footprint's first column and row
    const float inv_s = __frcp_rn((float)S);
    const int rx = mod_small(info.x & 0xFFFF, S, inv_s), ry = mod_small((info.x >> 16) & 0xFFFF, S, inv_s);
    const int cuv = (rx ? S - rx : 0) | ((ry ? S - ry : 0) << 16);
    entries[dst] = make_int4(info.x, cuv, info.z, k | (ech << 16));
#pragma unroll
    for (int p = 0; p < P; ++p) gamma[(int64_t)dst * P + p] = acc[p];
    runs[dst] = make_int2((int)first, (int)last);
}

// One block per tile.  Pass 1 stages the tile's records in shared memory: eps (1-f)
// psi-conj(vis) and eps (1-f) per polarisation, and lists the tile's gridded records.  With
// BULK (FP32 visibilities, 16-byte aligned tiles) the tile's visibilities and weights arrive
// by bulk asynchronous copies (TMA) into record-major staging arrays, issued before anything
// else, while the threads read the class bytes and flags; each thread then weighs its records
// in place.  Otherwise every record is read with vector loads into polarisation-major arrays.
// Pass 2: each listed record sums its run of compressed successors (same channel, following
// rows) from shared memory in row order, continuing into the following tiles through global
// memory when the run crosses the tile's end; it writes its entry, gamma and run, and adds
// zeta(sub-kernel) x sum eps (1-f) to the normaliser (all records of a run share the
// sub-kernel).
template <int P, typename VT, bool IL, bool BULK>
__global__ void __launch_bounds__(kCompactThreads, 2) k_compact(const int4* __restrict__ rinfo, const uint8_t* __restrict__ rclass,
                                                 const VT* __restrict__ vis, const float* __restrict__ vis_scale,
                                                 const float* __restrict__ weight, const uint8_t* __restrict__ flag,
                                                 int64_t rows, int rpb, int C, const int* __restrict__ tile_off,
                                                 const int* __restrict__ chan_base, PlaceParams pp,
                                                 int4* __restrict__ entries, float2* __restrict__ gamma,
                                                 int2* __restrict__ runs, int64_t cap_entries,
                                                 double* __restrict__ norm_priv, float2* __restrict__ carry_q,
                                                 int* __restrict__ carry_last, long long* __restrict__ scal, int vec)
{
    static_assert(!BULK || std::is_same<VT, float2>::value, "bulk staging takes FP32 visibilities");
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t tile = blockIdx.x;
    const int64_t row0 = tile * rpb;
    const int nrows = (int)min((int64_t)rpb, rows - row0);
    const int nrec = nrows * C;
    const int cap = rpb * C;
    float2* s_q = reinterpret_cast<float2*>(smem);                        // [P][cap] or [cap][P]
    float* s_w = reinterpret_cast<float*>(s_q + (size_t)cap * P);         // [P][cap] or [cap][P]
    float* s_norm = s_w + (size_t)cap * P;                                // [C][P]
    int* s_heads = reinterpret_cast<int*>(s_norm + (size_t)C * P);        // [cap]
    uint8_t* s_cls = reinterpret_cast<uint8_t*>(s_heads + cap);           // [cap]
    int* s_first = reinterpret_cast<int*>(s_cls + ((cap + 3) & ~3));     // [C]: list position of each channel's first head
    __shared__ int s_wtot[kCompactThreads / 32];
    __shared__ int s_abort;
    __shared__ unsigned long long s_bar;
    const int unweighted = pp.unweighted;

    // the bulk copies cover whole 16-byte units of the tile's visibilities and weights; a
    // ragged last tile reads its remaining records directly
    const unsigned bytes_v = BULK ? ((unsigned)nrec * P * 8u) & ~15u : 0u;
    const unsigned bytes_w = BULK ? ((unsigned)nrec * P * 4u) & ~15u : 0u;
    if constexpr (BULK) {
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) {
                mbar_init(&s_bar, 1);
                mbar_arrive_expect(&s_bar, bytes_v + bytes_w);
            }
            __syncwarp();
            const unsigned nv = (bytes_v + kBulkChunk - 1) / kBulkChunk, nw = (bytes_w + kBulkChunk - 1) / kBulkChunk;
            const char* gv = reinterpret_cast<const char*>(vis + row0 * C * P);
            const char* gw = reinterpret_cast<const char*>(weight + row0 * C * P);
            for (unsigned i = threadIdx.x; i < nv + nw; i += 32) {
                const bool isv = i < nv;
                const unsigned off = (isv ? i : i - nv) * kBulkChunk;
                const unsigned tot = isv ? bytes_v : bytes_w;
                bulk_to_smem(reinterpret_cast<char*>(isv ? (void*)s_q : (void*)s_w) + off, (isv ? gv : gw) + off,
                             min(kBulkChunk, tot - off), &s_bar);
            }
        }
    }
    if (threadIdx.x == 0) s_abort = 0;
    for (int i = threadIdx.x; i < C * P; i += blockDim.x) s_norm[i] = 0.f;
    __syncthreads();
    if constexpr (BULK) {
        constexpr int kU = 4;                    // records per thread whose class and flag loads are issued together
        bool waited = false, ok = true;
        for (int j0 = threadIdx.x; j0 < nrec; j0 += kU * blockDim.x) {
            int cls[kU];
            unsigned fl[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int j = j0 + u * (int)blockDim.x;
                cls[u] = 0;
                fl[u] = 0u;
                if (j < nrec) {
                    const int64_t rec = row0 * C + j;
                    cls[u] = rclass[rec];
                    fl[u] = flags_of<P>(flag, rec);
                }
            }
            if (!waited) {
                waited = true;
                ok = mbar_wait(&s_bar, 0, kWaitLimitNs);
                if (!ok) s_abort = 1;
            }
            if (!ok) continue;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int j = j0 + u * (int)blockDim.x;
                if (j >= nrec) continue;
                const int c = cls[u];
                s_cls[j] = (uint8_t)c;
                if (!(c & 4)) continue;                  // not griddable
                const int64_t rec = row0 * C + j;
                float2 v[P];
                float w[P];
                if ((unsigned)(j + 1) * P * 8u <= bytes_v && (unsigned)(j + 1) * P * 4u <= bytes_w)
                    stage_load<P, true>(s_q, s_w, cap, j, v, w);
                else                                             // the ragged end of the last tile
                    load_rec<P>(vis + rec * P, weight + rec * P, v, w);
                const bool neg = (c >> 3) & 1;
                unsigned f = fl[u];
                if constexpr (P == 4) {
                    // cross-hand swap (src_pol) with static indices: pol 1 takes pol 2's input and back
                    if (pp.cross_swap && neg) {
                        const float2 tv = v[1];
                        v[1] = v[2];
                        v[2] = tv;
                        const float tw = w[1];
                        w[1] = w[2];
                        w[2] = tw;
                        f = (f & 0xFF0000FFu) | ((f >> 8) & 0x0000FF00u) | ((f << 8) & 0x00FF0000u);
                    }
                }
                float2 q[P];
                float wf[P];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    wf[p] = unweighted ? 1.0f : w[p] * (1.0f - (float)((f >> (8 * p)) & 0xFFu));
                    q[p] = make_float2(wf[p] * v[p].x, (neg ? -1.f : 1.f) * (wf[p] * v[p].y));
                }
                stage_store_aos<P>(s_q, s_w, j, q, wf);
            }
        }
    } else {
        for (int j = threadIdx.x; j < nrec; j += blockDim.x) {
            const int64_t rec = row0 * C + j;
            const int cls = rclass[rec];
            s_cls[j] = (uint8_t)cls;
            if (!(cls & 4)) continue;                       // not griddable
            const float scale = vis_scale ? vis_scale[j % C] : 1.0f;
            const bool neg = (cls >> 3) & 1;
            if (vec) {
                float2 q[P];
                float wf[P];
                weighted_vec<P>(vis, weight, flag, rec, scale, neg, unweighted, pp.cross_swap, q, wf);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    s_q[(size_t)p * cap + j] = q[p];
                    s_w[(size_t)p * cap + j] = wf[p];
                }
            } else {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    float wf;
                    s_q[(size_t)p * cap + j] = weighted(vis, weight, flag, rec * P + src_pol(p, neg, pp.cross_swap),
                                                        scale, neg, unweighted, wf);
                    s_w[(size_t)p * cap + j] = wf;
                }
            }
        }
    }
    __syncthreads();
    if (BULK && s_abort) {                 // a bulk copy did not complete in time: nothing of the tile is written
        if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&scal[3]), 1ull);
        for (int i = threadIdx.x; i < C; i += blockDim.x) carry_last[tile * C + i] = -1;
        mbar_wait(&s_bar, 0, kWaitLimitNs);       // copies still in flight land before the block exits
        return;
    }

    // the tile's gridded records listed channel-major (interleaved: in natural order), which is
    // the order of their entries: a block scan of their flags gives each one its list position,
    // and its rank in its channel's list is that position less the channel's first one
    int nh;
    {
        const int T = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
        const int ept = (nrec + T - 1) / T;                  // list elements per thread
        const int k0 = min(nrec, t * ept), k1 = min(nrec, k0 + ept);
        const float inv_n = __frcp_rn((float)nrows);
        const int2 e0 = IL ? make_int2(0, 0) : divmod_small(k0, nrows, inv_n);   // (channel, row) of element k0
        int cnt = 0;
        {
            int ch = e0.x, rr = e0.y;
            for (int k = k0; k < k1; ++k) {
                cnt += s_cls[IL ? k : rr * C + ch] & 1;
                if (++rr == nrows) {
                    rr = 0;
                    ++ch;
                }
            }
        }
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) s_wtot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            const int nw = T >> 5;
            int v = lane < nw ? s_wtot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (lane < nw) s_wtot[lane] = v;                 // inclusive over warps
        }
        __syncthreads();
        int pos = inc - cnt + (wid > 0 ? s_wtot[wid - 1] : 0);
        {
            int ch = e0.x, rr = e0.y;
            for (int k = k0; k < k1; ++k) {
                const int j = IL ? k : rr * C + ch;
                if (!IL && rr == 0) s_first[ch] = pos;
                if (s_cls[j] & 1) s_heads[pos++] = j;
                if (++rr == nrows) {
                    rr = 0;
                    ++ch;
                }
            }
        }
        nh = s_wtot[(T >> 5) - 1];
        __syncthreads();
    }

    // pass 2: work items are the tile's gridded records (runs summed inside the tile) and, per
    // sequence (channel; the one natural-order sequence when interleaved), the compressed
    // records the tile starts with, which continue a run of an earlier tile: their sum is left
    // in carry[tile][sequence] for k_carry to add to that run's entry.  A run is walked with the
    // next record's class and values loaded together (one shared-memory latency per record).
    const int n_seq = IL ? 1 : C;
    for (int h = threadIdx.x; h < nh + n_seq; h += blockDim.x) {
        const bool is_carry = h >= nh;
        const int j = is_carry ? h - nh : s_heads[h];          // a carry starts at the sequence's first record
        const int rr = j / C, ch = j - rr * C;
        const int64_t row = row0 + rr, rec = row * C + ch;
        const int gch = IL ? 0 : ch;                           // the work-list list (and normaliser row)
        if (is_carry && !(s_cls[j] & 2)) {                     // no run continues into this tile
            carry_last[tile * C + gch] = -1;
            continue;
        }
        const int4 info = rinfo[rec];
        float2 acc[P];
        float wsum[P];
        stage_load<P, BULK>(s_q, s_w, cap, j, acc, wsum);
        // the run inside the tile: successors (next rows of the channel, or next records when
        // interleaved) while compressed; `last` is its last row (interleaved: record)
        const int step = IL ? 1 : C;
        const int jend = IL ? nrec : nrows * C;
        int j2 = j + step, jl = j;
        if (j2 < jend) {
            int c2 = s_cls[j2];
            float2 q[P];
            float w[P];
            stage_load<P, BULK>(s_q, s_w, cap, j2, q, w);
            while (c2 & 2) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    acc[p].x += q[p].x;
                    acc[p].y += q[p].y;
                    wsum[p] += w[p];
                }
                jl = j2;
                j2 += step;
                if (j2 >= jend) break;
                c2 = s_cls[j2];
                stage_load<P, BULK>(s_q, s_w, cap, j2, q, w);
            }
        }
        const int64_t last = IL ? row0 * C + jl : row0 + jl / C;
        const int rank = is_carry ? 0 : (IL ? h : h - s_first[ch]);
        emit_run<P>(info, is_carry, rank, tile, C, ch, gch, IL ? rec : row, last, acc, wsum, pp, s_norm, tile_off,
                    chan_base, entries, gamma, runs, cap_entries, carry_q, carry_last, scal);
    }
    __syncthreads();
    const int slot = (int)(tile % kNormSlots);
    for (int i = threadIdx.x; i < C * P; i += blockDim.x)
        if (s_norm[i] != 0.f) atomicAdd(&norm_priv[(int64_t)slot * C * P + i], (double)s_norm[i]);
}

// adds each tile's carried run part (compressed records continuing a run of an earlier tile) to
// that run's entry, the last entry of the sequence before the tile, and extends the run's end
template <int P>
__global__ void k_carry(const float2* __restrict__ carry_q, const int* __restrict__ carry_last, int64_t n_tiles, int C,
                        int n_seq, const int* __restrict__ tile_off, const int* __restrict__ chan_base,
                        float2* __restrict__ gamma, int2* __restrict__ runs, int64_t cap_entries,
                        long long* __restrict__ scal)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // tile * C + sequence
    if (c >= n_tiles * C) return;
    const int seq = (int)(c % C);
    if (seq >= n_seq) return;                            // interleaved: one sequence per tile
    const int last = carry_last[c];
    if (last < 0) return;
    const int64_t dst = (int64_t)chan_base[seq] + tile_off[c] - 1;
    if (dst < chan_base[seq] || dst >= cap_entries) {   // cannot happen: a compressed record follows its run's head
        atomicAdd(reinterpret_cast<unsigned long long*>(&scal[3]), 1ull);
        return;
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float2 q = carry_q[c * P + p];
        atomicAdd(&gamma[dst * P + p].x, q.x);
        atomicAdd(&gamma[dst * P + p].y, q.y);
    }
    atomicMax(reinterpret_cast<int*>(&runs[dst]) + 1, last);
}

// N_p of the batch: the sum of the privatised per-slot partials
__global__ void k_norm_sum(const double* __restrict__ norm_priv, int n, double* __restrict__ norm_batch)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < kNormSlots; ++k) s += norm_priv[(int64_t)k * n + i];
        norm_batch[i] = s;
    }
}

// per segment, the number of task blocks of its largest support; sets the segment count
__global__ void k_segments(const int4* __restrict__ entries, long long* __restrict__ scal,
                           const int* __restrict__ supports, int K, int seg_len, int slots,
                           int* __restrict__ seg_nblk)
{
    const long long n = scal[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[2] = (n + seg_len - 1) / seg_len;
    // seg_len is a multiple of 32, so the 32 entries of a warp's chunk share one segment: the
    // warp takes their maximum and one lane updates the segment
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp0 * 32; base < n; base += n_warps * 32) {
        const long long e = base + lane;
        int nb = 0;
        if (e < n) {
            const int k = entries[e].w & 0xFFF;
            nb = (k < K) ? nblk_of(__ldg(&supports[k]), slots) : 1;
        }
        const int m = __reduce_max_sync(0xffffffffu, nb);
        if (lane == 0) atomicMax(&seg_nblk[base / seg_len], m);
    }
}

__global__ void __launch_bounds__(1024) k_seg_scan(const int* __restrict__ seg_nblk, int* __restrict__ seg_off,
                                                   long long* __restrict__ scal, unsigned long long* __restrict__ stats)
{
    __shared__ int warp_tot[32];
    __shared__ int carry_s;
    const long long n_seg = scal[2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (long long base = 0; base < n_seg; base += blockDim.x) {
        const long long t = base + threadIdx.x;
        const int v = (t < n_seg) ? seg_nblk[t] : 0;
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int x = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            warp_tot[lane] = x;
        }
        __syncthreads();
        const int excl = carry + inc - v + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (t < n_seg) seg_off[t] = excl;
        if (threadIdx.x == blockDim.x - 1) carry_s = carry + warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
        carry = carry_s;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        seg_off[n_seg] = carry;
        scal[1] = carry;
        stats[ST_TASKS] = (unsigned long long)carry;
    }
}

static size_t classify_smem(int rpb, int C)
{
    const size_t cap = (size_t)rpb * C;
    return cap * sizeof(int4) + (cap + 1) * sizeof(int) + (rpb + 1) * 16 + cap + 16;
}

static size_t compact_smem(int rpb, int C, int P)
{
    const size_t cap = (size_t)rpb * C;
    return cap * P * (sizeof(float2) + sizeof(float)) + (size_t)C * P * sizeof(float) + cap * sizeof(int) +
           ((cap + 3) & ~(size_t)3) + (size_t)C * sizeof(int) + 16;
}

static PlaceParams place_params(const Table& t, int n, double du, int C, int P, int flags)
{
    PlaceParams pp;
    pp.N = n;
    pp.beta = t.beta;
    pp.K = t.K;
    pp.lo = -((t.beta - 1) / 2);
    pp.compress = (flags & WG_PREP_COMPRESS) ? 1 : 0;
    pp.unweighted = (flags & WG_PREP_UNWEIGHTED) ? 1 : 0;
    pp.interleave = (flags & WG_PREP_INTERLEAVE) ? 1 : 0;
    pp.cross_swap = (flags & WG_PREP_CROSS_SWAP) && P == 4 ? 1 : 0;
    pp.wstack = (flags & WG_PREP_WSTACK) ? 1 : 0;
    pp.C = C;
    pp.P = P;
    pp.w_max = t.w_max;
    pp.beta_over_du = (double)t.beta / du;
    pp.supports = t.supports_d;
    pp.offsets = t.offsets_d;
    pp.wbounds = t.wbounds_d;
    pp.wbounds_f = t.wbounds_f;
    pp.qlim = t.beta * (n / 2 + 2);
    pp.beta_log2 = -1;
    for (int b = 0; b < 16; ++b)
        if (t.beta == (1 << b)) pp.beta_log2 = b;
    pp.zeta_f = t.zeta_f;
    pp.flag_vec = 0;
    pp.kscale_f = (t.K > 1 && t.w_max > 0.0) ? (float)((t.K - 1) / std::sqrt(t.w_max)) : 0.0f;
    pp.chan0 = 0;
    return pp;
}

template <int P>
static int prep_impl(const Table& t, const Grid& g, const wg_vis_in& in, int flags, WorkList& wl,
                     cudaStream_t s)
{
    const int C = in.n_chan;
    const int64_t rows = in.n_rows;
    if (in.vis_dtype != WG_VIS_COMPLEX64 && in.vis_dtype != WG_VIS_COMPLEX_HALF)
        return fail(WG_E_INVALID_ARG, "unknown vis_dtype %d", in.vis_dtype);
    if (in.vis_dtype == WG_VIS_COMPLEX_HALF && rows > 0 && !in.vis_scale)
        return fail(WG_E_INVALID_ARG, "vis_scale is required for half-precision visibilities");
    const int rpb = std::max(1, kTileRecords / C);
    const int64_t n_tiles = (rows + rpb - 1) / rpb;
    if ((n_tiles + 1) * C > wl.tile_cap) return fail(WG_E_CAPACITY, "too many tiles for this work list");
    wl.rows = rows;
    wl.rpb = rpb;
    wl.n_tiles = n_tiles;
    wl.N = g.n;

    const bool app = (flags & WG_PREP_APPEND) != 0;
    PlaceParams pp = place_params(t, g.n, g.du, C, P, flags);
    pp.flag_vec = (reinterpret_cast<uintptr_t>(in.flag) % P) == 0;
    pp.chan0 = app ? in.chan0 : 0;
    wl.interleave = pp.interleave != 0;
    wl.cross_swap = pp.cross_swap != 0;
    wl.wstack_k = pp.wstack ? t.K : 1;
    wl.chan_hi = app ? std::max(wl.append ? wl.chan_hi : 0, in.chan0 + C) : 0;
    wl.append = app;

    double* lam_inv = reinterpret_cast<double*>(wl.norm_batch + (size_t)C * P);   // [C]
    double* sc = lam_inv + C;                                                     // [C]
    float* lam_f = reinterpret_cast<float*>(sc + C);                              // [C]
    float* sc_f = lam_f + C;                                                      // [C]

    WG_CUDA(cudaMemsetAsync(wl.norm_priv, 0, sizeof(double) * kNormSlots * C * P, s));
    WG_CUDA(cudaMemsetAsync(wl.stat_priv, 0, sizeof(unsigned long long) * kNormSlots * ST_N, s));
    if (app) {
        // keep the entry count and the dropped count of the earlier batches; the plan is redone
        WG_CUDA(cudaMemsetAsync(wl.scal + 1, 0, sizeof(long long) * 2, s));
    } else {
        WG_CUDA(cudaMemsetAsync(wl.stats, 0, sizeof(unsigned long long) * ST_N, s));
        WG_CUDA(cudaMemsetAsync(wl.scal, 0, sizeof(long long) * 4, s));
    }

    k_chan_scale<<<(C + 127) / 128, 128, 0, s>>>(in.freq_hz, C, pp.beta_over_du, lam_inv, sc, lam_f, sc_f);
    WG_LAUNCHED("k_chan_scale");
    if (rows > 0) {
        const size_t sm = classify_smem(rpb, C);
        if (sm > 48 * 1024) WG_CUDA(cudaFuncSetAttribute(k_classify<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_classify<P><<<(unsigned)n_tiles, 512, sm, s>>>(in.uvw, lam_inv, sc, lam_f, sc_f, in.flag, rows, rpb, pp,
                                                          wl.rinfo, wl.rclass, wl.tile_cnt, wl.stat_priv);
        WG_LAUNCHED("k_classify");
    }
    k_scan_tiles<<<C, 1024, 0, s>>>(wl.tile_cnt, n_tiles, C, wl.chan_base);
    WG_LAUNCHED("k_scan_tiles");
    k_finalize<<<1, 256, 0, s>>>(wl.chan_base, C, wl.stat_priv, wl.stats, wl.stats_batch, wl.scal, wl.ecap, app ? 1 : 0);
    WG_LAUNCHED("k_finalize");
    if (rows > 0) {
        const size_t sm = compact_smem(rpb, C, P);
        const uintptr_t va = reinterpret_cast<uintptr_t>(in.vis), wa = reinterpret_cast<uintptr_t>(in.weight),
                        fa = reinterpret_cast<uintptr_t>(in.flag);
        const int vec = (va % 16 == 0) && (wa % (4 * P) == 0) && (fa % P == 0);
        if (sm > 227 * 1024)
            return fail(WG_E_CAPACITY, "%d channels x %d polarisations do not fit one preparation tile", C, P);
        // bulk staging: FP32 visibilities and weights whose every tile starts on a 16-byte boundary,
        // at four polarisations (52 bytes a record).  At one polarisation (13 bytes a record) the
        // per-record loads of four blocks per SM measured faster: 5.0 against 6.7 ms a launch of
        // 470 M records.
        const bool bulk = P == 4 && in.vis_dtype == WG_VIS_COMPLEX64 && vec && va % 16 == 0 && wa % 16 == 0 &&
                          ((int64_t)rpb * C * P) % 4 == 0;
        auto launch = [&](auto vt, auto il, auto bk) -> int {
            using VT = decltype(vt);
            constexpr bool IL = decltype(il)::value;
            constexpr bool BULK = decltype(bk)::value;
            if (sm > 48 * 1024)
                WG_CUDA(cudaFuncSetAttribute(k_compact<P, VT, IL, BULK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm));
            k_compact<P, VT, IL, BULK><<<(unsigned)n_tiles, kCompactThreads, sm, s>>>(
                wl.rinfo, wl.rclass, reinterpret_cast<const VT*>(in.vis),
                std::is_same<VT, float2>::value ? nullptr : in.vis_scale, in.weight, in.flag, rows, rpb,
                C, wl.tile_cnt, wl.chan_base, pp, wl.entries, wl.gamma, wl.runs, wl.ecap, wl.norm_priv, wl.carry_q,
                wl.carry_last, wl.scal, std::is_same<VT, float2>::value ? vec : 0);
            return WG_OK;
        };
        int rc;
        using T = std::true_type;
        using F = std::false_type;
        if (in.vis_dtype == WG_VIS_COMPLEX_HALF)
            rc = pp.interleave ? launch(__half2{}, T{}, F{}) : launch(__half2{}, F{}, F{});
        else if (bulk)
            rc = pp.interleave ? launch(float2{}, T{}, T{}) : launch(float2{}, F{}, T{});
        else
            rc = pp.interleave ? launch(float2{}, T{}, F{}) : launch(float2{}, F{}, F{});
        if (rc != WG_OK) return rc;
        WG_LAUNCHED("k_compact");
    }
    if (rows > 0) {
        const int64_t nc = n_tiles * C;
        k_carry<P><<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(wl.carry_q, wl.carry_last, n_tiles, C,
                                                                 pp.interleave ? 1 : C, wl.tile_cnt, wl.chan_base,
                                                                 wl.gamma, wl.runs, wl.ecap, wl.scal);
        WG_LAUNCHED("k_carry");
    }
    k_norm_sum<<<1, 256, 0, s>>>(wl.norm_priv, C * P, wl.norm_batch);
    WG_LAUNCHED("k_norm_sum");
    if (app) {
        // the batch's N_p terms and statistics go into its grid channels now; the plan over
        // every appended batch is made by the next grid_vis (or worklist_plan)
        wl.plan_stale = true;
        return launch_accumulate(g, wl, in.chan0, s);
    }
    wl.plan_stale = false;
    return launch_plan(t, wl, s);
}

int launch_plan(const Table& t, WorkList& wl, cudaStream_t s)
{
    const int64_t n_seg_max = (wl.ecap + wl.seg_len - 1) / wl.seg_len + 1;
    WG_CUDA(cudaMemsetAsync(wl.seg_nblk, 0, sizeof(int) * std::min<int64_t>(n_seg_max, wl.seg_cap), s));
    k_segments<<<num_sms() * 4, 256, 0, s>>>(wl.entries, wl.scal, t.supports_d, t.K, wl.seg_len, wl.slots,
                                              wl.seg_nblk);
    WG_LAUNCHED("k_segments");
    k_seg_scan<<<1, 1024, 0, s>>>(wl.seg_nblk, wl.seg_off, wl.scal, wl.stats);
    WG_LAUNCHED("k_seg_scan");
    return WG_OK;
}

// ---- uniform and robust weighting (the thesis names the schemes, Sec. 2.1; it grids with
// natural weights) -----------------------------------------------------------------------
// density W_p(cell) = sum of eps_p (1 - f_p) of the griddable records in the grid cell of their
// placement; uniform eps' = eps / W; robust (Briggs) eps' = eps / (1 + W f^2) with
// f^2 = (5 10^-R)^2 / (sum_cells W^2 / sum eps (1 - f)).  Records that are not griddable keep eps.

// the grid cell (x, y) of a griddable record, from its footprint origin
__device__ __forceinline__ int2 cell_of(const int4& info, const int* __restrict__ supports)
{
    const int h = (__ldg(&supports[info.w & 0xFFF]) - 1) / 2;
    return make_int2((info.x & 0xFFFF) + h, ((info.x >> 16) & 0xFFFF) + h);
}

template <int P>
__global__ void __launch_bounds__(256) k_density(const double* __restrict__ uvw, const double* __restrict__ lam_inv,
                                                 const double* __restrict__ sc, const float* __restrict__ lam_f,
                                                 const float* __restrict__ sc_f, const float* __restrict__ weight,
                                                 const uint8_t* __restrict__ flag, int64_t rows, PlaceParams pp,
                                                 float* __restrict__ dens, double* __restrict__ sums)
{
    __shared__ double s_w[P];
    if (threadIdx.x < P) s_w[threadIdx.x] = 0.0;
    __syncthreads();
    const int C = pp.C;
    const int64_t n = rows * C;
    double acc[P] = {};
    for (int64_t rec = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; rec < n; rec += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = rec / C;
        const int ch = (int)(rec - row * C);
        const int4 info = place(uvw, row, row_f(uvw, row), lam_inv, sc, ch, lam_f[ch], sc_f[ch], flag, rec, P, pp).info;
        if (!((info.w >> kBitGd) & 1)) continue;
        const int2 xy = cell_of(info, pp.supports);
        const int gc = pp.interleave ? 0 : ch;
        float* d = dens + (((size_t)gc * pp.N + xy.y) * pp.N + xy.x) * P;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float wf = weight[rec * P + p] * (1.0f - (float)flag[rec * P + p]);
            if (wf != 0.f) atomicAdd(d + p, wf);
            acc[p] += wf;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        double x = acc[p];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x != 0.0) atomicAdd(&s_w[p], x);
    }
    __syncthreads();
    if (threadIdx.x < P && s_w[threadIdx.x] != 0.0) atomicAdd(&sums[threadIdx.x], s_w[threadIdx.x]);
}

// sums[P + p] += sum over cells of W_p^2
template <int P>
__global__ void __launch_bounds__(256) k_density_sq(const float* __restrict__ dens, int64_t n_cells,
                                                    double* __restrict__ sums)
{
    __shared__ double s_q[P];
    if (threadIdx.x < P) s_q[threadIdx.x] = 0.0;
    __syncthreads();
    double acc[P] = {};
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const double v = dens[c * P + p];
            acc[p] += v * v;
        }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        double x = acc[p];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x != 0.0) atomicAdd(&s_q[p], x);
    }
    __syncthreads();
    if (threadIdx.x < P && s_q[threadIdx.x] != 0.0) atomicAdd(&sums[P + threadIdx.x], s_q[threadIdx.x]);
}

template <int P>
__global__ void __launch_bounds__(256) k_reweight(const double* __restrict__ uvw, const double* __restrict__ lam_inv,
                                                  const double* __restrict__ sc, const float* __restrict__ lam_f,
                                                  const float* __restrict__ sc_f, const float* __restrict__ weight,
                                                  const uint8_t* __restrict__ flag, int64_t rows, PlaceParams pp,
                                                  const float* __restrict__ dens, const double* __restrict__ sums,
                                                  int scheme, double robust_f0, float* __restrict__ out)
{
    const int C = pp.C;
    const int64_t n = rows * C;
    double f2[P];
#pragma unroll
    for (int p = 0; p < P; ++p) f2[p] = (sums[P + p] > 0.0) ? robust_f0 * robust_f0 * sums[p] / sums[P + p] : 0.0;
    for (int64_t rec = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; rec < n; rec += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = rec / C;
        const int ch = (int)(rec - row * C);
        const int4 info = place(uvw, row, row_f(uvw, row), lam_inv, sc, ch, lam_f[ch], sc_f[ch], flag, rec, P, pp).info;
        const bool gd = (info.w >> kBitGd) & 1;
        const float* d = nullptr;
        if (gd) {
            const int2 xy = cell_of(info, pp.supports);
            d = dens + ((((size_t)(pp.interleave ? 0 : ch)) * pp.N + xy.y) * pp.N + xy.x) * P;
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float w = weight[rec * P + p];
            float o = w;
            if (gd) {
                const double W = d[p];
                if (scheme == WG_WEIGHT_UNIFORM) o = (W > 0.0) ? (float)((double)w / W) : 0.f;
                else o = (float)((double)w / (1.0 + W * f2[p]));
            }
            out[rec * P + p] = o;
        }
    }
}

template <int P>
static int weight_impl(const Table& t, const Grid& g, const wg_vis_in& in, int scheme, double robust, int flags,
                       float* out, cudaStream_t s)
{
    const int C = in.n_chan;
    const int64_t rows = in.n_rows;
    PlaceParams pp = place_params(t, g.n, g.du, C, P, flags);
    pp.flag_vec = (reinterpret_cast<uintptr_t>(in.flag) % P) == 0;
    const int gc = pp.interleave ? 1 : C;
    const int64_t n_cells = (int64_t)gc * g.n * g.n;
    const size_t bytes = sizeof(float) * (size_t)n_cells * P + sizeof(double) * (4 * C + 2 * P);
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(WG_E_OOM, "cannot allocate the weight-density grid (%zu bytes)", bytes);
    }
    float* dens = static_cast<float*>(scratch);
    double* lam_inv = reinterpret_cast<double*>(dens + (size_t)n_cells * P);
    double* sc = lam_inv + C;
    double* sums = sc + C;                                   // [2P]: sum eps (1-f), sum W^2
    float* lam_f = reinterpret_cast<float*>(sums + 2 * P);
    float* sc_f = lam_f + C;
    int rc = WG_OK;
    if (cudaMemsetAsync(scratch, 0, sizeof(float) * (size_t)n_cells * P, s) != cudaSuccess ||
        cudaMemsetAsync(sums, 0, sizeof(double) * 2 * P, s) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "weight density");
    } else {
        k_chan_scale<<<(C + 127) / 128, 128, 0, s>>>(in.freq_hz, C, pp.beta_over_du, lam_inv, sc, lam_f, sc_f);
        WG_LAUNCHED("k_chan_scale");
        const int blocks = num_sms() * 8;
        if (rows > 0) {
            k_density<P><<<blocks, 256, 0, s>>>(in.uvw, lam_inv, sc, lam_f, sc_f, in.weight, in.flag, rows, pp, dens, sums);
            WG_LAUNCHED("k_density");
            k_density_sq<P><<<blocks, 256, 0, s>>>(dens, n_cells, sums);
            WG_LAUNCHED("k_density_sq");
            k_reweight<P><<<blocks, 256, 0, s>>>(in.uvw, lam_inv, sc, lam_f, sc_f, in.weight, in.flag, rows, pp, dens,
                                                 sums, scheme, 5.0 * std::pow(10.0, -robust), out);
            WG_LAUNCHED("k_reweight");
        }
        if (cudaGetLastError() != cudaSuccess) rc = fail(WG_E_CUDA, "weighting kernels failed to launch");
    }
    cudaFreeAsync(scratch, s);
    return rc;
}

int launch_weight(const Table& t, const Grid& g, const wg_vis_in& in, int scheme, double robust, int flags,
                  float* out, cudaStream_t s)
{
    switch (in.n_pol) {
        case 1: return weight_impl<1>(t, g, in, scheme, robust, flags, out, s);
        case 2: return weight_impl<2>(t, g, in, scheme, robust, flags, out, s);
        case 4: return weight_impl<4>(t, g, in, scheme, robust, flags, out, s);
        default: return fail(WG_E_INVALID_ARG, "n_pol must be 1, 2 or 4 (got %d)", in.n_pol);
    }
}

int launch_prep(const Table& t, const Grid& g, const wg_vis_in& in, int flags, WorkList& wl, cudaStream_t s)
{
    switch (in.n_pol) {
        case 1: return prep_impl<1>(t, g, in, flags, wl, s);
        case 2: return prep_impl<2>(t, g, in, flags, wl, s);
        case 4: return prep_impl<4>(t, g, in, flags, wl, s);
        default: return fail(WG_E_INVALID_ARG, "n_pol must be 1, 2 or 4 (got %d)", in.n_pol);
    }
}

}  // namespace wg
