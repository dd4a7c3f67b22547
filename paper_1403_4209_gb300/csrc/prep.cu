// Preparation phase of the WImager algorithm (thesis Sec. 4.3.4) on the GPU.
//
// The input is tiled into blocks of whole rows x all channels (kTileRecords records), read in
// natural [row][chan][pol] order so every load is coalesced.
//   k_classify  (PreProcessUVW, Sec. 4.3.4): FP64 placement of each record (row, chan), its
//               griddability, the compression indicator c (eq. "ci": same footprint origin
//               and kernel pointer as the griddable predecessor (row-1, chan)), g = gd & !c,
//               normaliser terms eps (1-f) zeta (eq. "normalizer") and statistics; a block
//               scan of g in channel-major order gives each gridded record its rank inside
//               the tile (Index Create and Filter, Algorithm "index").
//   k_scan_tiles / k_finalize: per-channel exclusive scan of the tile counts and the
//               channel bases, so gridded records land channel-major, row-ordered.
//   k_compact   (Compress Index Generate + Compress and Weigh Visibilities, Algorithm
//               "compressindex", eqs. "compress1"/"conjugatetake"): each gridded record
//               walks its run of compressed successors and sums eps (1-f) psi-conj(vis).
//   k_segments + k_seg_scan (Plan Create / Plan Analyse, Algorithm "plan"): gridded entries
//               are cut into segments of seg_len entries; each segment needs one gridder task
//               per block of `slots` footprint points of its largest support.  The plan can be
//               redone with other parameters (launch_plan) without repeating the preparation.
#include <cstdio>

#include <cuda_fp16.h>

#include "internal.cuh"

namespace wg {

namespace {

__device__ __forceinline__ long long floor_div(long long a, long long b)
{
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

struct Placed {
    int4 info;   // {x0 | y0 << 16, cu | cv << 16, z, k | neg << kBitNeg | gd << kBitGd}
    int S;
};

// Placement of one record, FP64, each operation rounded once (no contraction).
__device__ __forceinline__ Placed place(const double* __restrict__ uvw, int64_t row, double lam_inv,
                                        double sc, const uint8_t* __restrict__ flag, int64_t rec,
                                        int P, const PlaceParams& pp)
{
    Placed o;
    o.info = make_int4(0, 0, 0, 0);
    o.S = 0;
    const double up = uvw[3 * row], vp = uvw[3 * row + 1], wp = uvw[3 * row + 2];
    double tu = __dmul_rn(up, sc), tv = __dmul_rn(vp, sc), w = __dmul_rn(wp, lam_inv);
    const bool neg = wp < 0.0;
    if (neg) {
        tu = -tu;
        tv = -tv;
        w = -w;
    }
    o.info.w = neg ? (1 << kBitNeg) : 0;
    const double qu = ceil(__dsub_rn(tu, 0.5)), qv = ceil(__dsub_rn(tv, 0.5));
    if (!(fabs(qu) < 1099511627776.0) || !(fabs(qv) < 1099511627776.0)) return o;   // 2^40
    const long long iqu = (long long)qu, iqv = (long long)qv, b = pp.beta;
    const long long xc = floor_div(2 * iqu + b - 1, 2 * b), yc = floor_div(2 * iqv + b - 1, 2 * b);
    const int fu = (int)(iqu - b * xc), fv = (int)(iqv - b * yc);
    int k = 0;
    if (pp.K > 1) {   // nearest plane in sqrt(w): k = number of b_1..b_{K-1} with w >= b_m
        if (!(w < __ldg(&pp.wbounds[pp.K - 1]))) return o;   // beyond the last plane (or NaN)
        int lo = 0, hi = pp.K - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (w >= __ldg(&pp.wbounds[mid - 1])) lo = mid; else hi = mid - 1;
        }
        k = lo;
    }
    const int S = __ldg(&pp.supports[k]);
    const int h = (S - 1) / 2;
    const long long x0 = pp.N / 2 + xc - h, y0 = pp.N / 2 + yc - h;
    if (x0 < 0 || y0 < 0 || x0 + S - 1 > pp.N - 1 || y0 + S - 1 > pp.N - 1) return o;
    bool unflagged = false;
    for (int p = 0; p < P; ++p) unflagged |= (flag[rec * P + p] == 0);
    if (!unflagged) return o;
    const int sub = (fv - pp.lo) * pp.beta + (fu - pp.lo);
    const int ix0 = (int)x0, iy0 = (int)y0;
    const int cu = (S - ix0 % S) % S, cv = (S - iy0 % S) % S;
    o.info.x = ix0 | (iy0 << 16);
    o.info.y = cu | (cv << 16);
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

// exclusive block scan of a[0..n) in place; a[n] = total.  Needs blockDim multiple of 32.
__device__ void block_exclusive_scan(int* a, int n, int* warp_tot)
{
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int ipt = (n + T - 1) / T;
    const int b0 = min(n, t * ipt), b1 = min(n, b0 + ipt);
    int s = 0;
    for (int i = b0; i < b1; ++i) s += a[i];
    int inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int nw = T >> 5;
        int v = (lane < nw) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < nw) warp_tot[lane] = v;   // inclusive
    }
    __syncthreads();
    int run = inc - s + (wid > 0 ? warp_tot[wid - 1] : 0);
    for (int i = b0; i < b1; ++i) {
        int v = a[i];
        a[i] = run;
        run += v;
    }
    __syncthreads();
    if (t == T - 1) a[n] = run + 0;
    __syncthreads();
    if (t == 0 && n > 0 && b1 < n) {}  // (all threads participated)
}

}  // namespace

__global__ void k_chan_scale(const double* __restrict__ freq, int C, double beta_over_du, double* lam_inv,
                             double* sc)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double li = __ddiv_rn(freq[c], 299792458.0);
    lam_inv[c] = li;
    sc[c] = __dmul_rn(li, beta_over_du);
}

template <int P>
__global__ void __launch_bounds__(512) k_classify(const double* __restrict__ uvw, const double* __restrict__ lam_inv,
                                                  const double* __restrict__ sc, const float* __restrict__ weight,
                                                  const uint8_t* __restrict__ flag, int64_t rows, int rpb,
                                                  PlaceParams pp, int4* __restrict__ rinfo,
                                                  uint8_t* __restrict__ rclass, int* __restrict__ tile_cnt,
                                                  double* __restrict__ norm_priv,
                                                  unsigned long long* __restrict__ stat_priv)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int C = pp.C;
    const int64_t tile = blockIdx.x;
    const int64_t row0 = tile * rpb;
    const int nrows = (int)min((int64_t)rpb, rows - row0);
    const int nrec = nrows * C;
    const int cap = rpb * C;
    int4* s_info = reinterpret_cast<int4*>(smem);
    int* s_scan = reinterpret_cast<int*>(s_info + cap);            // [cap + 1]
    float* s_norm = reinterpret_cast<float*>(s_scan + cap + 1);    // [C * P]
    unsigned char* s_gc = reinterpret_cast<unsigned char*>(s_norm + C * P);  // [cap]
    __shared__ int warp_tot[32];
    __shared__ unsigned long long s_stat[ST_N];

    for (int i = threadIdx.x; i < C * P; i += blockDim.x) s_norm[i] = 0.f;
    if (threadIdx.x < ST_N) s_stat[threadIdx.x] = 0ull;

    // pass 1: placement
    for (int j = threadIdx.x; j < nrec; j += blockDim.x) {
        const int rr = j / C, ch = j - rr * C;
        const int64_t row = row0 + rr, rec = row * C + ch;
        s_info[j] = place(uvw, row, lam_inv[ch], sc[ch], flag, rec, P, pp).info;
    }
    __syncthreads();

    // pass 2: compression indicator, g, normaliser terms, statistics
    unsigned long long n_gd = 0, n_g = 0, n_c = 0, u_g = 0, u_c = 0;
    for (int j = threadIdx.x; j < nrec; j += blockDim.x) {
        const int rr = j / C, ch = j - rr * C;
        const int64_t row = row0 + rr, rec = row * C + ch;
        const int4 info = s_info[j];
        const int gd = (info.w >> kBitGd) & 1;
        int c = 0;
        if (pp.compress && gd && row > 0) {
            int4 pinfo;
            if (rr > 0) pinfo = s_info[j - C];
            else pinfo = place(uvw, row - 1, lam_inv[ch], sc[ch], flag, rec - C, P, pp).info;
            c = ((pinfo.w >> kBitGd) & 1) && pinfo.x == info.x && pinfo.z == info.z;
        }
        const int g = gd & (c ^ 1);
        s_gc[j] = (unsigned char)(g | (c << 1) | (gd << 2));
        s_scan[ch * nrows + rr] = g;
        if (gd) {
            const int k = info.w & 0xFFF;
            const int S = __ldg(&pp.supports[k]);
            const unsigned long long s2 = (unsigned long long)S * S;
            n_gd += 1;
            n_g += g;
            n_c += c;
            u_g += g ? s2 : 0ull;
            u_c += c ? s2 : 0ull;
            const int sub = (info.z - __ldg(&pp.offsets[k])) / (S * S);
            const float zeta = __ldg(&pp.zeta_f[k * pp.beta * pp.beta + sub]);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float wf = pp.unweighted ? 1.0f : weight[rec * P + p] * (1.0f - (float)flag[rec * P + p]);
                atomicAdd(&s_norm[ch * P + p], wf * zeta);
            }
        }
    }
    // block statistics
    {
        unsigned long long v[5] = {n_gd, n_g, n_c, u_g, u_c};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            unsigned long long x = v[q];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_stat[q + 1], x);
        }
    }
    __syncthreads();

    // pass 3: channel-major exclusive scan of g -> rank inside the tile
    block_exclusive_scan(s_scan, nrec, warp_tot);

    // pass 4: outputs
    for (int j = threadIdx.x; j < nrec; j += blockDim.x) {
        const int rr = j / C, ch = j - rr * C;
        const int64_t rec = (row0 + rr) * C + ch;
        int4 info = s_info[j];
        const int gc = s_gc[j];
        const int rank = s_scan[ch * nrows + rr] - s_scan[ch * nrows];
        info.w |= ((gc & 1) << kBitG) | (((gc >> 1) & 1) << kBitC) | (rank << 16);
        rinfo[rec] = info;
        rclass[rec] = (uint8_t)gc;
    }
    for (int ch = threadIdx.x; ch < C; ch += blockDim.x)
        tile_cnt[tile * C + ch] = s_scan[(ch + 1) * nrows] - s_scan[ch * nrows];
    const int slot = (int)(tile % kNormSlots);
    for (int i = threadIdx.x; i < C * P; i += blockDim.x)
        if (s_norm[i] != 0.f) atomicAdd(&norm_priv[(int64_t)slot * C * P + i], (double)s_norm[i]);
    if (threadIdx.x == 0) {
        s_stat[ST_RECORDS] = (unsigned long long)nrec;
    }
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

template <int P>
__global__ void k_finalize(int* __restrict__ chan_base, int C, const double* __restrict__ norm_priv,
                           double* __restrict__ norm_batch, const unsigned long long* __restrict__ stat_priv,
                           unsigned long long* __restrict__ stats, long long* __restrict__ scal)
{
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int c = 0; c < C; ++c) {
            const int t = chan_base[c];
            chan_base[c] = (int)run;
            run += t;
        }
        chan_base[C] = (int)run;
        scal[0] = run;
    }
    for (int i = threadIdx.x; i < C * P; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < kNormSlots; ++k) s += norm_priv[(int64_t)k * C * P + i];
        norm_batch[i] = s;
    }
    for (int q = threadIdx.x; q < ST_TASKS; q += blockDim.x) {
        unsigned long long s = 0;
        for (int k = 0; k < kNormSlots; ++k) s += stat_priv[k * ST_N + q];
        stats[q] = s;
    }
}

// visibility element -> complex float (half-precision values carry a per-channel scale)
__device__ __forceinline__ float2 vis_value(const float2* __restrict__ v, int64_t i, float) { return v[i]; }
__device__ __forceinline__ float2 vis_value(const __half2* __restrict__ v, int64_t i, float scale)
{
    const float2 f = __half22float2(v[i]);
    return make_float2(scale * f.x, scale * f.y);
}

template <int P, typename VT>
__global__ void __launch_bounds__(512) k_compact(const int4* __restrict__ rinfo, const VT* __restrict__ vis,
                                                 const float* __restrict__ vis_scale,
                                                 const float* __restrict__ weight, const uint8_t* __restrict__ flag,
                                                 int64_t rows, int rpb, int C, const int* __restrict__ tile_off,
                                                 const int* __restrict__ chan_base, const int* __restrict__ supports,
                                                 int4* __restrict__ entries, float2* __restrict__ gamma,
                                                 int2* __restrict__ runs, int64_t cap,
                                                 long long* __restrict__ scal, int unweighted)
{
    const int64_t tile = blockIdx.x;
    const int64_t row0 = tile * rpb;
    const int nrows = (int)min((int64_t)rpb, rows - row0);
    const int nrec = nrows * C;
    for (int j = threadIdx.x; j < nrec; j += blockDim.x) {
        const int rr = j / C, ch = j - rr * C;
        const int64_t row = row0 + rr, rec = row * C + ch;
        const int4 info = rinfo[rec];
        if (!((info.w >> kBitG) & 1)) continue;
        const int rank = (info.w >> 16) & 0xFFFF;
        const int dst = chan_base[ch] + tile_off[tile * C + ch] + rank;
        const float scale = vis_scale ? vis_scale[ch] : 1.0f;
        if (dst < 0 || (int64_t)dst >= cap) {   // cannot happen with a consistent scan
            atomicAdd(reinterpret_cast<unsigned long long*>(&scal[3]), 1ull);
            continue;
        }
        float2 acc[P];
        {
            const float sg = ((info.w >> kBitNeg) & 1) ? -1.f : 1.f;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float wf = unweighted ? 1.0f : weight[rec * P + p] * (1.0f - (float)flag[rec * P + p]);
                const float2 v = vis_value(vis, rec * P + p, scale);
                acc[p] = make_float2(wf * v.x, sg * (wf * v.y));
            }
        }
        int64_t last = row;
        for (int64_t r2 = row + 1; r2 < rows; ++r2) {
            const int64_t rc2 = r2 * C + ch;
            const int4 i2 = rinfo[rc2];
            if (!((i2.w >> kBitC) & 1)) break;
            const float sg = ((i2.w >> kBitNeg) & 1) ? -1.f : 1.f;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float wf = unweighted ? 1.0f : weight[rc2 * P + p] * (1.0f - (float)flag[rc2 * P + p]);
                const float2 v = vis_value(vis, rc2 * P + p, scale);
                acc[p].x += wf * v.x;
                acc[p].y += sg * (wf * v.y);
            }
            last = r2;
        }
        const int k = info.w & 0xFFF;
        entries[dst] = make_int4(info.x, info.y, info.z, k | (ch << 16));
#pragma unroll
        for (int p = 0; p < P; ++p) gamma[(int64_t)dst * P + p] = acc[p];
        runs[dst] = make_int2((int)row, (int)last);
    }
}

// per segment, the number of task blocks of its largest support; sets the segment count
__global__ void k_segments(const int4* __restrict__ entries, long long* __restrict__ scal,
                           const int* __restrict__ supports, int K, int seg_len, int slots,
                           int* __restrict__ seg_nblk)
{
    const long long n = scal[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[2] = (n + seg_len - 1) / seg_len;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int k = entries[e].w & 0xFFF;
        const int nb = (k < K) ? nblk_of(__ldg(&supports[k]), slots) : 1;
        atomicMax(&seg_nblk[e / seg_len], nb);
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

static size_t classify_smem(int rpb, int C, int P)
{
    const size_t cap = (size_t)rpb * C;
    return cap * sizeof(int4) + (cap + 1) * sizeof(int) + (size_t)C * P * sizeof(float) + cap + 16;
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

    PlaceParams pp;
    pp.N = g.n;
    pp.beta = t.beta;
    pp.K = t.K;
    pp.lo = -((t.beta - 1) / 2);
    pp.compress = (flags & WG_PREP_COMPRESS) ? 1 : 0;
    pp.unweighted = (flags & WG_PREP_UNWEIGHTED) ? 1 : 0;
    pp.C = C;
    pp.P = P;
    pp.w_max = t.w_max;
    pp.beta_over_du = (double)t.beta / g.du;
    pp.supports = t.supports_d;
    pp.offsets = t.offsets_d;
    pp.wbounds = t.wbounds_d;
    pp.zeta_f = t.zeta_f;

    double* lam_inv = reinterpret_cast<double*>(wl.norm_batch + (size_t)C * P);   // [C]
    double* sc = lam_inv + C;                                                     // [C]

    WG_CUDA(cudaMemsetAsync(wl.norm_priv, 0, sizeof(double) * kNormSlots * C * P, s));
    WG_CUDA(cudaMemsetAsync(wl.stat_priv, 0, sizeof(unsigned long long) * kNormSlots * ST_N, s));
    WG_CUDA(cudaMemsetAsync(wl.stats, 0, sizeof(unsigned long long) * ST_N, s));
    WG_CUDA(cudaMemsetAsync(wl.scal, 0, sizeof(long long) * 4, s));

    k_chan_scale<<<(C + 127) / 128, 128, 0, s>>>(in.freq_hz, C, pp.beta_over_du, lam_inv, sc);
    WG_LAUNCHED("k_chan_scale");
    if (rows > 0) {
        const size_t sm = classify_smem(rpb, C, P);
        if (sm > 48 * 1024) WG_CUDA(cudaFuncSetAttribute(k_classify<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_classify<P><<<(unsigned)n_tiles, 512, sm, s>>>(in.uvw, lam_inv, sc, in.weight, in.flag, rows, rpb, pp,
                                                          wl.rinfo, wl.rclass, wl.tile_cnt, wl.norm_priv, wl.stat_priv);
        WG_LAUNCHED("k_classify");
    }
    k_scan_tiles<<<C, 1024, 0, s>>>(wl.tile_cnt, n_tiles, C, wl.chan_base);
    WG_LAUNCHED("k_scan_tiles");
    k_finalize<P><<<1, 256, 0, s>>>(wl.chan_base, C, wl.norm_priv, wl.norm_batch, wl.stat_priv, wl.stats, wl.scal);
    WG_LAUNCHED("k_finalize");
    if (rows > 0) {
        if (in.vis_dtype == WG_VIS_COMPLEX_HALF)
            k_compact<P, __half2><<<(unsigned)n_tiles, 512, 0, s>>>(
                wl.rinfo, reinterpret_cast<const __half2*>(in.vis), in.vis_scale, in.weight, in.flag, rows, rpb, C,
                wl.tile_cnt, wl.chan_base, t.supports_d, wl.entries, wl.gamma, wl.runs, wl.cap, wl.scal,
                pp.unweighted);
        else
            k_compact<P, float2><<<(unsigned)n_tiles, 512, 0, s>>>(
                wl.rinfo, reinterpret_cast<const float2*>(in.vis), nullptr, in.weight, in.flag, rows, rpb, C,
                wl.tile_cnt, wl.chan_base, t.supports_d, wl.entries, wl.gamma, wl.runs, wl.cap, wl.scal,
                pp.unweighted);
        WG_LAUNCHED("k_compact");
    }
    return launch_plan(t, wl, s);
}

int launch_plan(const Table& t, WorkList& wl, cudaStream_t s)
{
    const int64_t n_seg_max = (wl.cap + wl.seg_len - 1) / wl.seg_len + 1;
    WG_CUDA(cudaMemsetAsync(wl.seg_nblk, 0, sizeof(int) * std::min<int64_t>(n_seg_max, wl.seg_cap), s));
    k_segments<<<num_sms() * 4, 256, 0, s>>>(wl.entries, wl.scal, t.supports_d, t.K, wl.seg_len, wl.slots,
                                              wl.seg_nblk);
    WG_LAUNCHED("k_segments");
    k_seg_scan<<<1, 1024, 0, s>>>(wl.seg_nblk, wl.seg_off, wl.scal, wl.stats);
    WG_LAUNCHED("k_seg_scan");
    return WG_OK;
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
