// C-ABI entry points of include/wgrid.h: argument validation, handle lifetime, error reporting.
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace wg {

std::atomic<uint64_t> g_launches{0};
static thread_local char t_err[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { t_err[0] = 0; }

int cuda_fail(cudaError_t e, const char* what)
{
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? WG_E_OOM : WG_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace wg

using namespace wg;

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Device allocations of grid_create and worklist_create go through this gate.  With the
// allocation-failure fake armed (wg_debug_fail_allocations), the allocation after the next
// `after` successful ones fails as cudaMalloc would, without calling the runtime; disarmed
// (the default, -1) it is cudaMalloc.
static std::atomic<long long> g_fail_allocs_after{-1};

static cudaError_t dev_malloc(void** p, size_t bytes)
{
    long long n = g_fail_allocs_after.load();
    while (n > 0 && !g_fail_allocs_after.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

extern "C" {

const char* wg_last_error(void) { return t_err; }

uint64_t wg_launch_count(void) { return g_launches.load(); }

int wg_debug_fail_allocations(int64_t after)
{
    g_fail_allocs_after.store(after < 0 ? -1 : (long long)after);
    return WG_OK;
}

// ---- grid -----------------------------------------------------------------------------
int grid_create(const wg_grid_desc* d, wg_grid** out)
{
    t_err[0] = 0;
    if (!d || !out) return fail(WG_E_INVALID_ARG, "grid_create: null argument");
    *out = nullptr;
    if (d->n < 8 || d->n > 32768 || (d->n & 1)) return fail(WG_E_INVALID_ARG, "grid side N=%d must be even in [8, 32768]", d->n);
    if (d->n_pol != 1 && d->n_pol != 2 && d->n_pol != 4) return fail(WG_E_INVALID_ARG, "n_pol=%d must be 1, 2 or 4", d->n_pol);
    if (d->n_chan < 1 || d->n_chan > 4096) return fail(WG_E_INVALID_ARG, "n_chan=%d must be in [1, 4096]", d->n_chan);
    if (!(d->du > 0.0)) return fail(WG_E_INVALID_ARG, "cell size du must be positive");
    if (d->data && (reinterpret_cast<uintptr_t>(d->data) & 15)) return fail(WG_E_INVALID_ARG, "external grid buffer must be 16-byte aligned");
    if (d->flags & ~WG_GRID_COMPENSATED) return fail(WG_E_INVALID_ARG, "unknown grid flags %d", d->flags);
    wg_grid* h = new (std::nothrow) wg_grid;
    if (!h) return fail(WG_E_OOM, "host allocation failed");
    Grid& g = h->g;
    g.n = d->n;
    g.n_pol = d->n_pol;
    g.n_chan = d->n_chan;
    g.du = d->du;
    const size_t bytes = sizeof(float2) * (size_t)g.n * g.n * g.n_pol * g.n_chan;
    if (d->data) {
        g.data = static_cast<float2*>(d->data);
    } else {
        if (dev_malloc((void**)&g.data, bytes) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(WG_E_OOM, "cannot allocate a %zu-byte grid", bytes);
        }
        g.owns = true;
    }
    g.comp = (d->flags & WG_GRID_COMPENSATED) != 0;
    if (dev_malloc((void**)&g.norm, sizeof(double) * g.n_chan * g.n_pol) != cudaSuccess ||
        dev_malloc((void**)&g.counters, sizeof(unsigned long long) * ST_N) != cudaSuccess ||
        (g.comp && dev_malloc((void**)&g.err, bytes) != cudaSuccess)) {
        cudaGetLastError();
        grid_destroy(h);
        return fail(WG_E_OOM, "cannot allocate normaliser");
    }
    int rc = grid_zero(h, nullptr);
    if (rc == WG_OK && cudaDeviceSynchronize() != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "grid_create");
    if (rc != WG_OK) {
        grid_destroy(h);
        return rc;
    }
    *out = h;
    return WG_OK;
}

int grid_destroy(wg_grid* h)
{
    if (!h) return WG_OK;
    Grid& g = h->g;
    if (g.owns) cudaFree(g.data);
    cudaFree(g.norm);
    cudaFree(g.counters);
    cudaFree(g.err);
    cudaFree(g.scratch);
    cudaFree(g.corr);
    cudaFree(g.icorr);
    cudaFree(g.inv_norm);
    if (g.plan_ok) cufftDestroy(g.plan);
    if (g.plan_c_ok) cufftDestroy(g.plan_c);
    delete h;
    return WG_OK;
}

int grid_zero(wg_grid* h, void* stream)
{
    if (!h) return fail(WG_E_INVALID_ARG, "grid_zero: null grid");
    Grid& g = h->g;
    WG_CUDA(cudaMemsetAsync(g.data, 0, sizeof(float2) * (size_t)g.n * g.n * g.n_pol * g.n_chan, S(stream)));
    if (g.err) WG_CUDA(cudaMemsetAsync(g.err, 0, sizeof(float2) * (size_t)g.n * g.n * g.n_pol * g.n_chan, S(stream)));
    WG_CUDA(cudaMemsetAsync(g.norm, 0, sizeof(double) * g.n_chan * g.n_pol, S(stream)));
    WG_CUDA(cudaMemsetAsync(g.counters, 0, sizeof(unsigned long long) * ST_N, S(stream)));
    return WG_OK;
}

int grid_device_ptrs(const wg_grid* h, void** data, double** normaliser)
{
    if (!h) return fail(WG_E_INVALID_ARG, "grid_device_ptrs: null grid");
    if (data) *data = h->g.data;
    if (normaliser) *normaliser = h->g.norm;
    return WG_OK;
}

// ---- table ----------------------------------------------------------------------------
int conv_table_build(const wg_table_desc* d, wg_table** out, void* stream)
{
    t_err[0] = 0;
    if (!d || !out) return fail(WG_E_INVALID_ARG, "conv_table_build: null argument");
    *out = nullptr;
    if (d->n_wplanes < 1 || d->n_wplanes > 4095) return fail(WG_E_INVALID_ARG, "n_wplanes=%d must be in [1, 4095]", d->n_wplanes);
    if (d->oversample < 1 || d->oversample > kMaxBeta) return fail(WG_E_INVALID_ARG, "oversample=%d must be in [1, %d]", d->oversample, kMaxBeta);
    if (d->taper_support < 1 || d->taper_support > 255) return fail(WG_E_INVALID_ARG, "taper_support=%d must be in [1, 255]", d->taper_support);
    if (d->n_k != 0 && (d->n_k < 8 || (d->n_k & 1))) return fail(WG_E_INVALID_ARG, "n_k=%d must be 0 or even >= 8", d->n_k);
    if (!(d->du > 0.0)) return fail(WG_E_INVALID_ARG, "du must be positive");
    if (d->n_wplanes > 1 && !(d->w_max > 0.0)) return fail(WG_E_INVALID_ARG, "w_max must be positive with more than one w-plane");
    if (d->store_dtype != WG_F32 && d->store_dtype != WG_BF16 && d->store_dtype != WG_F16)
        return fail(WG_E_INVALID_ARG, "store_dtype %d not supported", d->store_dtype);
    if ((d->support_mode & ~(WG_TABLE_WSTACK | 0xFF)) != 0) return fail(WG_E_INVALID_ARG, "unknown support_mode %d", d->support_mode);
    const int smode = d->support_mode & 0xFF;
    if (smode == WG_SUPPORT_PRESCRIBED) {
        if (!d->supports) return fail(WG_E_INVALID_ARG, "prescribed supports missing");
        for (int k = 0; k < d->n_wplanes; ++k) {
            if (d->supports[k] < 1 || d->supports[k] % 2 == 0) return fail(WG_E_INVALID_ARG, "support %d of plane %d must be odd and positive", d->supports[k], k);
            if (d->supports[k] > kMaxSupport) return fail(WG_E_OOB_SUPPORT, "support %d of plane %d exceeds %d", d->supports[k], k, kMaxSupport);
        }
    } else if (smode == WG_SUPPORT_THRESHOLD) {
        if (!(d->threshold > 0.0)) return fail(WG_E_INVALID_ARG, "threshold must be positive");
    } else {
        return fail(WG_E_INVALID_ARG, "unknown support_mode %d", d->support_mode);
    }
    wg_table* h = new (std::nothrow) wg_table;
    if (!h) return fail(WG_E_OOM, "host allocation failed");
    int rc = build_table(*d, h->t, S(stream));
    if (rc == WG_OK && d->store_dtype != WG_F32) {
        rc = set_table_store(h->t, d->store_dtype);
        if (rc != WG_OK) free_table(h->t);
    }
    if (rc != WG_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return WG_OK;
}

int table_set_store(wg_table* h, int32_t store_dtype)
{
    t_err[0] = 0;
    if (!h) return fail(WG_E_INVALID_ARG, "table_set_store: null table");
    return set_table_store(h->t, store_dtype);
}

int conv_table_import(int32_t K, int32_t beta, double w_max, double du, int32_t s0, const int32_t* supports,
                      const double* data, const double* zeta, wg_table** out)
{
    t_err[0] = 0;
    if (!supports || !data || !zeta || !out) return fail(WG_E_INVALID_ARG, "conv_table_import: null argument");
    *out = nullptr;
    if (K < 1 || K > 4095 || beta < 1 || beta > kMaxBeta || !(du > 0.0) || s0 < 1 || s0 > 255)
        return fail(WG_E_INVALID_ARG, "conv_table_import: K, beta, du or taper support out of range");
    if (K > 1 && !(w_max > 0.0)) return fail(WG_E_INVALID_ARG, "w_max must be positive with more than one w-plane");
    wg_table* h = new (std::nothrow) wg_table;
    if (!h) return fail(WG_E_OOM, "host allocation failed");
    int rc = import_table(K, beta, w_max, du, s0, supports, data, zeta, h->t);
    if (rc != WG_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return WG_OK;
}

int table_destroy(wg_table* h)
{
    if (!h) return WG_OK;
    free_table(h->t);
    delete h;
    return WG_OK;
}

int table_info(const wg_table* h, wg_table_info* info)
{
    if (!h || !info) return fail(WG_E_INVALID_ARG, "table_info: null argument");
    const Table& t = h->t;
    info->n_wplanes = t.K;
    info->oversample = t.beta;
    info->taper_support = t.s0;
    info->max_support = t.max_support;
    info->n_samples = t.n_samples;
    info->w_max = t.w_max;
    info->du = t.du;
    info->data = t.data;
    info->zeta = t.zeta;
    info->supports = t.supports_d;
    info->offsets = t.offsets_d;
    info->store_dtype = t.store;
    info->reserved = 0;
    info->data_lp = t.data_lp;
    return WG_OK;
}

int table_copy_to_host(const wg_table* h, float* data, double* zeta, int32_t* supports, int32_t* offsets)
{
    if (!h) return fail(WG_E_INVALID_ARG, "table_copy_to_host: null table");
    const Table& t = h->t;
    if (data) WG_CUDA(cudaMemcpy(data, t.data, sizeof(float2) * t.n_samples, cudaMemcpyDeviceToHost));
    if (zeta) WG_CUDA(cudaMemcpy(zeta, t.zeta, sizeof(double) * t.K * t.beta * t.beta, cudaMemcpyDeviceToHost));
    if (supports) std::memcpy(supports, t.supports.data(), sizeof(int) * t.K);
    if (offsets) std::memcpy(offsets, t.offsets.data(), sizeof(int) * t.K);
    return WG_OK;
}

// ---- work list ------------------------------------------------------------------------
int worklist_destroy(wg_worklist* h)
{
    if (!h) return WG_OK;
    WorkList& w = h->w;
    void* ptrs[] = {w.rinfo, w.rclass, w.tile_cnt, w.carry_q, w.carry_last, w.entries, w.gamma, w.runs, w.dacc, w.seg_nblk, w.seg_off,
                    w.scal, w.chan_base, w.norm_priv, w.norm_batch, w.stat_priv, w.stats, w.stats_batch, w.task_counter};
    for (void* p : ptrs) cudaFree(p);
    delete h;
    return WG_OK;
}

// a work list for batches of up to max_records records and max_entries gridded entries in all
// (appended batches); `dacc` adds the degridder's per-entry accumulator
static int create_worklist(int64_t max_records, int64_t max_entries, int32_t C, int32_t P, bool dacc,
                           wg_worklist** out)
{
    t_err[0] = 0;
    if (!out) return fail(WG_E_INVALID_ARG, "worklist_create: null argument");
    *out = nullptr;
    if (max_records < 1 || max_records > ((int64_t)1 << 31) - 1)
        return fail(WG_E_INVALID_ARG, "max_records=%lld must be in [1, 2^31 - 1]", (long long)max_records);
    if (max_entries < 1 || max_entries > ((int64_t)1 << 31) - 1)
        return fail(WG_E_INVALID_ARG, "max_entries=%lld must be in [1, 2^31 - 1]", (long long)max_entries);
    if (C < 1 || C > 4096) return fail(WG_E_INVALID_ARG, "n_chan=%d must be in [1, 4096]", C);
    if (P != 1 && P != 2 && P != 4) return fail(WG_E_INVALID_ARG, "n_pol=%d must be 1, 2 or 4", P);
    wg_worklist* h = new (std::nothrow) wg_worklist;
    if (!h) return fail(WG_E_OOM, "host allocation failed");
    WorkList& w = h->w;
    w.cap = max_records;
    w.ecap = max_entries;
    w.C = C;
    w.P = P;
    const int rpb = std::max(1, kTileRecords / C);
    const int64_t rows_max = (max_records + C - 1) / C;
    w.tile_cap = ((rows_max + rpb - 1) / rpb + 2) * C;
    w.seg_cap = max_entries / kSegLenMin + 2;
    bool ok = true;
    auto al = [&](void** p, size_t bytes) {
        if (ok && dev_malloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
    };
    al((void**)&w.rinfo, sizeof(int4) * max_records);
    al((void**)&w.rclass, max_records);
    al((void**)&w.tile_cnt, sizeof(int) * w.tile_cap);
    al((void**)&w.carry_q, sizeof(float2) * w.tile_cap * P);
    al((void**)&w.carry_last, sizeof(int) * w.tile_cap);
    al((void**)&w.entries, sizeof(int4) * max_entries);
    al((void**)&w.gamma, sizeof(float2) * max_entries * P);
    al((void**)&w.runs, sizeof(int2) * max_entries);
    if (dacc) al((void**)&w.dacc, sizeof(float2) * max_entries * P);
    al((void**)&w.seg_nblk, sizeof(int) * w.seg_cap);
    al((void**)&w.seg_off, sizeof(int) * (w.seg_cap + 1));
    al((void**)&w.scal, sizeof(long long) * 8);
    al((void**)&w.chan_base, sizeof(int) * (C + 1));
    al((void**)&w.norm_priv, sizeof(double) * kNormSlots * C * P);
    al((void**)&w.norm_batch, sizeof(double) * (C * P + 3 * C));
    al((void**)&w.stat_priv, sizeof(unsigned long long) * kNormSlots * ST_N);
    al((void**)&w.stats, sizeof(unsigned long long) * ST_N);
    al((void**)&w.stats_batch, sizeof(unsigned long long) * ST_N);
    al((void**)&w.task_counter, sizeof(unsigned int) * 4);
    if (!ok) {
        worklist_destroy(h);
        return fail(WG_E_OOM, "cannot allocate a work list for %lld records and %lld entries", (long long)max_records,
                    (long long)max_entries);
    }
    if (cudaMemset(w.scal, 0, sizeof(long long) * 8) != cudaSuccess ||
        cudaMemset(w.stats, 0, sizeof(unsigned long long) * ST_N) != cudaSuccess ||
        cudaMemset(w.stats_batch, 0, sizeof(unsigned long long) * ST_N) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        worklist_destroy(h);
        return cuda_fail(cudaGetLastError(), "worklist_create");
    }
    *out = h;
    return WG_OK;
}

int worklist_create(int64_t max_records, int32_t C, int32_t P, wg_worklist** out)
{
    return create_worklist(max_records, max_records, C, P, true, out);
}

int worklist_create2(int64_t max_records, int64_t max_entries, int32_t C, int32_t P, wg_worklist** out)
{
    return create_worklist(max_records, max_entries, C, P, false, out);
}

int worklist_clear(wg_worklist* wh, void* stream)
{
    t_err[0] = 0;
    if (!wh) return fail(WG_E_INVALID_ARG, "worklist_clear: null work list");
    WorkList& w = wh->w;
    WG_CUDA(cudaMemsetAsync(w.scal, 0, sizeof(long long) * 8, S(stream)));
    WG_CUDA(cudaMemsetAsync(w.stats, 0, sizeof(unsigned long long) * ST_N, S(stream)));
    w.append = false;
    w.chan_hi = 0;
    w.plan_stale = false;
    w.N = 0;
    return WG_OK;
}

// grid channels per input channel: 1, 0 (interleaved: one grid channel), or K (w-stacking)
static int check_vis(const Grid& g, const Table& t, const wg_vis_in* in, int per_chan)
{
    if (!in) return fail(WG_E_INVALID_ARG, "null vis input");
    if (in->n_rows < 0) return fail(WG_E_INVALID_ARG, "n_rows must be >= 0");
    if (per_chan == 0 && (g.n_chan != 1 || in->n_pol != g.n_pol || in->n_chan < 1))
        return fail(WG_E_SHAPE, "interleaved channels need a one-channel grid with the vis polarisations "
                                "(grid: %d channels, %d pols; vis: %d pols)", g.n_chan, g.n_pol, in->n_pol);
    if (per_chan > 0 && ((int64_t)in->n_chan * per_chan != g.n_chan || in->n_pol != g.n_pol))
        return fail(WG_E_SHAPE, "vis shape (chan %d x %d planes, pol %d) differs from the grid's (%d, %d)", in->n_chan,
                    per_chan, in->n_pol, g.n_chan, g.n_pol);
    if ((int64_t)in->n_chan * (per_chan > 0 ? per_chan : 1) > 65535)
        return fail(WG_E_SHAPE, "%d channels x %d planes exceed 65535 grid channels", in->n_chan, per_chan);
    if (in->n_rows > 0 && (!in->uvw || !in->freq_hz || !in->vis || !in->weight || !in->flag))
        return fail(WG_E_INVALID_ARG, "null input array");
    if (std::fabs(t.du - g.du) > 1e-12 * g.du) return fail(WG_E_SHAPE, "table du %.17g differs from grid du %.17g", t.du, g.du);
    if (t.max_support > g.n) return fail(WG_E_OOB_SUPPORT, "support %d larger than the grid (%d)", t.max_support, g.n);
    if (in->vis_dtype != WG_VIS_COMPLEX64 && in->vis_dtype != WG_VIS_COMPLEX_HALF)
        return fail(WG_E_INVALID_ARG, "unknown vis_dtype %d", in->vis_dtype);
    if (in->vis_dtype == WG_VIS_COMPLEX_HALF && in->n_rows > 0 && !in->vis_scale)
        return fail(WG_E_INVALID_ARG, "vis_scale is required for half-precision visibilities");
    if ((reinterpret_cast<uintptr_t>(in->vis) & (in->vis_dtype == WG_VIS_COMPLEX64 ? 7 : 3)))
        return fail(WG_E_INVALID_ARG, "vis is not aligned to its element size");
    return WG_OK;
}

int vis_compress(const wg_grid* gh, const wg_table* th, const wg_vis_in* in, int32_t flags, wg_worklist* wh,
                 void* stream)
{
    t_err[0] = 0;
    if (!gh || !th || !wh) return fail(WG_E_INVALID_ARG, "vis_compress: null handle");
    WorkList& w = wh->w;
    if (flags & WG_PREP_APPEND) {
        // the batch is a channel slice of the grid: check it against a view of those channels
        if (flags & (WG_PREP_INTERLEAVE | WG_PREP_WSTACK))
            return fail(WG_E_INVALID_ARG, "WG_PREP_APPEND is not combined with WG_PREP_INTERLEAVE or WG_PREP_WSTACK");
        if (!in) return fail(WG_E_INVALID_ARG, "null vis input");
        if (in->chan0 < 0 || (int64_t)in->chan0 + in->n_chan > gh->g.n_chan)
            return fail(WG_E_SHAPE, "channels %d..%d of the batch exceed the grid's %d", in->chan0,
                        in->chan0 + in->n_chan - 1, gh->g.n_chan);
        if (!w.append && w.N != 0)
            return fail(WG_E_INVALID_ARG, "the work list holds a batch prepared without WG_PREP_APPEND: call worklist_clear first");
        Grid slice = gh->g;
        slice.n_chan = in->n_chan;
        int rc = check_vis(slice, th->t, in, 1);
        if (rc != WG_OK) return rc;
    } else {
        if (in && in->chan0 != 0) return fail(WG_E_INVALID_ARG, "chan0 is used only with WG_PREP_APPEND");
        int rc = check_vis(gh->g, th->t, in, (flags & WG_PREP_INTERLEAVE) ? 0 : (flags & WG_PREP_WSTACK) ? th->t.K : 1);
        if (rc != WG_OK) return rc;
    }
    if (in->n_chan != w.C || in->n_pol != w.P) return fail(WG_E_SHAPE, "work list was created for %d channels, %d pols", w.C, w.P);
    if (in->n_rows * (int64_t)in->n_chan > w.cap)
        return fail(WG_E_CAPACITY, "%lld records exceed the work list capacity %lld", (long long)(in->n_rows * (int64_t)in->n_chan), (long long)w.cap);
    if (flags & ~(WG_PREP_COMPRESS | WG_PREP_UNWEIGHTED | WG_PREP_INTERLEAVE | WG_PREP_CROSS_SWAP | WG_PREP_WSTACK |
                  WG_PREP_APPEND))
        return fail(WG_E_INVALID_ARG, "unknown vis_compress flags %d", flags);
    if ((flags & WG_PREP_WSTACK) && ((flags & WG_PREP_INTERLEAVE) || !th->t.stacking))
        return fail(WG_E_INVALID_ARG, "WG_PREP_WSTACK needs a WG_TABLE_WSTACK table and no interleaving");
    if ((flags & WG_PREP_CROSS_SWAP) && in->n_pol != 4)
        return fail(WG_E_INVALID_ARG, "WG_PREP_CROSS_SWAP needs n_pol = 4 (got %d)", in->n_pol);
    return launch_prep(th->t, gh->g, *in, flags, w, S(stream));
}

int worklist_stats(const wg_worklist* wh, wg_stats* out, void* stream)
{
    if (!wh || !out) return fail(WG_E_INVALID_ARG, "worklist_stats: null argument");
    const WorkList& w = wh->w;
    unsigned long long st[ST_N];
    long long sc[4];
    WG_CUDA(cudaMemcpyAsync(st, w.stats, sizeof(st), cudaMemcpyDeviceToHost, S(stream)));
    WG_CUDA(cudaMemcpyAsync(sc, w.scal, sizeof(sc), cudaMemcpyDeviceToHost, S(stream)));
    WG_CUDA(cudaStreamSynchronize(S(stream)));
    out->records = (int64_t)st[ST_RECORDS];
    out->griddable = (int64_t)st[ST_GRIDDABLE];
    out->gridded = (int64_t)st[ST_GRIDDED];
    out->compressed = (int64_t)st[ST_COMPRESSED];
    out->updates = (int64_t)st[ST_UPD] * w.P;
    out->updates_saved = (int64_t)st[ST_UPD_SAVED] * w.P;
    out->tasks = (int64_t)st[ST_TASKS];
    out->dropped = sc[3];
    return WG_OK;
}

int worklist_view(const wg_worklist* wh, const int32_t** entries, const void** gamma, const int32_t** runs,
                  const uint8_t** rec_class, int64_t* n_entries, void* stream)
{
    if (!wh) return fail(WG_E_INVALID_ARG, "worklist_view: null work list");
    const WorkList& w = wh->w;
    if (entries) *entries = reinterpret_cast<const int32_t*>(w.entries);
    if (gamma) *gamma = w.gamma;
    if (runs) *runs = reinterpret_cast<const int32_t*>(w.runs);
    if (rec_class) *rec_class = w.rclass;
    if (n_entries) {
        long long n = 0;
        WG_CUDA(cudaMemcpyAsync(&n, w.scal, sizeof(n), cudaMemcpyDeviceToHost, S(stream)));
        WG_CUDA(cudaStreamSynchronize(S(stream)));
        *n_entries = n;
    }
    return WG_OK;
}

int grid_vis(wg_grid* gh, const wg_table* th, const wg_worklist* wh, void* stream)
{
    t_err[0] = 0;
    if (!gh || !th || !wh) return fail(WG_E_INVALID_ARG, "grid_vis: null handle");
    Grid& g = gh->g;
    WorkList& w = const_cast<WorkList&>(wh->w);      // a stale plan of appended batches is redone
    if (w.append) {
        if (w.chan_hi > g.n_chan || w.P != g.n_pol)
            return fail(WG_E_SHAPE, "appended batches use %d grid channels, the grid has %d", w.chan_hi, g.n_chan);
    } else if ((w.interleave ? 1 : w.C * w.wstack_k) != g.n_chan || w.P != g.n_pol) {
        return fail(WG_E_SHAPE, "work list shape differs from the grid's");
    }
    if (w.N != 0 && w.N != g.n) return fail(WG_E_SHAPE, "work list was prepared for N=%d, grid has N=%d", w.N, g.n);
    if (w.plan_stale) {
        if (int rc = launch_plan(th->t, w, S(stream))) return rc;
        w.plan_stale = false;
    }
    return launch_grid(g, th->t, w, S(stream));
}


// ---- gridder plan ---------------------------------------------------------------------
static int check_plan(const wg_plan& p)
{
    if (p.seg_len < kSegLenMin || p.seg_len > kSegLenMax || p.seg_len % 32)
        return fail(WG_E_INVALID_ARG, "seg_len=%d must be a multiple of 32 in [%d, %d]", p.seg_len, kSegLenMin,
                    kSegLenMax);
    if (p.slots < kSlotsMin || p.slots > kSlotsMax || p.slots % 32)
        return fail(WG_E_INVALID_ARG, "slots=%d must be a multiple of 32 in [%d, %d]", p.slots, kSlotsMin, kSlotsMax);
    if (p.flags & ~WG_PLAN_FIXED_R) return fail(WG_E_INVALID_ARG, "unknown plan flags %d", p.flags);
    return WG_OK;
}

int worklist_plan(wg_worklist* wh, const wg_table* th, const wg_plan* plan, void* stream)
{
    t_err[0] = 0;
    if (!wh || !th || !plan) return fail(WG_E_INVALID_ARG, "worklist_plan: null argument");
    if (int rc = check_plan(*plan)) return rc;
    WorkList& w = wh->w;
    w.seg_len = plan->seg_len;
    w.slots = plan->slots;
    w.fixed_r = (plan->flags & WG_PLAN_FIXED_R) != 0;
    if (w.N == 0) return WG_OK;     // nothing prepared yet: the next vis_compress uses the plan
    w.plan_stale = false;
    return launch_plan(th->t, w, S(stream));
}

int worklist_get_plan(const wg_worklist* wh, wg_plan* plan)
{
    if (!wh || !plan) return fail(WG_E_INVALID_ARG, "worklist_get_plan: null argument");
    plan->seg_len = wh->w.seg_len;
    plan->slots = wh->w.slots;
    plan->flags = wh->w.fixed_r ? WG_PLAN_FIXED_R : 0;
    plan->reserved = 0;
    return WG_OK;
}

int grid_autotune(wg_grid* gh, const wg_table* th, wg_worklist* wh, const wg_plan* cands, int32_t n_cands,
                  int32_t repeats, wg_plan* best_out, float* best_ms, void* stream)
{
    t_err[0] = 0;
    if (!gh || !th || !wh) return fail(WG_E_INVALID_ARG, "grid_autotune: null handle");
    if (repeats < 1 || repeats > 1000) return fail(WG_E_INVALID_ARG, "repeats=%d must be in [1, 1000]", repeats);
    std::vector<wg_plan> list;
    if (cands && n_cands > 0) {
        list.assign(cands, cands + n_cands);
    } else {
        for (int seg : {64, 128, 256})
            for (int slots : {128, 256})
                for (int flags : {0, WG_PLAN_FIXED_R}) list.push_back(wg_plan{seg, slots, flags, 0});
    }
    for (const wg_plan& p : list)
        if (int rc = check_plan(p)) return rc;
    WorkList& w = wh->w;
    if (w.N == 0) return fail(WG_E_INVALID_ARG, "grid_autotune: the work list holds no prepared batch");
    cudaStream_t s = S(stream);
    cudaEvent_t ev[2];
    WG_CUDA(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail(cudaGetLastError(), "grid_autotune");
    }
    float best = -1.f;
    wg_plan best_plan{w.seg_len, w.slots, w.fixed_r ? WG_PLAN_FIXED_R : 0, 0};
    int rc = WG_OK;
    for (const wg_plan& p : list) {
        if ((rc = worklist_plan(wh, th, &p, stream))) break;
        if ((rc = grid_vis(gh, th, wh, stream))) break;      // warm-up (occupancy query, caches)
        if (cudaEventRecord(ev[0], s) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "grid_autotune");
            break;
        }
        for (int r = 0; r < repeats && rc == WG_OK; ++r) rc = grid_vis(gh, th, wh, stream);
        if (rc) break;
        float ms = 0.f;
        if (cudaEventRecord(ev[1], s) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "grid_autotune");
            break;
        }
        ms /= repeats;
        if (best < 0.f || ms < best) {
            best = ms;
            best_plan = p;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    if ((rc = worklist_plan(wh, th, &best_plan, stream))) return rc;
    if ((rc = grid_zero(gh, stream))) return rc;
    WG_CUDA(cudaStreamSynchronize(s));
    if (best_out) *best_out = best_plan;
    if (best_ms) *best_ms = best;
    return WG_OK;
}

int vis_weight(const wg_grid* gh, const wg_table* th, const wg_vis_in* in, int32_t scheme, double robust,
               int32_t flags, float* weight_out, void* stream)
{
    t_err[0] = 0;
    if (!gh || !th || !weight_out) return fail(WG_E_INVALID_ARG, "vis_weight: null argument");
    if (scheme != WG_WEIGHT_UNIFORM && scheme != WG_WEIGHT_ROBUST)
        return fail(WG_E_INVALID_ARG, "unknown weighting scheme %d", scheme);
    if (!std::isfinite(robust) || std::fabs(robust) > 10.0)
        return fail(WG_E_INVALID_ARG, "robustness %g must be finite, within +-10", robust);
    if (flags & ~(WG_PREP_INTERLEAVE | WG_PREP_COMPRESS | WG_PREP_UNWEIGHTED | WG_PREP_CROSS_SWAP | WG_PREP_WSTACK))
        return fail(WG_E_INVALID_ARG, "unknown flags %d", flags);
    int rc = check_vis(gh->g, th->t, in, (flags & WG_PREP_INTERLEAVE) ? 0 : (flags & WG_PREP_WSTACK) ? th->t.K : 1);
    if (rc != WG_OK) return rc;
    if (reinterpret_cast<uintptr_t>(weight_out) & 3) return fail(WG_E_INVALID_ARG, "weight_out must be 4-byte aligned");
    return launch_weight(th->t, gh->g, *in, scheme, robust, flags & WG_PREP_INTERLEAVE, weight_out, S(stream));
}

int degrid_vis(const wg_grid* gh, const wg_table* th, const wg_vis_in* in, const wg_worklist* wh, int32_t mode,
               void* vis_out, void* stream)
{
    t_err[0] = 0;
    if (!gh || !th || !wh || !vis_out) return fail(WG_E_INVALID_ARG, "degrid_vis: null argument");
    if (mode != WG_DEGRID_PREDICT && mode != WG_DEGRID_ADJOINT) return fail(WG_E_INVALID_ARG, "unknown degrid mode %d", mode);
    const WorkList& w = wh->w;
    if (w.append) return fail(WG_E_INVALID_ARG, "degrid_vis: the work list holds WG_PREP_APPEND batches");
    int rc = check_vis(gh->g, th->t, in, w.interleave ? 0 : w.wstack_k);
    if (rc != WG_OK) return rc;
    if (w.rows != in->n_rows || w.C != in->n_chan) return fail(WG_E_SHAPE, "work list was prepared for a different batch");
    if (reinterpret_cast<uintptr_t>(vis_out) & 7) return fail(WG_E_INVALID_ARG, "vis_out must be 8-byte aligned");
    return launch_degrid(gh->g, th->t, *in, w, mode, static_cast<float2*>(vis_out), S(stream));
}

int grid_correct(wg_grid* gh, const wg_table* th, int32_t mode, float* image_out, void* stream)
{
    t_err[0] = 0;
    if (!gh || !th || !image_out) return fail(WG_E_INVALID_ARG, "grid_correct: null argument");
    if (mode < WG_IMAGE_PER_POL || mode > WG_IMAGE_WSTACK)
        return fail(WG_E_INVALID_ARG, "unknown image mode %d", mode);
    if (mode == WG_IMAGE_WSTACK && (!th->t.stacking || gh->g.n_chan % th->t.K != 0))
        return fail(WG_E_INVALID_ARG, "WG_IMAGE_WSTACK needs a WG_TABLE_WSTACK table and n_chan a multiple of its %d planes",
                    th->t.K);
    if (std::fabs(th->t.du - gh->g.du) > 1e-12 * gh->g.du) return fail(WG_E_SHAPE, "table du differs from grid du");
    return launch_correct(gh->g, th->t, mode, image_out, S(stream));
}

}  // extern "C"
