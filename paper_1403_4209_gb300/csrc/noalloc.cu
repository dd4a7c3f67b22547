// grid_vis_noalloc: preparation + gridding of one small batch with no device allocation.
//
// Some callers cannot call cudaMalloc: code running while a stream is being captured into a
// CUDA graph (allocation breaks the capture), processes whose device memory is fully
// reserved by another allocator or a fixed budget, and real-time or embedded loops that must
// not touch the driver's allocator.  This entry point gives them the same result as
// vis_compress followed by grid_vis, without a work list: its scratch (the work list's
// buffers) lives in the file-scope array g_noalloc_scratch below, a fixed kNoallocBytes
// that every GPU loading this library holds until the process exits.
//
// Limits: at most WG_NOALLOC_MAX_RECORDS records (rows x channels) and WG_NOALLOC_MAX_CHAN
// channels per call; larger batches are rejected with WG_E_CAPACITY.  Every call uses the same
// scratch, which keeps the previous call's contents: the accumulators that must start at zero
// are cleared (cudaMemsetAsync) at the start of each call, and calls that overlap on the GPU
// (on different streams, or from different host threads) race on the scratch.
//
// Set-up: the first call on each device asks the runtime for the scratch's device address
// (cudaGetSymbolAddress, with that device current) and caches it; make that first call before
// any stream capture begins.
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace wg {

namespace {

constexpr int64_t kNoallocBytes = 6 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

struct Carver {
    unsigned char* base;
    int64_t off = 0;
    template <typename T>
    T* take(int64_t count)
    {
        off = (off + 255) & ~int64_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * (int64_t)sizeof(T);
        return p;
    }
};

int scratch_address(void** out)
{
    int dev = 0;
    WG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(WG_E_INVALID_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return WG_OK;
}

}  // namespace

}  // namespace wg

using namespace wg;

extern "C" int grid_vis_noalloc(const wg_grid_view* view, const wg_table* th, const wg_vis_in* in, int32_t compress,
                                void* stream)
{
    clear_error();
    if (!view || !th || !in) return fail(WG_E_INVALID_ARG, "grid_vis_noalloc: null argument");
    const Table& t = th->t;
    if (view->n < 8 || view->n > 32768 || (view->n & 1)) return fail(WG_E_INVALID_ARG, "grid side N=%d must be even in [8, 32768]", view->n);
    if (!(view->du > 0.0) || !std::isfinite(view->du))
        return fail(WG_E_INVALID_ARG, "cell size du must be positive and finite");
    if (view->n_pol != 1 && view->n_pol != 2 && view->n_pol != 4) return fail(WG_E_INVALID_ARG, "n_pol must be 1, 2 or 4");
    if (view->n_chan < 1 || view->n_chan > WG_NOALLOC_MAX_CHAN)
        return fail(WG_E_CAPACITY, "n_chan=%d exceeds the no-allocation limit %d", view->n_chan, WG_NOALLOC_MAX_CHAN);
    if (!view->data || !view->normaliser) return fail(WG_E_INVALID_ARG, "grid_vis_noalloc: null grid or normaliser");
    if (reinterpret_cast<uintptr_t>(view->data) & 15) return fail(WG_E_INVALID_ARG, "grid buffer must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(view->dropped) & 7) return fail(WG_E_INVALID_ARG, "dropped must be 8-byte aligned");
    if (in->n_chan != view->n_chan || in->n_pol != view->n_pol) return fail(WG_E_SHAPE, "vis shape differs from the grid's");
    if (in->n_rows < 0) return fail(WG_E_INVALID_ARG, "n_rows must be >= 0");
    if (compress != 0 && compress != WG_PREP_COMPRESS)
        return fail(WG_E_INVALID_ARG, "compress must be 0 or WG_PREP_COMPRESS (got %d)", compress);
    if (in->n_rows > 0 && (!in->uvw || !in->freq_hz || !in->vis || !in->weight || !in->flag))
        return fail(WG_E_INVALID_ARG, "null input array");
    if (in->vis_dtype != WG_VIS_COMPLEX64 && in->vis_dtype != WG_VIS_COMPLEX_HALF)
        return fail(WG_E_INVALID_ARG, "unknown vis_dtype %d", in->vis_dtype);
    if (in->vis_dtype == WG_VIS_COMPLEX_HALF && in->n_rows > 0 && !in->vis_scale)
        return fail(WG_E_INVALID_ARG, "vis_scale is required for half-precision visibilities");
    // the element size: 8 bytes for complex64, 4 for complex half (as vis_compress checks)
    if (reinterpret_cast<uintptr_t>(in->vis) & (in->vis_dtype == WG_VIS_COMPLEX64 ? 7 : 3))
        return fail(WG_E_INVALID_ARG, "vis is not aligned to its element size");
    if (std::fabs(t.du - view->du) > 1e-12 * view->du) return fail(WG_E_SHAPE, "table du differs from grid du");
    if (t.max_support > view->n) return fail(WG_E_OOB_SUPPORT, "support %d larger than the grid (%d)", t.max_support, view->n);
    const int64_t records = in->n_rows * (int64_t)in->n_chan;
    if (records > WG_NOALLOC_MAX_RECORDS)
        return fail(WG_E_CAPACITY, "%lld records exceed the no-allocation limit %d", (long long)records, WG_NOALLOC_MAX_RECORDS);

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != WG_OK) return rc;

    const int C = view->n_chan, P = view->n_pol;
    const int64_t cap = WG_NOALLOC_MAX_RECORDS;
    WorkList w;
    w.cap = cap;
    w.ecap = cap;
    w.C = C;
    w.P = P;
    const int rpb = std::max(1, kTileRecords / C);
    const int64_t rows_max = (cap + C - 1) / C;
    w.tile_cap = ((rows_max + rpb - 1) / rpb + 2) * C;
    w.seg_cap = cap / kSegLenMin + 2;
    Carver cv{static_cast<unsigned char*>(base)};
    w.rinfo = cv.take<int4>(cap);
    w.rclass = cv.take<uint8_t>(cap);
    w.tile_cnt = cv.take<int>(w.tile_cap);
    w.carry_q = cv.take<float2>(w.tile_cap * P);
    w.carry_last = cv.take<int>(w.tile_cap);
    w.entries = cv.take<int4>(cap);
    w.gamma = cv.take<float2>(cap * P);
    w.runs = cv.take<int2>(cap);
    w.seg_nblk = cv.take<int>(w.seg_cap);
    w.seg_off = cv.take<int>(w.seg_cap + 1);
    w.scal = cv.take<long long>(8);
    w.chan_base = cv.take<int>(C + 1);
    w.norm_priv = cv.take<double>((int64_t)kNormSlots * C * P);
    w.norm_batch = cv.take<double>((int64_t)C * P + 3 * C);
    w.stat_priv = cv.take<unsigned long long>((int64_t)kNormSlots * ST_N);
    w.stats = cv.take<unsigned long long>(ST_N);
    w.stats_batch = cv.take<unsigned long long>(ST_N);
    w.task_counter = cv.take<unsigned int>(4);
    unsigned long long* counters = cv.take<unsigned long long>(ST_N);
    if (cv.off > kNoallocBytes) return fail(WG_E_CAPACITY, "no-allocation scratch layout exceeds %lld bytes", (long long)kNoallocBytes);

    Grid g;   // non-owning view: nothing is allocated or freed
    g.n = view->n;
    g.n_pol = P;
    g.n_chan = C;
    g.du = view->du;
    g.data = static_cast<float2*>(view->data);
    g.norm = view->normaliser;
    g.counters = counters;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the statistics slot is written by every call but read by none: start it at zero so it
    // holds this call's counts rather than a sum over earlier callers
    WG_CUDA(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * ST_N, s));
    rc = launch_prep(t, g, *in, compress, w, s);
    if (rc != WG_OK) return rc;
    rc = launch_grid(g, t, w, s);
    if (rc != WG_OK) return rc;
    // entries rejected by the device-side bounds checks of preparation and gridding (cleared by
    // launch_prep), copied out for the caller
    if (view->dropped)
        WG_CUDA(cudaMemcpyAsync(view->dropped, w.scal + 3, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    return WG_OK;
}
