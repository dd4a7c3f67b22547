// Convolution-function generator on the GPU: thesis Sec. 4.2, Algorithm "convgen".
//
// Per w-plane k (w_k = w_max (k/(K-1))^2, square-root spacing, Sec. 4.2.1):
//   1. sample taper(l) taper(m) gbar_w(l, m) on an N_k x N_k image patch covering the field of
//      view l, m in [-1/(2 du), 1/(2 du)); gbar_w = 1/g_w = exp(+j 2 pi w (n - 1)) (Sec. 2.2.1);
//      the taper is psi_0(c, eta), eta = 2 du l, c = pi S0 / 2; the eta = -1 sample (no +1
//      partner) is zero; screen samples outside l^2 + m^2 < 1 are zero;
//   2. zero-pad to M = beta N_k and take a forward FFT (cuFFT Z2Z, FP64); the result samples
//      C_w at du / beta (eq. "local:o"); centring uses the (-1)^(i+j) modulation on both sides;
//   3. normalise by C_0(0,0) (Sec. 4.2.3);
//   4. support: outermost sample with |C| > threshold (Chebyshev radius R in oversampled units,
//      S = 2 ceil(R / beta) + 1), or the prescribed support ("normal" mode, Sec. 4.2.1);
//   5. trim into beta^2 sub-kernels of S x S row-major samples: sample [i][j] of sub-kernel
//      (fv, fu) is C(beta (i - h) - fv, beta (j - h) - fu), h = (S-1)/2, rows <-> v (eq.
//      "choose"), sub-kernels ordered (fv, fu), fv, fu in (-beta/2, beta/2];
//   6. zeta = sum of real parts of each sub-kernel (eq. "sum"), in FP64 before rounding to FP32.
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace wg {

__global__ void k_taper_patch(const double* coef, int ncoef, int n_k, double* t)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_k) return;
    double eta = 2.0 * (double)(i - n_k / 2) / (double)n_k;
    t[i] = (i == 0) ? 0.0 : pswf_eval_dev(coef, ncoef, eta);
}

// n - 1 = -r^2 / (1 + sqrt(1 - r^2)), zero screen outside the unit disk
__device__ __forceinline__ double2 screen(double w, double l, double m)
{
    double r2 = l * l + m * m;
    if (!(r2 < 1.0)) return make_double2(0.0, 0.0);
    double nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
    double s, c;
    sincospi(2.0 * w * nm1, &s, &c);
    return make_double2(c, s);
}

// padded patch with the centring modulation (-1)^(iu + iv)
__global__ void k_fill_plane(const double* t, int n_k, int M, double du, double w, double2* out)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M * M) return;
    int iv = (int)(idx / M), iu = (int)(idx - (int64_t)iv * M);
    int o = M / 2 - n_k / 2;
    int pv = iv - o, pu = iu - o;
    double2 v = make_double2(0.0, 0.0);
    if (pv >= 0 && pv < n_k && pu >= 0 && pu < n_k) {
        double tt = t[pv] * t[pu];
        if (tt != 0.0) {
            double l = (2.0 * (double)(pu - n_k / 2) / (double)n_k) / (2.0 * du);
            double m = (2.0 * (double)(pv - n_k / 2) / (double)n_k) / (2.0 * du);
            double2 s = screen(w, l, m);
            v = make_double2(tt * s.x, tt * s.y);
            if ((iu + iv) & 1) v = make_double2(-v.x, -v.y);
        }
    }
    out[idx] = v;
}

// C_0(0,0) of the un-normalised FFT: sum over the patch of taper x taper x screen(w = 0)
__global__ void k_dc(const double* t, int n_k, double du, double* out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int idx = threadIdx.x; idx < n_k * n_k; idx += blockDim.x) {
        int pv = idx / n_k, pu = idx - pv * n_k;
        double tt = t[pv] * t[pu];
        double l = (2.0 * (double)(pu - n_k / 2) / (double)n_k) / (2.0 * du);
        double m = (2.0 * (double)(pv - n_k / 2) / (double)n_k) / (2.0 * du);
        s += tt * screen(0.0, l, m).x;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Chebyshev radius (oversampled units) of the outermost sample with |C| > thr * norm
__global__ void k_support_radius(const double2* C, int M, double thr2, int* radius)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int r = -1;
    if (idx < (int64_t)M * M) {
        double2 v = C[idx];
        if (v.x * v.x + v.y * v.y > thr2) {
            int iv = (int)(idx / M), iu = (int)(idx - (int64_t)iv * M);
            r = max(abs(iv - M / 2), abs(iu - M / 2));
        }
    }
    for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0 && r >= 0) atomicMax(radius, r);
}

// one block per sub-kernel: trim, normalise, round to float, and zeta
__global__ void k_trim(const double2* C, int M, int beta, int S, const double* normp, float2* out,
                       double* zeta)
{
    __shared__ double red[256];
    const int sub = blockIdx.x;                      // (fv - lo) * beta + (fu - lo)
    const int lo = -((beta - 1) / 2);
    const int fv = sub / beta + lo, fu = sub % beta + lo;
    const int h = (S - 1) / 2;
    const double inv = 1.0 / *normp;
    double acc = 0.0;
    float2* dst = out + (int64_t)sub * S * S;
    for (int s = threadIdx.x; s < S * S; s += blockDim.x) {
        int i = s / S, j = s - i * S;
        int ov = beta * (i - h) - fv, ou = beta * (j - h) - fu;
        int kv = ov + M / 2, ku = ou + M / 2;
        double re = 0.0, im = 0.0;
        if (kv >= 0 && kv < M && ku >= 0 && ku < M) {
            double2 v = C[(int64_t)kv * M + ku];
            double sg = ((kv + ku) & 1) ? -inv : inv;
            re = v.x * sg;
            im = v.y * sg;
        }
        dst[s] = make_float2((float)re, (float)im);
        acc += re;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) zeta[sub] = red[0];
}

static int default_nk(int s_max)
{
    int n = 64;
    while (n < 2 * s_max) n *= 2;
    return n;
}

__global__ void k_table_lp(const float2* __restrict__ src, int64_t n, int store, void* __restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 v = src[i];
    if (store == WG_BF16)
        reinterpret_cast<__nv_bfloat162*>(dst)[i] = __floats2bfloat162_rn(v.x, v.y);
    else
        reinterpret_cast<__half2*>(dst)[i] = __floats2half2_rn(v.x, v.y);
}

int set_table_store(Table& t, int store)
{
    if (store != WG_F32 && store != WG_BF16 && store != WG_F16) return fail(WG_E_INVALID_ARG, "unknown store dtype %d", store);
    cudaFree(t.data_lp);
    t.data_lp = nullptr;
    t.store = WG_F32;
    if (store == WG_F32) return WG_OK;
    if (cudaMalloc(&t.data_lp, 4 * (size_t)std::max<int64_t>(t.n_samples, 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(WG_E_OOM, "cannot allocate the low-precision table");
    }
    if (t.n_samples > 0) {
        k_table_lp<<<(unsigned)((t.n_samples + 255) / 256), 256>>>(t.data, t.n_samples, store, t.data_lp);
        WG_LAUNCHED("k_table_lp");
    }
    WG_CUDA(cudaDeviceSynchronize());
    t.store = store;
    return WG_OK;
}

int free_table(Table& t)
{
    cudaFree(t.data_lp);
    t.data_lp = nullptr;
    cudaFree(t.data);
    cudaFree(t.zeta);
    cudaFree(t.supports_d);
    cudaFree(t.offsets_d);
    cudaFree(t.wbounds_d);
    cudaFree(t.wbounds_f);
    cudaFree(t.zeta_f);
    t.data = nullptr;
    t.zeta = nullptr;
    t.supports_d = t.offsets_d = nullptr;
    t.wbounds_d = nullptr;
    t.wbounds_f = nullptr;
    t.zeta_f = nullptr;
    return WG_OK;
}

static int finish_layout(Table& t)
{
    t.offsets.resize(t.K);
    int64_t off = 0;
    t.max_support = 0;
    for (int k = 0; k < t.K; ++k) {
        t.offsets[k] = (int)off;
        off += (int64_t)t.beta * t.beta * t.supports[k] * t.supports[k];
        t.max_support = std::max(t.max_support, t.supports[k]);
    }
    if (off >= (int64_t)1 << 31) return fail(WG_E_OOB_SUPPORT, "kernel table has %lld samples (limit 2^31)", (long long)off);
    t.n_samples = off;
    if (cudaMalloc(&t.data, sizeof(float2) * std::max<int64_t>(off, 1)) != cudaSuccess ||
        cudaMalloc(&t.zeta, sizeof(double) * t.K * t.beta * t.beta) != cudaSuccess ||
        cudaMalloc(&t.supports_d, sizeof(int) * t.K) != cudaSuccess ||
        cudaMalloc(&t.offsets_d, sizeof(int) * t.K) != cudaSuccess ||
        cudaMalloc(&t.wbounds_d, sizeof(double) * t.K) != cudaSuccess ||
        cudaMalloc(&t.wbounds_f, sizeof(float) * t.K) != cudaSuccess ||
        cudaMalloc(&t.zeta_f, sizeof(float) * t.K * t.beta * t.beta) != cudaSuccess) {
        cudaGetLastError();
        free_table(t);
        return fail(WG_E_OOM, "cannot allocate the kernel table (%lld samples)", (long long)off);
    }
    WG_CUDA(cudaMemcpy(t.supports_d, t.supports.data(), sizeof(int) * t.K, cudaMemcpyHostToDevice));
    WG_CUDA(cudaMemcpy(t.offsets_d, t.offsets.data(), sizeof(int) * t.K, cudaMemcpyHostToDevice));
    // nearest plane in sqrt(w): plane k is chosen when b_k <= w < b_{k+1}, with
    // b_m = w_max (t t), t = (m - 1/2) / (K - 1), m = 1..K (b_K bounds the last plane)
    std::vector<double> wb(t.K, 0.0);
    if (t.K > 1)
        for (int m = 1; m <= t.K; ++m) {
            const double tm = (m - 0.5) / (double)(t.K - 1);
            wb[m - 1] = t.w_max * (tm * tm);
        }
    WG_CUDA(cudaMemcpy(t.wbounds_d, wb.data(), sizeof(double) * t.K, cudaMemcpyHostToDevice));
    std::vector<float> wbf(t.K);
    for (int m = 0; m < t.K; ++m) wbf[m] = (float)wb[m];     // round to nearest
    WG_CUDA(cudaMemcpy(t.wbounds_f, wbf.data(), sizeof(float) * t.K, cudaMemcpyHostToDevice));
    return WG_OK;
}

__global__ void k_zeta_f32(const double* __restrict__ z, int n, float* __restrict__ zf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) zf[i] = (float)z[i];
}

int build_table(const wg_table_desc& d, Table& t, cudaStream_t s)
{
    const int K = d.n_wplanes, beta = d.oversample;
    t.K = K;
    t.beta = beta;
    t.s0 = d.taper_support;
    t.w_max = d.w_max;
    t.du = d.du;
    t.pswf = pswf_coefficients(M_PI * d.taper_support / 2.0);
    int n_k = d.n_k;
    if (n_k == 0) {
        if ((d.support_mode & 0xFF) == WG_SUPPORT_PRESCRIBED) {
            int smax = 1;
            for (int k = 0; k < K; ++k) smax = std::max(smax, d.supports[k]);
            n_k = default_nk(smax);
        } else {
            n_k = 256;
        }
    }
    const int M = beta * n_k;
    if ((int64_t)M * M > ((int64_t)1 << 31)) return fail(WG_E_INVALID_ARG, "beta * n_k = %d too large", M);
    // device scratch
    double *coef = nullptr, *taper = nullptr, *norm = nullptr;
    double2* plane = nullptr;
    int* radius = nullptr;
    auto cleanup = [&]() {
        cudaFree(coef); cudaFree(taper); cudaFree(norm); cudaFree(plane); cudaFree(radius);
    };
    if (cudaMalloc(&coef, sizeof(double) * t.pswf.size()) != cudaSuccess ||
        cudaMalloc(&taper, sizeof(double) * n_k) != cudaSuccess ||
        cudaMalloc(&norm, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&plane, sizeof(double2) * (size_t)M * M) != cudaSuccess ||
        cudaMalloc(&radius, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(WG_E_OOM, "cannot allocate the %dx%d FFT plane", M, M);
    }
    cufftHandle plan;
    if (cufftPlan2d(&plan, M, M, CUFFT_Z2Z) != CUFFT_SUCCESS) {
        cleanup();
        return fail(WG_E_CUDA, "cufftPlan2d(%d) failed", M);
    }
    cufftSetStream(plan, s);
    int rc = WG_OK;
    std::vector<double> wk(K);
    for (int k = 0; k < K; ++k) wk[k] = (K == 1) ? 0.0 : d.w_max * ((double)k / (K - 1)) * ((double)k / (K - 1));
    // w-stacking: every plane holds the w = 0 kernel; the plane values w_k stay for the correction
    t.stacking = (d.support_mode & WG_TABLE_WSTACK) != 0;
    t.w_planes = wk;
    std::vector<double> wscreen(K);
    for (int k = 0; k < K; ++k) wscreen[k] = t.stacking ? 0.0 : wk[k];
    do {
        if (cudaMemcpyAsync(coef, t.pswf.data(), sizeof(double) * t.pswf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) { rc = fail(WG_E_CUDA, "copy"); break; }
        k_taper_patch<<<(n_k + 127) / 128, 128, 0, s>>>(coef, (int)t.pswf.size(), n_k, taper);
        count_launch();
        k_dc<<<1, 256, 0, s>>>(taper, n_k, d.du, norm);
        count_launch();
        const int64_t tot = (int64_t)M * M;
        const int nb = (int)((tot + 255) / 256);
        // supports
        t.supports.assign(K, 1);
        if ((d.support_mode & 0xFF) == WG_SUPPORT_PRESCRIBED) {
            for (int k = 0; k < K; ++k) t.supports[k] = d.supports[k];
        } else {
            double nrm = 0;
            if (cudaMemcpyAsync(&nrm, norm, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) { rc = fail(WG_E_CUDA, "norm readback"); break; }
            const double thr2 = (d.threshold * nrm) * (d.threshold * nrm);
            for (int k = 0; k < K && rc == WG_OK; ++k) {
                k_fill_plane<<<nb, 256, 0, s>>>(taper, n_k, M, d.du, wscreen[k], plane);
                count_launch();
                if (cufftExecZ2Z(plan, plane, plane, CUFFT_FORWARD) != CUFFT_SUCCESS) { rc = fail(WG_E_CUDA, "cufftExecZ2Z"); break; }
                cudaMemsetAsync(radius, 0xff, sizeof(int), s);
                k_support_radius<<<nb, 256, 0, s>>>(plane, M, thr2, radius);
                count_launch();
                int R = -1;
                if (cudaMemcpyAsync(&R, radius, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) { rc = fail(WG_E_CUDA, "support readback"); break; }
                t.supports[k] = (R < 0) ? 1 : 2 * ((R + beta - 1) / beta) + 1;
            }
            if (rc != WG_OK) break;
        }
        for (int k = 0; k < K; ++k) {
            if (t.supports[k] < 1 || t.supports[k] % 2 == 0) { rc = fail(WG_E_INVALID_ARG, "support %d of plane %d must be odd and positive", t.supports[k], k); break; }
            if (t.supports[k] > kMaxSupport) { rc = fail(WG_E_OOB_SUPPORT, "support %d of plane %d exceeds %d", t.supports[k], k, kMaxSupport); break; }
        }
        if (rc != WG_OK) break;
        rc = finish_layout(t);
        if (rc != WG_OK) break;
        for (int k = 0; k < K; ++k) {
            k_fill_plane<<<nb, 256, 0, s>>>(taper, n_k, M, d.du, wscreen[k], plane);
            count_launch();
            if (cufftExecZ2Z(plan, plane, plane, CUFFT_FORWARD) != CUFFT_SUCCESS) { rc = fail(WG_E_CUDA, "cufftExecZ2Z"); break; }
            k_trim<<<beta * beta, 256, 0, s>>>(plane, M, beta, t.supports[k], norm, t.data + t.offsets[k],
                                                t.zeta + (int64_t)k * beta * beta);
            count_launch();
        }
        if (rc != WG_OK) break;
        {
            const int nz = K * beta * beta;
            k_zeta_f32<<<(nz + 255) / 256, 256, 0, s>>>(t.zeta, nz, t.zeta_f);
            count_launch();
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "conv_table_build");
    } while (0);
    cufftDestroy(plan);
    cleanup();
    if (rc != WG_OK) free_table(t);
    return rc;
}

int import_table(int K, int beta, double w_max, double du, int s0, const int* supports,
                 const double* data, const double* zeta, Table& t)
{
    t.K = K;
    t.beta = beta;
    t.s0 = s0;
    t.w_max = w_max;
    t.stacking = false;
    t.w_planes.assign(K, 0.0);
    for (int k = 0; k < K && K > 1; ++k) t.w_planes[k] = w_max * ((double)k / (K - 1)) * ((double)k / (K - 1));
    t.du = du;
    t.pswf = pswf_coefficients(M_PI * s0 / 2.0);
    t.supports.assign(supports, supports + K);
    for (int k = 0; k < K; ++k)
        if (t.supports[k] < 1 || t.supports[k] % 2 == 0 || t.supports[k] > kMaxSupport)
            return fail(WG_E_INVALID_ARG, "support %d of plane %d must be odd, in [1, %d]", t.supports[k], k, kMaxSupport);
    int rc = finish_layout(t);
    if (rc != WG_OK) return rc;
    std::vector<float2> h((size_t)t.n_samples);
    for (int64_t i = 0; i < t.n_samples; ++i) h[i] = make_float2((float)data[2 * i], (float)data[2 * i + 1]);
    std::vector<float> zf((size_t)K * beta * beta);
    for (size_t i = 0; i < zf.size(); ++i) zf[i] = (float)zeta[i];
    if (cudaMemcpy(t.data, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.zeta, zeta, sizeof(double) * K * beta * beta, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.zeta_f, zf.data(), sizeof(float) * zf.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_table(t);
        return fail(WG_E_CUDA, "table upload failed");
    }
    return WG_OK;
}

}  // namespace wg
