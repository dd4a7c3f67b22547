// Image finaliser (thesis Sec. 4.7, Algorithm "finalizer") for one grid:
//   1. inverse FFT of each polarised grid: cuFFT C2C (FP32), batched over polarisations with
//      stride P; centring (u = 0 at N/2 -> l = 0 at N/2) by the (-1)^(x+y) modulation before
//      and (-1)^(mx+my) after the transform (N even);
//   2. real part, divided by the normaliser N_p (eq. "normalizer"); Stokes I as the mean of
//      polarisations 0 and P-1;
//   3. divided by the taper psi_0(c, 2 du l) psi_0(c, 2 du m) (eq. "convgrid");
//   4. divided by sinc(pi l du / beta) sinc(pi m du / beta) (eq. "coversampled"),
//      with l = (k - N/2) / (N du), so 2 du l = 2 (k - N/2) / N and pi l du / beta =
//      pi (k - N/2) / (N beta).
// A polarisation whose normaliser is zero (no data) gives a zero image.
#include "internal.cuh"

namespace wg {

__global__ void k_corr_vec(const double* __restrict__ coef, int ncoef, int N, int beta, double* __restrict__ corr)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const double eta = 2.0 * (double)(k - N / 2) / (double)N;
    const double t = pswf_eval_dev(coef, ncoef, eta);
    const double x = M_PI * (double)(k - N / 2) / ((double)N * beta);
    const double sn = (x == 0.0) ? 1.0 : sin(x) / x;
    corr[k] = t * sn;
}

__global__ void k_modulate(const float2* __restrict__ src, float2* __restrict__ dst, int N, int P)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)N * N * P) return;
    const int64_t pix = idx / P;
    const int y = (int)(pix / N), x = (int)(pix - (int64_t)y * N);
    float2 v = src[idx];
    if ((x + y) & 1) v = make_float2(-v.x, -v.y);
    dst[idx] = v;
}

__global__ void k_finish(const float2* __restrict__ f, int N, int P, const double* __restrict__ corr,
                         const double* __restrict__ norm, int mode, float* __restrict__ img)
{
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (int64_t)N * N) return;
    const int my = (int)(pix / N), mx = (int)(pix - (int64_t)my * N);
    const double sg = ((mx + my) & 1) ? -1.0 : 1.0;
    const double c = corr[mx] * corr[my];
    double v0 = 0.0;
    for (int p = 0; p < P; ++p) {
        const double np = norm[p];
        const double v = (np != 0.0) ? sg * (double)f[pix * P + p].x / (np * c) : 0.0;
        if (mode == WG_IMAGE_PER_POL) {
            img[(int64_t)p * N * N + pix] = (float)v;
        } else if (p == 0) {
            v0 = v;
        }
        if (mode == WG_IMAGE_STOKES_I && p == P - 1) img[pix] = (float)((P == 1) ? v : 0.5 * (v0 + v));
    }
}

int launch_correct(Grid& g, const Table& t, int mode, float* image, cudaStream_t s)
{
    const int N = g.n, P = g.n_pol;
    if (!g.scratch) {
        if (cudaMalloc(&g.scratch, sizeof(float2) * (size_t)N * N * P) != cudaSuccess ||
            cudaMalloc(&g.corr, sizeof(double) * N) != cudaSuccess) {
            cudaGetLastError();
            return fail(WG_E_OOM, "cannot allocate the FFT scratch grid");
        }
    }
    if (!g.plan_ok) {
        int n[2] = {N, N};
        if (cufftPlanMany(&g.plan, 2, n, n, P, 1, n, P, 1, CUFFT_C2C, P) != CUFFT_SUCCESS)
            return fail(WG_E_CUDA, "cufftPlanMany(%d x %d, batch %d) failed", N, N, P);
        g.plan_ok = true;
    }
    if (g.corr_s0 != t.s0 || g.corr_beta != t.beta) {
        double* coef = nullptr;
        WG_CUDA(cudaMalloc(&coef, sizeof(double) * t.pswf.size()));
        WG_CUDA(cudaMemcpy(coef, t.pswf.data(), sizeof(double) * t.pswf.size(), cudaMemcpyHostToDevice));
        k_corr_vec<<<(N + 127) / 128, 128, 0, s>>>(coef, (int)t.pswf.size(), N, t.beta, g.corr);
        WG_LAUNCHED("k_corr_vec");
        WG_CUDA(cudaStreamSynchronize(s));
        cudaFree(coef);
        g.corr_s0 = t.s0;
        g.corr_beta = t.beta;
    }
    if (cufftSetStream(g.plan, s) != CUFFT_SUCCESS) return fail(WG_E_CUDA, "cufftSetStream failed");
    const int64_t tot = (int64_t)N * N * P;
    const size_t img_stride = (mode == WG_IMAGE_PER_POL) ? (size_t)P * N * N : (size_t)N * N;
    for (int c = 0; c < g.n_chan; ++c) {
        k_modulate<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g.data + (size_t)c * tot, g.scratch, N, P);
        WG_LAUNCHED("k_modulate");
        if (cufftExecC2C(g.plan, reinterpret_cast<cufftComplex*>(g.scratch), reinterpret_cast<cufftComplex*>(g.scratch),
                         CUFFT_INVERSE) != CUFFT_SUCCESS)
            return fail(WG_E_CUDA, "cufftExecC2C failed");
        k_finish<<<(unsigned)(((int64_t)N * N + 255) / 256), 256, 0, s>>>(g.scratch, N, P, g.corr, g.norm + (size_t)c * P,
                                                                          mode, image + (size_t)c * img_stride);
        WG_LAUNCHED("k_finish");
    }
    return WG_OK;
}

}  // namespace wg
