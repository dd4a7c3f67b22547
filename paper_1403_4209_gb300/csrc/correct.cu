// Image finaliser (thesis Sec. 4.7, Algorithm "finalizer") for one grid:
//   1. inverse FFT of each polarised grid: cuFFT C2C (FP32) over contiguous N x N planes; the
//      needed polarisations of a group of channels (groups sized to a 1 GiB scratch) are first
//      split out of the pixel-interleaved grid, so Stokes I copies and transforms only the
//      parallel hands.  Centring (u = 0 at N/2 -> l = 0 at N/2) uses the
//      (-1)^(x+y) modulation before and (-1)^(mx+my) after the transform (N even);
//   2. real part, divided by the normaliser N_p (eq. "normalizer"); Stokes I as the mean of
//      polarisations 0 and P-1;
//   3. divided by the taper psi_0(c, 2 du l) psi_0(c, 2 du m) (eq. "convgrid");
//   4. divided by sinc(pi l du / beta) sinc(pi m du / beta) (eq. "coversampled"),
//      with l = (k - N/2) / (N du), so 2 du l = 2 (k - N/2) / N and pi l du / beta =
//      pi (k - N/2) / (N beta).
// The divisions are multiplications by reciprocals prepared once in FP64 and applied in FP32.
// A polarisation whose normaliser is zero (no data) gives a zero image.
// WG_IMAGE_WSTACK sums the planes of each channel after the inverse FFT, each multiplied by its
// exp(+j2pi w_k (n-1)) (eq. "stacking"), then takes steps 2-4 with the channel's N_p.
// WG_IMAGE_STOKES_LINEAR / _CIRCULAR combine the complex per-polarisation images, each divided by
// its own N_p, into I, Q, U, V (step 2 "convert to multiple-Stokes image and normalise").
// WG_IMAGE_PER_POL_RAW skips the division by N_p; WG_IMAGE_TRANSPOSE applies the exact transpose
// of that map (the adjoint of Re(inverse FFT) under the real inner product is the forward FFT of
// the real image): grid = (-1)^(x+y) FFT_forward((-1)^(mx+my) img / (taper sinc)).
#include "internal.cuh"

namespace wg {

__global__ void k_corr_vec(const double* __restrict__ coef, int ncoef, int N, int beta, double* __restrict__ corr,
                           float* __restrict__ icorr)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const double eta = 2.0 * (double)(k - N / 2) / (double)N;
    const double t = pswf_eval_dev(coef, ncoef, eta);
    const double x = M_PI * (double)(k - N / 2) / ((double)N * beta);
    const double sn = (x == 0.0) ? 1.0 : sin(x) / x;
    corr[k] = t * sn;
    icorr[k] = (float)(1.0 / (t * sn));
}

__global__ void k_inv_norm(const double* __restrict__ norm, int n, float* __restrict__ inv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) inv[i] = (norm[i] != 0.0) ? (float)(1.0 / norm[i]) : 0.f;
}

__global__ void k_modulate(const float2* __restrict__ src, float2* __restrict__ dst, int N, int P, int64_t total)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int64_t pix = idx / P;
    const int64_t rem = pix % ((int64_t)N * N);
    const int y = (int)(rem / N), x = (int)(rem - (int64_t)y * N);
    float2 v = src[idx];
    if ((x + y) & 1) v = make_float2(-v.x, -v.y);
    dst[idx] = v;
}

// step 1 input for a group of G channels: the needed polarisations (np of them, listed in pols)
// of each pixel, times (-1)^(x+y), into contiguous planes f[pi][gch][N][N] for unit-stride FFTs
__global__ void k_split(const float2* __restrict__ grid, float2* __restrict__ f, int N, int P, int G, int np,
                        int4 pols)
{
    const int64_t nn = (int64_t)N * N;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;     // over G x N x N pixels
    if (q >= (int64_t)G * nn) return;
    const int64_t gch = q / nn, pix = q - gch * nn;
    const int y = (int)(pix / N), x = (int)(pix - (int64_t)y * N);
    const float sg = ((x + y) & 1) ? -1.f : 1.f;
    const float2* src = grid + q * P;
    const int pl[4] = {pols.x, pols.y, pols.z, pols.w};
    for (int pi = 0; pi < np; ++pi) {
        const float2 v = src[pl[pi]];
        f[((int64_t)pi * G + gch) * nn + pix] = make_float2(sg * v.x, sg * v.y);
    }
}

// steps 2-4 from the planes of k_split after their inverse FFTs (one thread per pixel of the group)
__global__ void k_finish_planes(const float2* __restrict__ f, int N, int P, int G, int64_t npix,
                                const float* __restrict__ icorr, const float* __restrict__ inv_norm, int mode,
                                float* __restrict__ img)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npix) return;
    const int64_t nn = (int64_t)N * N;
    const int64_t gch = q / nn, pix = q - gch * nn;
    const int my = (int)(pix / N), mx = (int)(pix - (int64_t)my * N);
    const float cc = ((mx + my) & 1 ? -1.f : 1.f) * icorr[mx] * icorr[my];
    const float* in = inv_norm ? inv_norm + gch * P : nullptr;
    auto plane = [&](int pi) { return f[((int64_t)pi * G + gch) * nn + pix]; };
    if (mode == WG_IMAGE_STOKES_I) {
        const float v0 = plane(0).x * in[0] * cc;
        img[gch * nn + pix] = (P == 1) ? v0 : 0.5f * (v0 + plane(1).x * in[P - 1] * cc);
        return;
    }
    if (mode == WG_IMAGE_PER_POL || mode == WG_IMAGE_PER_POL_RAW) {
        for (int p = 0; p < P; ++p) img[(gch * P + p) * nn + pix] = plane(p).x * (in ? in[p] : 1.f) * cc;
        return;
    }
    // Stokes from the complex per-polarisation images z_p = f_p / N_p (step 2)
    float2 z[4];
    for (int p = 0; p < P; ++p) {
        const float2 v = plane(p);
        z[p] = make_float2(v.x * in[p] * cc, v.y * in[p] * cc);
    }
    float* o = img + (gch * P) * nn + pix;
    if (P == 1) {
        o[0] = z[0].x;
    } else if (P == 2) {
        o[0] = 0.5f * (z[0].x + z[1].x);
        o[nn] = 0.5f * (z[0].x - z[1].x);
    } else {
        const float par_s = 0.5f * (z[0].x + z[3].x), par_d = 0.5f * (z[0].x - z[3].x);
        const float crs_s = 0.5f * (z[1].x + z[2].x), crs_d = 0.5f * (z[1].y - z[2].y);   // Re(-j(z1 - z2))/2
        o[0] = par_s;                                                                      // I
        if (mode == WG_IMAGE_STOKES_LINEAR) {
            o[nn] = par_d;            // Q = (XX - YY)/2
            o[2 * nn] = crs_s;        // U = (XY + YX)/2
            o[3 * nn] = crs_d;        // V = -j (XY - YX)/2
        } else {
            o[nn] = crs_s;            // Q = (RL + LR)/2
            o[2 * nn] = crs_d;        // U = -j (RL - LR)/2
            o[3 * nn] = par_d;        // V = (RR - LL)/2
        }
    }
}

// transpose, step 1: scratch = (-1)^(mx+my) img / (taper sinc) as complex, per group of channels
__global__ void k_image_in(const float* __restrict__ img, int N, int P, int64_t npix, const float* __restrict__ icorr,
                           float2* __restrict__ f)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npix) return;
    const int64_t nn = (int64_t)N * N;
    const int64_t gch = q / nn, pix = q - gch * nn;
    const int my = (int)(pix / N), mx = (int)(pix - (int64_t)my * N);
    const float cc = ((mx + my) & 1 ? -1.f : 1.f) * icorr[mx] * icorr[my];
    for (int p = 0; p < P; ++p) f[q * P + p] = make_float2(img[(gch * P + p) * nn + pix] * cc, 0.f);
}

// w-stacking (eq. "stacking"): n - 1 at every pixel, NaN outside the unit disk (l^2 + m^2 >= 1)
__global__ void k_nm1(int N, double du, double* __restrict__ nm1)
{
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (int64_t)N * N) return;
    const int my = (int)(pix / N), mx = (int)(pix - (int64_t)my * N);
    const double l = (double)(mx - N / 2) / ((double)N * du), m = (double)(my - N / 2) / ((double)N * du);
    const double r2 = l * l + m * m;
    nm1[pix] = (r2 < 1.0) ? -r2 / (1.0 + sqrt(1.0 - r2)) : __longlong_as_double(0x7FF8000000000000ll);
}

// acc[p][pix] += f[pix][p] exp(+j 2 pi w_k (n - 1)) for the P polarisations of one grid channel
// (the (-1)^(mx+my) demodulation, common to all planes, is applied at the end)
__global__ void k_stack_acc(const float2* __restrict__ f, int P, int64_t nn, const double* __restrict__ nm1, double wk,
                            float2* __restrict__ acc)
{
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= nn) return;
    const double v = nm1[pix];
    if (!(v == v)) return;                              // outside the unit disk: screen 0
    const double x = wk * v;
    float sn, cs;
    sincospif((float)(2.0 * (x - rint(x))), &sn, &cs);
    for (int p = 0; p < P; ++p) {
        const float2 a = f[pix * P + p];
        float2& o = acc[p * nn + pix];
        o.x += a.x * cs - a.y * sn;
        o.y += a.x * sn + a.y * cs;
    }
}

// image[c][p][pix] = Re(acc) (-1)^(mx+my) / (taper sinc)(l) / (taper sinc)(m) / N_p(c)
__global__ void k_stack_finish(const float2* __restrict__ acc, int N, int P, int64_t npix, const float* __restrict__ icorr,
                               const float* __restrict__ inv_norm, int K, float* __restrict__ img)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over channels x pols x pixels
    if (q >= npix) return;
    const int64_t nn = (int64_t)N * N;
    const int64_t cp = q / nn, pix = q - cp * nn;
    const int c = (int)(cp / P), p = (int)(cp - (int64_t)c * P);
    const int my = (int)(pix / N), mx = (int)(pix - (int64_t)my * N);
    const float cc = ((mx + my) & 1 ? -1.f : 1.f) * icorr[mx] * icorr[my];
    img[q] = acc[q].x * cc * inv_norm[((int64_t)c * K) * P + p];
}

int launch_correct(Grid& g, const Table& t, int mode, float* image, cudaStream_t s)
{
    const int N = g.n, P = g.n_pol, C = g.n_chan;
    const int64_t per_chan = (int64_t)N * N * P;
    if (!g.scratch) {
        // channels per group: the largest divisor of C whose scratch fits in 1 GiB
        int G = 1;
        for (int d = 1; d <= C; ++d)
            if (C % d == 0 && (int64_t)d * per_chan * (int64_t)sizeof(float2) <= ((int64_t)1 << 30)) G = d;
        if (cudaMalloc(&g.scratch, sizeof(float2) * (size_t)G * per_chan) != cudaSuccess ||
            cudaMalloc(&g.corr, sizeof(double) * N) != cudaSuccess ||
            cudaMalloc(&g.icorr, sizeof(float) * N) != cudaSuccess ||
            cudaMalloc(&g.inv_norm, sizeof(float) * C * P) != cudaSuccess) {
            cudaGetLastError();
            return fail(WG_E_OOM, "cannot allocate the FFT scratch grid");
        }
        g.scratch_chans = G;
    }
    const int G = g.scratch_chans;
    if (!g.plan_ok) {
        int n[2] = {N, N};
        if (cufftPlanMany(&g.plan, 2, n, n, P, (int)per_chan, n, P, (int)per_chan, CUFFT_C2C, G) != CUFFT_SUCCESS)
            return fail(WG_E_CUDA, "cufftPlanMany(%d x %d, stride %d, batch %d) failed", N, N, P, G);
        g.plan_ok = true;
    }
    if (g.corr_s0 != t.s0 || g.corr_beta != t.beta) {
        double* coef = nullptr;
        WG_CUDA(cudaMalloc(&coef, sizeof(double) * t.pswf.size()));
        WG_CUDA(cudaMemcpy(coef, t.pswf.data(), sizeof(double) * t.pswf.size(), cudaMemcpyHostToDevice));
        k_corr_vec<<<(N + 127) / 128, 128, 0, s>>>(coef, (int)t.pswf.size(), N, t.beta, g.corr, g.icorr);
        WG_LAUNCHED("k_corr_vec");
        WG_CUDA(cudaStreamSynchronize(s));
        cudaFree(coef);
        g.corr_s0 = t.s0;
        g.corr_beta = t.beta;
    }
    if (cufftSetStream(g.plan, s) != CUFFT_SUCCESS) return fail(WG_E_CUDA, "cufftSetStream failed");
    const int64_t tot = (int64_t)G * per_chan, npix = (int64_t)G * N * N;
    if (mode == WG_IMAGE_TRANSPOSE) {
        for (int c0 = 0; c0 < C; c0 += G) {
            k_image_in<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(image + (size_t)c0 * P * N * N, N, P, npix,
                                                                      g.icorr, g.scratch);
            WG_LAUNCHED("k_image_in");
            for (int p = 0; p < P; ++p) {
                cufftComplex* d = reinterpret_cast<cufftComplex*>(g.scratch + p);
                if (cufftExecC2C(g.plan, d, d, CUFFT_FORWARD) != CUFFT_SUCCESS) return fail(WG_E_CUDA, "cufftExecC2C failed");
            }
            k_modulate<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g.scratch, g.data + (size_t)c0 * per_chan, N, P, tot);
            WG_LAUNCHED("k_modulate");
        }
        return WG_OK;
    }
    if (mode == WG_IMAGE_WSTACK) {
        const int K = t.K, Cin = C / K;
        const int64_t nn = (int64_t)N * N;
        void* buf = nullptr;
        const size_t acc_bytes = sizeof(float2) * (size_t)Cin * P * nn;
        if (cudaMallocAsync(&buf, acc_bytes + sizeof(double) * (size_t)nn, s) != cudaSuccess) {
            cudaGetLastError();
            return fail(WG_E_OOM, "cannot allocate the w-stacking accumulators (%zu bytes)", acc_bytes);
        }
        float2* acc = static_cast<float2*>(buf);
        double* nm1 = reinterpret_cast<double*>(static_cast<char*>(buf) + acc_bytes);
        int rc = WG_OK;
        if (cudaMemsetAsync(acc, 0, acc_bytes, s) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "w-stacking");
        if (rc == WG_OK) {
            k_nm1<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(N, g.du, nm1);
            WG_LAUNCHED("k_nm1");
            k_inv_norm<<<(C * P + 127) / 128, 128, 0, s>>>(g.norm, C * P, g.inv_norm);
            WG_LAUNCHED("k_inv_norm");
        }
        for (int c0 = 0; c0 < C && rc == WG_OK; c0 += G) {
            k_modulate<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g.data + (size_t)c0 * per_chan, g.scratch, N, P, tot);
            WG_LAUNCHED("k_modulate");
            for (int p = 0; p < P && rc == WG_OK; ++p) {
                cufftComplex* d = reinterpret_cast<cufftComplex*>(g.scratch + p);
                if (cufftExecC2C(g.plan, d, d, CUFFT_INVERSE) != CUFFT_SUCCESS) rc = fail(WG_E_CUDA, "cufftExecC2C failed");
            }
            for (int gc = c0; gc < c0 + G && rc == WG_OK; ++gc) {
                k_stack_acc<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(g.scratch + (size_t)(gc - c0) * per_chan, P, nn,
                                                                         nm1, t.w_planes[gc % K],
                                                                         acc + (size_t)(gc / K) * P * nn);
                WG_LAUNCHED("k_stack_acc");
            }
        }
        if (rc == WG_OK) {
            const int64_t npix_all = (int64_t)Cin * P * nn;
            k_stack_finish<<<(unsigned)((npix_all + 255) / 256), 256, 0, s>>>(acc, N, P, npix_all, g.icorr, g.inv_norm, K,
                                                                              image);
            WG_LAUNCHED("k_stack_finish");
        }
        cudaFreeAsync(buf, s);
        return rc;
    }
    const bool raw = (mode == WG_IMAGE_PER_POL_RAW);
    if (!raw) {
        k_inv_norm<<<(C * P + 127) / 128, 128, 0, s>>>(g.norm, C * P, g.inv_norm);
        WG_LAUNCHED("k_inv_norm");
    }
    if (!g.plan_c_ok) {
        int n[2] = {N, N};
        if (cufftPlanMany(&g.plan_c, 2, n, nullptr, 1, N * N, nullptr, 1, N * N, CUFFT_C2C, G) != CUFFT_SUCCESS)
            return fail(WG_E_CUDA, "cufftPlanMany(%d x %d, contiguous, batch %d) failed", N, N, G);
        g.plan_c_ok = true;
    }
    if (cufftSetStream(g.plan_c, s) != CUFFT_SUCCESS) return fail(WG_E_CUDA, "cufftSetStream failed");
    // the polarisations the mode needs: Stokes I only the parallel hands
    int np = P;
    int4 pols = make_int4(0, 1, 2, 3);
    if (mode == WG_IMAGE_STOKES_I) {
        np = (P == 1) ? 1 : 2;
        pols = make_int4(0, P - 1, 0, 0);
    }
    const size_t img_stride = (mode == WG_IMAGE_STOKES_I) ? (size_t)N * N : (size_t)P * N * N;
    for (int c0 = 0; c0 < C; c0 += G) {
        k_split<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(g.data + (size_t)c0 * per_chan, g.scratch, N, P, G, np,
                                                               pols);
        WG_LAUNCHED("k_split");
        for (int pi = 0; pi < np; ++pi) {
            cufftComplex* d = reinterpret_cast<cufftComplex*>(g.scratch + (size_t)pi * G * N * N);
            if (cufftExecC2C(g.plan_c, d, d, CUFFT_INVERSE) != CUFFT_SUCCESS) return fail(WG_E_CUDA, "cufftExecC2C failed");
        }
        k_finish_planes<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(g.scratch, N, P, G, npix, g.icorr,
                                                                       raw ? nullptr : g.inv_norm + (size_t)c0 * P, mode,
                                                                       image + (size_t)c0 * img_stride);
        WG_LAUNCHED("k_finish");
    }
    return WG_OK;
}

}  // namespace wg
