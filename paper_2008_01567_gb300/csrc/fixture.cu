// Blind correction of fixtures outside the field of view (Appendix A,
// Algorithm 2).  Given the measurements y and a reconstruction x = recon(y, A):
//   x^m = mask(x)        cylinder of radius r_mask about the rotation axis
//   e   = y - A x^m      (the projector's forward)
//   p   = blur(e)        separable Gaussian along u then v of every view
//   c   = <e, p> / <p, p>   (FP64, one scalar for the scan)
//   y^corr = y - c p
// The fixtures' shadow is smooth (broad tubes, blurred by the rotation), so the
// blur keeps it and removes what is left of the object's projection.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace msf {

constexpr int FIX_MAX_R = 64;                 // largest blur radius (taps 2R + 1)
constexpr int FIX_BLOCKS = 152 * 8;
__constant__ float c_fix_taps[2 * FIX_MAX_R + 1];

// x^m = x inside the cylinder |(x, y)| <= r_mask (voxel centres), 0 outside.
__global__ void fix_mask_kernel(const float* __restrict__ x, float* __restrict__ xm, int nx, int ny, size_t N,
                                double vox, double r2) {
    const size_t plane = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i % plane;
        const double yc = ((double)(r / nx) - 0.5 * (ny - 1)) * vox;
        const double xc = ((double)(r % nx) - 0.5 * (nx - 1)) * vox;
        xm[i] = (xc * xc + yc * yc <= r2) ? x[i] : 0.0f;
    }
}

// e = y - e (e holds A x^m)
__global__ void fix_resid_kernel(const float* __restrict__ y, float* __restrict__ e, size_t M) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x)
        e[i] = y[i] - e[i];
}

// One blur pass over every detector row (AXIS 0: along u, rows of nu) or
// column (AXIS 1: along v) of every view; taps outside the detector are zero.
// Grid-stride over output pixels; FP32 sums in a fixed tap order.
template <int AXIS>
__global__ void fix_blur_kernel(const float* __restrict__ in, float* __restrict__ out, int nu, int nv, size_t M,
                                int R) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
        const int iu = (int)(i % nu);
        const int iv = (int)((i / nu) % nv);
        float acc = 0.0f;
        if (AXIS == 0) {
            for (int k = -R; k <= R; ++k) {
                const int u = iu + k;
                if (u >= 0 && u < nu) acc = fmaf(c_fix_taps[k + R], in[i + k], acc);
            }
        } else {
            for (int k = -R; k <= R; ++k) {
                const int v = iv + k;
                if (v >= 0 && v < nv) acc = fmaf(c_fix_taps[k + R], in[i + (ptrdiff_t)k * nu], acc);
            }
        }
        out[i] = acc;
    }
}

// per-block partial sums of e.p and p.p (FP64)
__global__ void __launch_bounds__(256) fix_dot_kernel(const float* __restrict__ e, const float* __restrict__ p,
                                                      size_t M, double* __restrict__ part) {
    double ep = 0.0, pp = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
        const double pv = p[i];
        ep += (double)e[i] * pv;
        pp += pv * pv;
    }
    ep = block_sum_f64(ep);
    pp = block_sum_f64(pp);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ep;
        part[FIX_BLOCKS + blockIdx.x] = pp;
    }
}

// c = sum(e.p) / sum(p.p) over the partials in a fixed order (0 when p = 0)
__global__ void fix_coef_kernel(const double* __restrict__ part, double* __restrict__ c) {
    double ep = 0.0, pp = 0.0;
    for (int i = threadIdx.x; i < FIX_BLOCKS; i += blockDim.x) {
        ep += part[i];
        pp += part[FIX_BLOCKS + i];
    }
    ep = block_sum_f64(ep);
    pp = block_sum_f64(pp);
    if (threadIdx.x == 0) c[0] = pp > 0.0 ? ep / pp : 0.0;
}

// y^corr = y - c p (in place on p)
__global__ void fix_apply_kernel(const float* __restrict__ y, float* __restrict__ p, const double* __restrict__ c,
                                 size_t M) {
    const float cf = (float)c[0];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x)
        p[i] = fmaf(-cf, p[i], y[i]);
}

}  // namespace msf

struct msf_fixcorr {
    msf_projector* proj = nullptr;
    msf_vol vol;
    size_t N = 0, M = 0;
    float *d_xm = nullptr, *d_e = nullptr, *d_tmp = nullptr;
    double *d_part = nullptr, *d_c = nullptr, *h_c = nullptr;
};

using namespace msf;

extern "C" msf_status msf_fixcorr_create(msf_projector* p, msf_fixcorr** out) {
    MSF_REQUIRE(p && out, "msf_fixcorr_create: NULL argument");
    *out = nullptr;
    MSF_TRY(check_device());
    msf_fixcorr* f = new msf_fixcorr();
    f->proj = p;
    f->vol = *projector_volume(p);
    f->N = (size_t)f->vol.nx * f->vol.ny * f->vol.nz * f->vol.nt;
    f->M = projector_sino_size(p);
    if (cudaMalloc(&f->d_xm, f->N * 4) != cudaSuccess || cudaMalloc(&f->d_e, f->M * 4) != cudaSuccess ||
        cudaMalloc(&f->d_tmp, f->M * 4) != cudaSuccess || cudaMalloc(&f->d_part, 2 * FIX_BLOCKS * 8) != cudaSuccess ||
        cudaMalloc(&f->d_c, 8) != cudaSuccess || cudaMallocHost(&f->h_c, 8) != cudaSuccess) {
        cudaGetLastError();
        msf_fixcorr_destroy(f);
        return fail(MSF_ERR_NOMEM, "msf_fixcorr_create: out of device memory");
    }
    *out = f;
    return MSF_OK;
}

extern "C" void msf_fixcorr_destroy(msf_fixcorr* f) {
    if (!f) return;
    cudaFree(f->d_xm); cudaFree(f->d_e); cudaFree(f->d_tmp); cudaFree(f->d_part); cudaFree(f->d_c);
    if (f->h_c) cudaFreeHost(f->h_c);
    delete f;
}

extern "C" msf_status msf_fixture_correct(msf_fixcorr* f, const float* d_y, const float* d_x, double r_mask,
                                          double blur_sigma, float* d_ycorr, double* h_c, void* stream) {
    MSF_REQUIRE(f && d_y && d_x && d_ycorr, "msf_fixture_correct: NULL argument");
    MSF_REQUIRE(d_ycorr != d_y, "msf_fixture_correct: y and y_corr must differ");
    MSF_REQUIRE(r_mask > 0 && isfinite(r_mask), "msf_fixture_correct: r_mask must be positive");
    MSF_REQUIRE(blur_sigma > 0 && ceil(3.0 * blur_sigma) <= FIX_MAX_R,
                "msf_fixture_correct: blur_sigma must lie in (0, %g] pixels", FIX_MAX_R / 3.0);
    const int R = (int)ceil(3.0 * blur_sigma);
    std::vector<double> g(2 * R + 1);
    double sum = 0.0;
    for (int k = -R; k <= R; ++k) sum += (g[k + R] = exp(-(double)k * k / (2.0 * blur_sigma * blur_sigma)));
    std::vector<float> gf(2 * R + 1);
    for (int k = 0; k <= 2 * R; ++k) gf[k] = (float)(g[k] / sum);
    cudaStream_t st = as_stream(stream);
    MSF_TRY_CUDA(cudaMemcpyToSymbolAsync(c_fix_taps, gf.data(), gf.size() * sizeof(float), 0, cudaMemcpyHostToDevice,
                                         st));
    const msf_vol& v = f->vol;
    {
        MSF_PROF("fix_mask", st);
        fix_mask_kernel<<<FIX_BLOCKS, 256, 0, st>>>(d_x, f->d_xm, v.nx, v.ny, f->N, v.voxel, r_mask * r_mask);
        MSF_LAUNCH_CHECK();
    }
    MSF_TRY(msf_project(f->proj, f->d_xm, f->d_e, reinterpret_cast<void*>(st)));
    int gnu = 0, gnv = 0;
    projector_detector(f->proj, &gnu, &gnv);
    {
        MSF_PROF("fix_resid", st);
        fix_resid_kernel<<<FIX_BLOCKS, 256, 0, st>>>(d_y, f->d_e, f->M);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("fix_blur", st);
        fix_blur_kernel<0><<<FIX_BLOCKS, 256, 0, st>>>(f->d_e, f->d_tmp, gnu, gnv, f->M, R);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("fix_blur", st);
        fix_blur_kernel<1><<<FIX_BLOCKS, 256, 0, st>>>(f->d_tmp, d_ycorr, gnu, gnv, f->M, R);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("fix_dot", st);
        fix_dot_kernel<<<FIX_BLOCKS, 256, 0, st>>>(f->d_e, d_ycorr, f->M, f->d_part);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("fix_dot", st);
        fix_coef_kernel<<<1, 1024, 0, st>>>(f->d_part, f->d_c);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("fix_apply", st);
        fix_apply_kernel<<<FIX_BLOCKS, 256, 0, st>>>(d_y, d_ycorr, f->d_c, f->M);
        MSF_LAUNCH_CHECK();
    }
    if (h_c) {
        MSF_TRY_CUDA(cudaMemcpyAsync(f->h_c, f->d_c, 8, cudaMemcpyDeviceToHost, st));
        MSF_TRY_CUDA(cudaStreamSynchronize(st));
        *h_c = *f->h_c;
    }
    return MSF_OK;
}
