// 4D q-GGMRF prior proximal map (Sec. III, Eq. (5) with the 4D MRF prior of
// Sec. VII: 26 spatial + 2 temporal neighbours) by 16-colour ICD, and the
// direct MAP solve of Eq. (3) with that prior (the MBIR + 4D-MRF comparison of
// Sec. VI) by majorise-minimise with CG on the surrogate problem.
//
// The 16 parity colours ((pt*2+pz)*2+py)*2+px never contain two neighbours,
// so all voxels of one colour update in parallel and the sweep is
// deterministic: the GPU reproduces a sequential colour-ordered sweep exactly
// in real arithmetic.  One launch per colour.
#include <math.h>

#include "common.cuh"

namespace msf {

struct MrfDims {
    int nx, ny, nz, nt;
    int px, py, pz, pt;          // parities of the colour
    int hx, hy, hz, ht;          // voxels of that colour along each axis
    float inv_s2;                // 1/sigma^2
    float inv_tsx;               // 1/(T sigma_x)
    float pq;                    // p - q
    float q_over_p;
    float inv_2sx2;              // 1/(2 sigma_x^2)  (p = 2)
    float bf, be, bc, bt;        // face, edge, corner, temporal weights
};

// Surrogate coefficient a(D) = rho'(D)/(2D) of the q-GGMRF potential with p = 2:
//   a(D) = 1/(2 sx^2) * (1 + (q/p) r)/(1 + r)^2,   r = |D/(T sx)|^(p-q).
// r is formed as exp2((p-q) log2 |D/(T sx)|) with the hardware approximations
// (about 2^-21 relative), far inside the FP32 tolerance of the agent.
__device__ __forceinline__ float qggmrf_coef(float D, const MrfDims& m) {
    const float r = m.pq == 0.0f ? 1.0f : exp2f(m.pq * __log2f(fabsf(D) * m.inv_tsx));
    const float op = 1.0f + r;
    return m.inv_2sx2 * (1.0f + m.q_over_p * r) / (op * op);
}

__global__ void __launch_bounds__(128) icd_colour_kernel(const float* __restrict__ v,
                                                         float* __restrict__ z, MrfDims m) {
    const int hxv = blockIdx.x * 32 + threadIdx.x;
    const int hyv = blockIdx.y * 4 + threadIdx.y;
    const int hzv = blockIdx.z % m.hz;
    const int htv = blockIdx.z / m.hz;
    if (hxv >= m.hx || hyv >= m.hy) return;
    const int ix = 2 * hxv + m.px, iy = 2 * hyv + m.py, iz = 2 * hzv + m.pz, t = 2 * htv + m.pt;
    const size_t sxy = (size_t)m.nx * m.ny;
    const size_t fs = sxy * m.nz;
    const size_t s = (size_t)t * fs + (size_t)iz * sxy + (size_t)iy * m.nx + ix;
    const float zs = z[s];
    float num = v[s] * m.inv_s2, den = m.inv_s2;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int jz = iz + dz;
        if (jz < 0 || jz >= m.nz) continue;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int jy = iy + dy;
            if (jy < 0 || jy >= m.ny) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int jx = ix + dx;
                if ((dx | dy | dz) == 0 || jx < 0 || jx >= m.nx) continue;
                const int mm = (dx != 0) + (dy != 0) + (dz != 0);
                const float b = mm == 1 ? m.bf : (mm == 2 ? m.be : m.bc);
                const float zr = z[(size_t)t * fs + (size_t)jz * sxy + (size_t)jy * m.nx + jx];
                const float ba = b * qggmrf_coef(zs - zr, m);
                num += 2.0f * ba * zr;
                den += 2.0f * ba;
            }
        }
    }
    if (t > 0) {
        const float zr = z[s - fs];
        const float ba = m.bt * qggmrf_coef(zs - zr, m);
        num += 2.0f * ba * zr;
        den += 2.0f * ba;
    }
    if (t + 1 < m.nt) {
        const float zr = z[s + fs];
        const float ba = m.bt * qggmrf_coef(zs - zr, m);
        num += 2.0f * ba * zr;
        den += 2.0f * ba;
    }
    z[s] = num / den;
}

// ------------------------------------------------------------------ direct MAP

constexpr int MAP_BLOCKS = 152 * 8;

// (L_a x)_s = sum_r b_sr a(anchor_s - anchor_r) (x_s - x_r) over the 26 spatial
// and 2 temporal neighbours of s (free boundaries): half the gradient of the
// prior's quadratic surrogate built at `anchor`.
__device__ __forceinline__ float surrogate_lap(const float* __restrict__ anchor, const float* __restrict__ x,
                                               size_t s, int ix, int iy, int iz, int t, const MrfDims& m) {
    const size_t sxy = (size_t)m.nx * m.ny, fs = sxy * m.nz;
    const float as = anchor[s], xs = x[s];
    float acc = 0.0f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int jz = iz + dz;
        if (jz < 0 || jz >= m.nz) continue;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int jy = iy + dy;
            if (jy < 0 || jy >= m.ny) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int jx = ix + dx;
                if ((dx | dy | dz) == 0 || jx < 0 || jx >= m.nx) continue;
                const int mm = (dx != 0) + (dy != 0) + (dz != 0);
                const float b = mm == 1 ? m.bf : (mm == 2 ? m.be : m.bc);
                const size_t r = (size_t)t * fs + (size_t)jz * sxy + (size_t)jy * m.nx + jx;
                acc = fmaf(b * qggmrf_coef(as - anchor[r], m), xs - x[r], acc);
            }
        }
    }
    if (t > 0) acc = fmaf(m.bt * qggmrf_coef(as - anchor[s - fs], m), xs - x[s - fs], acc);
    if (t + 1 < m.nt) acc = fmaf(m.bt * qggmrf_coef(as - anchor[s + fs], m), xs - x[s + fs], acc);
    return acc;
}

enum MapLapMode { MAP_INIT = 0, MAP_Q = 1 };

// MAP_INIT: r = data - 2 beta L_a x  (data = A^T Lambda (y - A x) held in r),
//           d = r, partial r.r
// MAP_Q:    q = data + 2 beta L_a d  (data = A^T Lambda A d held in q), partial d.q
// One grid-stride pass over all voxels; per-block FP64 partials.
template <int MODE>
__global__ void __launch_bounds__(256) map_lap_kernel(const float* __restrict__ anchor, const float* __restrict__ x,
                                                      float* __restrict__ out, float* __restrict__ out2,
                                                      float two_beta, MrfDims m, double* __restrict__ partial) {
    const size_t sxy = (size_t)m.nx * m.ny, fs = sxy * m.nz, N = fs * m.nt;
    double dot = 0.0;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < N; s += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(s / fs);
        const size_t r = s - (size_t)t * fs;
        const int iz = (int)(r / sxy);
        const int rr = (int)(r - (size_t)iz * sxy);
        const int iy = rr / m.nx, ix = rr - iy * m.nx;
        const float L = surrogate_lap(anchor, x, s, ix, iy, iz, t, m);
        if (MODE == MAP_INIT) {
            const float v = fmaf(-two_beta, L, out[s]);
            out[s] = v;
            out2[s] = v;
            dot += (double)v * (double)v;
        } else {
            const float v = fmaf(two_beta, L, out[s]);
            out[s] = v;
            dot += (double)x[s] * (double)v;
        }
    }
    const double b = block_sum_f64(dot);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// x += alpha d ; r -= alpha q ; partial r.r
__global__ void __launch_bounds__(256) map_update_kernel(float* __restrict__ x, float* __restrict__ r,
                                                         const float* __restrict__ d, const float* __restrict__ q,
                                                         const double* __restrict__ scal, size_t N,
                                                         double* __restrict__ partial) {
    const float a = (float)scal[1];
    double dot = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        x[i] = fmaf(a, d[i], x[i]);
        const float rn = fmaf(-a, q[i], r[i]);
        r[i] = rn;
        dot += (double)rn * (double)rn;
    }
    const double b = block_sum_f64(dot);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// d = r + beta_cg d
__global__ void __launch_bounds__(256) map_dir_kernel(float* __restrict__ d, const float* __restrict__ r,
                                                      const double* __restrict__ scal, size_t N) {
    const float b = (float)scal[2];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
        d[i] = fmaf(b, d[i], r[i]);
}

enum MapFin { MFIN_RR0 = 0, MFIN_ALPHA = 1, MFIN_BETA = 2 };

// scal = {rr, alpha, beta}: one block sums the MAP_BLOCKS partials in a fixed order.
template <int MODE>
__global__ void map_finalize_kernel(const double* __restrict__ partial, double* __restrict__ scal,
                                    int* __restrict__ status) {
    double s = 0.0;
    for (int i = threadIdx.x; i < MAP_BLOCKS; i += blockDim.x) s += partial[i];
    s = block_sum_f64(s);
    if (threadIdx.x == 0) {
        if (!isfinite(s)) atomicExch(status, (int)MSF_ERR_NUMERIC);
        if (MODE == MFIN_RR0) {
            scal[0] = s;
        } else if (MODE == MFIN_ALPHA) {
            scal[1] = (s != 0.0) ? scal[0] / s : 0.0;
        } else {
            scal[2] = (scal[0] != 0.0) ? s / scal[0] : 0.0;
            scal[0] = s;
        }
    }
}

// Sinogram weighting: RES: s = Lambda (y - s); LAM: s = Lambda s; COST: partial
// sums of Lambda (y - s)^2.
enum MapSino { MS_RES = 0, MS_LAM = 1, MS_COST = 2 };
template <int MODE>
__global__ void __launch_bounds__(256) map_sino_kernel(float* __restrict__ s, const float* __restrict__ y,
                                                       const float* __restrict__ lam, size_t M,
                                                       double* __restrict__ partial) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
        if (MODE == MS_RES) {
            s[i] = lam[i] * (y[i] - s[i]);
        } else if (MODE == MS_LAM) {
            s[i] = lam[i] * s[i];
        } else {
            const double e = (double)y[i] - (double)s[i];
            acc += (double)lam[i] * e * e;
        }
    }
    if (MODE == MS_COST) {
        const double b = block_sum_f64(acc);
        if (threadIdx.x == 0) partial[blockIdx.x] = b;
    }
}

// rho(D) = D^2/(2 sx^2) * u/(1+u), u = |D/(T sx)|^(q-2)  (p = 2), in FP64.
__device__ __forceinline__ double qggmrf_rho64(double D, double q, double tsx, double sx) {
    const double ad = fabs(D);
    if (ad == 0.0) return 0.0;
    const double u = pow(ad / tsx, q - 2.0);
    return D * D / (2.0 * sx * sx) * (u / (1.0 + u));
}

// Partial sums of h(x) = sum over unordered neighbour pairs b_sr rho(x_s - x_r)
// (each pair once: the neighbours at a positive lexicographic offset).
__global__ void __launch_bounds__(256) map_prior_cost_kernel(const float* __restrict__ x, MrfDims m, double q,
                                                             double T, double sx, double* __restrict__ partial) {
    const size_t sxy = (size_t)m.nx * m.ny, fs = sxy * m.nz, N = fs * m.nt;
    const double s_ = 6.0 + 12.0 / sqrt(2.0) + 8.0 / sqrt(3.0);
    const double bf = 1.0 / s_, be = 1.0 / (sqrt(2.0) * s_), bc = 1.0 / (sqrt(3.0) * s_);
    double acc = 0.0;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < N; s += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(s / fs);
        const size_t r0 = s - (size_t)t * fs;
        const int iz = (int)(r0 / sxy);
        const int rr = (int)(r0 - (size_t)iz * sxy);
        const int iy = rr / m.nx, ix = rr - iy * m.nx;
        const double xs = x[s];
        for (int dz = 0; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const bool pos = dz > 0 || (dy > 0 || (dy == 0 && dx > 0));
                    if (!pos) continue;
                    const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                    if (jx < 0 || jx >= m.nx || jy < 0 || jy >= m.ny || jz >= m.nz) continue;
                    const int mm = (dx != 0) + (dy != 0) + (dz != 0);
                    const double b = mm == 1 ? bf : (mm == 2 ? be : bc);
                    acc += b * qggmrf_rho64(xs - (double)x[(size_t)t * fs + (size_t)jz * sxy + (size_t)jy * m.nx + jx],
                                            q, T * sx, sx);
                }
        if (t + 1 < m.nt) acc += (double)m.bt * qggmrf_rho64(xs - (double)x[s + fs], q, T * sx, sx);
    }
    const double b = block_sum_f64(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

__global__ void map_cost_finalize_kernel(const double* __restrict__ pdata, const double* __restrict__ pprior,
                                         double* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < MAP_BLOCKS; i += blockDim.x) {
        a += pdata[i];
        b += pprior[i];
    }
    a = block_sum_f64(a);
    b = block_sum_f64(b);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

static msf_status mrf_dims(const msf_vol* vol, const msf_mrf* prm, double sigma, MrfDims* out) {
    MSF_REQUIRE(prm->p == 2.0 && prm->q >= 1.0 && prm->q <= 2.0,
                "q-GGMRF: need p == 2 and 1 <= q <= 2 (got p=%g q=%g)", prm->p, prm->q);
    MSF_REQUIRE(prm->T > 0 && prm->sigma_x > 0 && prm->b_temporal >= 0,
                "q-GGMRF: T and sigma_x must be positive and b_temporal >= 0");
    MrfDims& m = *out;
    m.nx = vol->nx; m.ny = vol->ny; m.nz = vol->nz; m.nt = vol->nt;
    m.px = m.py = m.pz = m.pt = 0;
    m.hx = m.hy = m.hz = m.ht = 0;
    m.inv_s2 = (float)(1.0 / (sigma * sigma));
    m.inv_tsx = (float)(1.0 / (prm->T * prm->sigma_x));
    m.pq = (float)(prm->p - prm->q);
    m.q_over_p = (float)(prm->q / prm->p);
    m.inv_2sx2 = (float)(1.0 / (2.0 * prm->sigma_x * prm->sigma_x));
    const double s = 6.0 + 12.0 / sqrt(2.0) + 8.0 / sqrt(3.0);
    m.bf = (float)(1.0 / s);
    m.be = (float)(1.0 / (sqrt(2.0) * s));
    m.bc = (float)(1.0 / (sqrt(3.0) * s));
    m.bt = (float)prm->b_temporal;
    return MSF_OK;
}

}  // namespace msf

struct msf_map {
    msf_projector* proj = nullptr;
    msf_vol vol;
    size_t N = 0, M = 0;
    float *d_r = nullptr, *d_d = nullptr, *d_q = nullptr, *d_anchor = nullptr, *d_s = nullptr;
    double *d_part = nullptr, *d_part2 = nullptr, *d_scal = nullptr, *d_cost = nullptr;
    double* h_cost = nullptr;   // pinned [2]
    int* d_status = nullptr;
    int* h_status = nullptr;    // pinned
};

using namespace msf;

extern "C" msf_status msf_map_create(msf_projector* p, msf_map** out) {
    MSF_REQUIRE(p && out, "msf_map_create: NULL argument");
    *out = nullptr;
    MSF_TRY(check_device());
    msf_map* m = new msf_map();
    m->proj = p;
    m->vol = *projector_volume(p);
    m->N = (size_t)m->vol.nx * m->vol.ny * m->vol.nz * m->vol.nt;
    m->M = projector_sino_size(p);
    if (cudaMalloc(&m->d_r, m->N * 4) != cudaSuccess || cudaMalloc(&m->d_d, m->N * 4) != cudaSuccess ||
        cudaMalloc(&m->d_q, m->N * 4) != cudaSuccess || cudaMalloc(&m->d_anchor, m->N * 4) != cudaSuccess ||
        cudaMalloc(&m->d_s, m->M * 4) != cudaSuccess || cudaMalloc(&m->d_part, MAP_BLOCKS * 8) != cudaSuccess ||
        cudaMalloc(&m->d_part2, MAP_BLOCKS * 8) != cudaSuccess || cudaMalloc(&m->d_scal, 4 * 8) != cudaSuccess ||
        cudaMalloc(&m->d_cost, 2 * 8) != cudaSuccess || cudaMalloc(&m->d_status, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&m->h_cost, 2 * 8) != cudaSuccess || cudaMallocHost(&m->h_status, sizeof(int)) != cudaSuccess ||
        cudaMemset(m->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        msf_map_destroy(m);
        return fail(MSF_ERR_NOMEM, "msf_map_create: out of device memory");
    }
    *out = m;
    return MSF_OK;
}

extern "C" void msf_map_destroy(msf_map* m) {
    if (!m) return;
    cudaFree(m->d_r); cudaFree(m->d_d); cudaFree(m->d_q); cudaFree(m->d_anchor); cudaFree(m->d_s);
    cudaFree(m->d_part); cudaFree(m->d_part2); cudaFree(m->d_scal); cudaFree(m->d_cost); cudaFree(m->d_status);
    if (m->h_cost) cudaFreeHost(m->h_cost);
    if (m->h_status) cudaFreeHost(m->h_status);
    delete m;
}

extern "C" msf_status msf_map_solve(msf_map* m, const msf_mrf* prm, double beta, const float* d_y,
                                    const float* d_lambda, float* d_x, int n_outer, int n_cg, void* stream) {
    MSF_REQUIRE(m && prm && d_y && d_lambda && d_x, "msf_map_solve: NULL argument");
    MSF_REQUIRE(beta > 0 && isfinite(beta), "msf_map_solve: beta must be positive");
    MSF_REQUIRE(n_outer >= 0 && n_cg >= 0, "msf_map_solve: iteration counts must be >= 0");
    MrfDims md;
    MSF_TRY(mrf_dims(&m->vol, prm, 1.0, &md));
    if (n_outer == 0 || n_cg == 0) return MSF_OK;
    cudaStream_t st = as_stream(stream);
    void* sv = reinterpret_cast<void*>(st);
    const float two_beta = (float)(2.0 * beta);
    const size_t N = m->N, M = m->M;
    for (int o = 0; o < n_outer; ++o) {
        MSF_TRY_CUDA(cudaMemcpyAsync(m->d_anchor, d_x, N * 4, cudaMemcpyDeviceToDevice, st));
        // r = A^T Lambda (y - A x) - 2 beta L_a x ; d = r ; rr = r.r
        MSF_TRY(msf_project(m->proj, d_x, m->d_s, sv));
        {
            MSF_PROF("map_sino", st);
            map_sino_kernel<MS_RES><<<MAP_BLOCKS, 256, 0, st>>>(m->d_s, d_y, d_lambda, M, nullptr);
            MSF_LAUNCH_CHECK();
        }
        MSF_TRY(msf_backproject(m->proj, m->d_s, m->d_r, sv));
        {
            MSF_PROF("map_lap", st);
            map_lap_kernel<MAP_INIT><<<MAP_BLOCKS, 256, 0, st>>>(m->d_anchor, d_x, m->d_r, m->d_d, two_beta, md,
                                                                 m->d_part);
            MSF_LAUNCH_CHECK();
        }
        {
            MSF_PROF("map_finalize", st);
            map_finalize_kernel<MFIN_RR0><<<1, 1024, 0, st>>>(m->d_part, m->d_scal, m->d_status);
            MSF_LAUNCH_CHECK();
        }
        for (int k = 0; k < n_cg; ++k) {
            // q = A^T Lambda A d + 2 beta L_a d ; alpha = rr / d.q
            MSF_TRY(msf_project(m->proj, m->d_d, m->d_s, sv));
            {
                MSF_PROF("map_sino", st);
                map_sino_kernel<MS_LAM><<<MAP_BLOCKS, 256, 0, st>>>(m->d_s, nullptr, d_lambda, M, nullptr);
                MSF_LAUNCH_CHECK();
            }
            MSF_TRY(msf_backproject(m->proj, m->d_s, m->d_q, sv));
            {
                MSF_PROF("map_lap", st);
                map_lap_kernel<MAP_Q><<<MAP_BLOCKS, 256, 0, st>>>(m->d_anchor, m->d_d, m->d_q, nullptr, two_beta, md,
                                                                  m->d_part);
                MSF_LAUNCH_CHECK();
            }
            {
                MSF_PROF("map_finalize", st);
                map_finalize_kernel<MFIN_ALPHA><<<1, 1024, 0, st>>>(m->d_part, m->d_scal, m->d_status);
                MSF_LAUNCH_CHECK();
            }
            {   // x += alpha d ; r -= alpha q
                MSF_PROF("map_update", st);
                map_update_kernel<<<MAP_BLOCKS, 256, 0, st>>>(d_x, m->d_r, m->d_d, m->d_q, m->d_scal, N, m->d_part);
                MSF_LAUNCH_CHECK();
            }
            {   // beta_cg = r.r / rr
                MSF_PROF("map_finalize", st);
                map_finalize_kernel<MFIN_BETA><<<1, 1024, 0, st>>>(m->d_part, m->d_scal, m->d_status);
                MSF_LAUNCH_CHECK();
            }
            {   // d = r + beta_cg d
                MSF_PROF("map_dir", st);
                map_dir_kernel<<<MAP_BLOCKS, 256, 0, st>>>(m->d_d, m->d_r, m->d_scal, N);
                MSF_LAUNCH_CHECK();
            }
        }
    }
    return MSF_OK;
}

extern "C" msf_status msf_map_cost(msf_map* m, const msf_mrf* prm, double beta, const float* d_y,
                                   const float* d_lambda, const float* d_x, double* h_cost, void* stream) {
    MSF_REQUIRE(m && prm && d_y && d_lambda && d_x && h_cost, "msf_map_cost: NULL argument");
    MrfDims md;
    MSF_TRY(mrf_dims(&m->vol, prm, 1.0, &md));
    cudaStream_t st = as_stream(stream);
    MSF_TRY(msf_project(m->proj, d_x, m->d_s, reinterpret_cast<void*>(st)));
    {
        MSF_PROF("map_cost", st);
        map_sino_kernel<MS_COST><<<MAP_BLOCKS, 256, 0, st>>>(m->d_s, d_y, d_lambda, m->M, m->d_part);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("map_cost", st);
        map_prior_cost_kernel<<<MAP_BLOCKS, 256, 0, st>>>(d_x, md, prm->q, prm->T, prm->sigma_x, m->d_part2);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("map_cost", st);
        map_cost_finalize_kernel<<<1, 1024, 0, st>>>(m->d_part, m->d_part2, m->d_cost);
        MSF_LAUNCH_CHECK();
    }
    MSF_TRY_CUDA(cudaMemcpyAsync(m->h_cost, m->d_cost, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSF_TRY_CUDA(cudaMemcpyAsync(m->h_status, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MSF_TRY_CUDA(cudaStreamSynchronize(st));
    if (*m->h_status != 0) return fail(MSF_ERR_NUMERIC, "msf_map_solve: a non-finite CG scalar occurred");
    h_cost[0] = 0.5 * m->h_cost[0] + beta * m->h_cost[1];
    return MSF_OK;
}

extern "C" msf_status msf_prox_qggmrf(const msf_vol* vol, const msf_mrf* prm, const float* d_v, float* d_x,
                                      double sigma, int n_sweeps, void* stream) {
    MSF_REQUIRE(vol && prm && d_v && d_x, "msf_prox_qggmrf: NULL argument");
    MSF_REQUIRE(vol->nx > 0 && vol->ny > 0 && vol->nz > 0 && vol->nt > 0,
                "msf_prox_qggmrf: volume sizes must be positive");
    MSF_REQUIRE(prm->p == 2.0 && prm->q >= 1.0 && prm->q <= 2.0,
                "msf_prox_qggmrf: need p == 2 and 1 <= q <= 2 (got p=%g q=%g)", prm->p, prm->q);
    MSF_REQUIRE(prm->T > 0 && prm->sigma_x > 0 && prm->b_temporal >= 0 && sigma > 0,
                "msf_prox_qggmrf: T, sigma_x, sigma must be positive and b_temporal >= 0");
    MSF_REQUIRE(n_sweeps >= 0, "msf_prox_qggmrf: n_sweeps must be >= 0");
    MSF_REQUIRE((long long)((vol->nz + 1) / 2) * ((vol->nt + 1) / 2) <= 65535,
                "msf_prox_qggmrf: nz*nt too large for the launch grid");
    cudaStream_t st = as_stream(stream);
    MrfDims m;
    m.nx = vol->nx; m.ny = vol->ny; m.nz = vol->nz; m.nt = vol->nt;
    m.inv_s2 = (float)(1.0 / (sigma * sigma));
    m.inv_tsx = (float)(1.0 / (prm->T * prm->sigma_x));
    m.pq = (float)(prm->p - prm->q);
    m.q_over_p = (float)(prm->q / prm->p);
    m.inv_2sx2 = (float)(1.0 / (2.0 * prm->sigma_x * prm->sigma_x));
    const double s = 6.0 + 12.0 / sqrt(2.0) + 8.0 / sqrt(3.0);
    m.bf = (float)(1.0 / s);
    m.be = (float)(1.0 / (sqrt(2.0) * s));
    m.bc = (float)(1.0 / (sqrt(3.0) * s));
    m.bt = (float)prm->b_temporal;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        for (int col = 0; col < 16; ++col) {
            m.px = col & 1; m.py = (col >> 1) & 1; m.pz = (col >> 2) & 1; m.pt = (col >> 3) & 1;
            m.hx = (m.nx - m.px + 1) / 2; m.hy = (m.ny - m.py + 1) / 2;
            m.hz = (m.nz - m.pz + 1) / 2; m.ht = (m.nt - m.pt + 1) / 2;
            if (m.hx <= 0 || m.hy <= 0 || m.hz <= 0 || m.ht <= 0) continue;
            dim3 grid((m.hx + 31) / 32, (m.hy + 3) / 4, m.hz * m.ht);
            MSF_PROF("qggmrf_icd", st);
            icd_colour_kernel<<<grid, dim3(32, 4), 0, st>>>(d_v, d_x, m);
            MSF_LAUNCH_CHECK();
        }
    }
    return MSF_OK;
}
