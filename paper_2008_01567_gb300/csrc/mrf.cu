// 4D q-GGMRF prior proximal map (Sec. III, Eq. (5) with the 4D MRF prior of
// Sec. VII: 26 spatial + 2 temporal neighbours) by 16-colour ICD.
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

}  // namespace msf

using namespace msf;

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
