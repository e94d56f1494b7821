// Cone-beam Joseph projector pair and the CG data proximal map.
//
// A_n (Sec. II, Eq. (2)) is modelled as a Joseph ray-driven projector on a
// circular orbit with a flat detector (the paper defers the model to its
// cone-beam reference; the geometry is documented in msf.h).  The adjoint is a
// voxel-driven gather: each voxel enumerates the rays whose bilinear footprint
// touches it and recomputes the forward's interpolation coordinates with the
// same FP32 operations (the z crossing to within a few 1e-5 voxel): A^T is the
// transpose of the FP32 A up to rounding, without atomics.
//
// Per (view, detector column) constants are computed once in FP64 and stored
// in FP32.  A ray's direction has d_x, d_y fixed by its column and d_z = v, so
// the in-plane constants are per column and the z constants are v times
// per-column factors.  Along the major axis the crossing point at plane k is
//     f_a(k) = fa_mid + (k - c_maj) * ba          (minor in-plane axis)
//     f_z(k) = (c_z + v*c1) + (k - c_maj) * (v*inv_dmaj)
// in fractional voxel indices, and the chord per plane is
//     step = sqrt(|d_xy|^2 + v^2) * voxel/|d_maj|.
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace msf {

struct ColParams {
    float fa_mid, ba, c1, inv_dmaj;   // minor-axis line, z factors
    float dxy2, vox_over_adm, xmajor, pad;
};

struct ProjDims {
    int nx, ny, nz, nt, nu, nv, views;
    float cx, cy, cz, cu, cv;   // (n-1)/2 of each axis
    float vox, du, dv;
    float dso, dsd;
};

struct RayZ {
    float fz_mid, bz, step;
};

// The one place where a ray's z constants are formed; forward and adjoint
// both call it, with explicit round-to-nearest intrinsics so the compiler
// cannot contract the two call sites differently.
__device__ __forceinline__ RayZ ray_z(const ColParams& c, float v, float cz) {
    RayZ r;
    r.fz_mid = __fmaf_rn(v, c.c1, cz);
    r.bz = __fmul_rn(v, c.inv_dmaj);
    r.step = __fmul_rn(__fsqrt_rn(__fmaf_rn(v, v, c.dxy2)), c.vox_over_adm);
    return r;
}

__device__ __forceinline__ float det_v(int iv, const ProjDims& d) {
    return __fmul_rn(__fsub_rn((float)iv, d.cv), d.dv);
}

__device__ __forceinline__ ColParams load_col(const float4* __restrict__ col, size_t idx) {
    float4 a = __ldg(col + 2 * idx), b = __ldg(col + 2 * idx + 1);
    ColParams c;
    c.fa_mid = a.x; c.ba = a.y; c.c1 = a.z; c.inv_dmaj = a.w;
    c.dxy2 = b.x; c.vox_over_adm = b.y; c.xmajor = b.z; c.pad = b.w;
    return c;
}

// ------------------------------------------------------------------ FP64 table

// One thread per (frame-view g, column iu).  Writes the column constants and
// flags geometry the model does not cover: a plane crossing outside the
// source-detector segment (0 < lambda < 1) on the first or last plane.
__global__ void column_table_kernel(const double* __restrict__ angles, float4* __restrict__ col,
                                    int* __restrict__ vflag, int* __restrict__ bad, ProjDims d,
                                    double vox, double du, double dso, double dsd) {
    const int iu = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (iu >= d.nu) return;
    const double th = angles[g];
    const double c = cos(th), s = sin(th);
    const double u = (iu - 0.5 * (d.nu - 1)) * du;
    const double sx = dso * c, sy = dso * s;
    const double px = -(dsd - dso) * c - u * s;
    const double py = -(dsd - dso) * s + u * c;
    const double dx = px - sx, dy = py - sy;
    const bool xmaj = fabs(dx) >= fabs(dy);
    const double dmaj = xmaj ? dx : dy, smaj = xmaj ? sx : sy;
    const double da = xmaj ? dy : dx, sa = xmaj ? sy : sx;
    const int nmaj = xmaj ? d.nx : d.ny, na = xmaj ? d.ny : d.nx;
    const double lam0 = -smaj / dmaj;
    float4 a, b;
    a.x = (float)((sa + lam0 * da) / vox + 0.5 * (na - 1));
    a.y = (float)(da / dmaj);
    a.z = (float)(lam0 / vox);
    a.w = (float)(1.0 / dmaj);
    b.x = (float)(dx * dx + dy * dy);
    b.y = (float)(vox / fabs(dmaj));
    b.z = xmaj ? 1.0f : 0.0f;
    b.w = 0.0f;
    const size_t idx = (size_t)g * d.nu + iu;
    col[2 * idx] = a;
    col[2 * idx + 1] = b;
    atomicOr(vflag + g, xmaj ? 1 : 2);   // which major axes occur in this view
    const double lfirst = lam0 + (0 - 0.5 * (nmaj - 1)) * vox / dmaj;
    const double llast = lam0 + (nmaj - 1 - 0.5 * (nmaj - 1)) * vox / dmaj;
    if (!(fmin(lfirst, llast) > 0.0 && fmax(lfirst, llast) < 1.0)) atomicExch(bad, 1);
    (void)na;
}

// ------------------------------------------------------------------ z-paired copies

// Per frame and z-slice, the two copies of a volume v that the forward reads:
// py[z][y][x] = (v(z, y, x), v(z + 1, y, x)) and px[z][x][y], the same pairs
// transposed (x-major rays read y-contiguous data), with v(nz, ., .) = 0, so
// that a ray's four bilinear taps are two 8-byte loads.
// FUSED: v = r + beta_t p (the CG direction update) with p = in; v is also
// written to pnext (a different buffer: neighbouring slices still read p).
template <bool FUSED>
__global__ void pair_kernel(const float* __restrict__ in, float2* __restrict__ px, float2* __restrict__ py,
                            const float* __restrict__ r, float* __restrict__ pnext, const double* __restrict__ beta,
                            int nx, int ny, int nz) {
    __shared__ float2 tile[32][33];
    const int slice = blockIdx.z;             // t * nz + z
    const int t = slice / nz, z = slice % nz;
    const size_t plane = (size_t)nx * ny;
    const size_t base = (size_t)slice * plane;
    const bool up = z + 1 < nz;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    float bt = 0.0f;
    if (FUSED) bt = (float)beta[t];
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int x = x0 + threadIdx.x, y = y0 + k;
        if (x < nx && y < ny) {
            const size_t i = base + (size_t)y * nx + x;
            float lo, hi = 0.0f;
            if (FUSED) {
                lo = __fmaf_rn(bt, in[i], r[i]);
                if (up) hi = __fmaf_rn(bt, in[i + plane], r[i + plane]);
                pnext[i] = lo;
            } else {
                lo = in[i];
                if (up) hi = in[i + plane];
            }
            const float2 v = make_float2(lo, hi);
            py[i] = v;
            tile[k][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int y = y0 + threadIdx.x, x = x0 + k;
        if (x < nx && y < ny) px[base + (size_t)x * ny + y] = tile[threadIdx.x][k];
    }
}

// ------------------------------------------------------------------ forward

enum FwdMode { FWD_PLAIN = 0, FWD_LAMBDA = 1, FWD_RESIDUAL = 2 };

// Rays per thread of the forward: consecutive detector rows of one column,
// which share the column's in-plane crossing (f_a, its floor and weight).
constexpr int FWD_R = 2;

// Narrows [kmin, kmax] to the planes k where f(k) = f0 + (k - cmaj) b lies in
// [lo, hi], one plane inside the exact bounds on each side (so that FP32
// rounding of f never leaves [lo, hi] inside the range).
__device__ __forceinline__ void planes_within(float f0, float b, float lo, float hi, float cmaj, float& kmin,
                                              float& kmax) {
    if (fabsf(b) > 1e-12f) {
        const float k1 = (lo - f0) / b + cmaj, k2 = (hi - f0) / b + cmaj;
        kmin = fmaxf(kmin, ceilf(fminf(k1, k2)) + 1.0f);
        kmax = fminf(kmax, floorf(fmaxf(k1, k2)) - 1.0f);
    } else if (!(f0 >= lo && f0 <= hi)) {
        kmax = kmin - 1.0f;
    }
}

// One thread per FWD_R rays (detector rows FWD_R*i .. FWD_R*i + FWD_R - 1 of one
// column); a block covers blockDim.x columns x FWD_R*blockDim.y rows of one view
// (128 threads; the shape is chosen per plan by msf_projector_autotune).  x-major
// rays read the z-paired transposed frame px [nz][nx][ny], y-major rays the
// z-paired natural frame py [nz][ny][nx] (pair_kernel), so the minor in-plane
// axis is contiguous and each (a, z) tap pair is one 8-byte load.  Planes
// where every bilinear tap of every ray of the thread lies inside the grid run
// without bounds checks; the planes at either end check each tap.  The
// interpolation is v00 + w_a (v01 - v00) along a, then the same along z.
//   FWD_PLAIN:    out = A x
//   FWD_LAMBDA:   out = step * Lambda * (A x)
//   FWD_RESIDUAL: out = step * Lambda * (meas - A x)
// (the CG modes write the step-weighted sinogram e' = step * e that the gather
// adjoint consumes)
// PAR (the ICD agent's projection of a group step): x is zero outside one
// voxel parity group, so an x-major ray only visits planes x = kpx (mod 2) and
// a y-major ray planes y = kpy (mod 2), and on a visited plane it loads only
// the z-pair of the minor-axis tap with the group's parity (the other is zero);
// the skipped terms are exact zeros, so the result equals the full projection
// bit for bit.
template <int MODE, bool PAR = false>
__global__ void __launch_bounds__(128) joseph_fwd_kernel(
    const float2* __restrict__ px, const float2* __restrict__ py, const float4* __restrict__ col,
    float* __restrict__ out, const float* __restrict__ lam, const float* __restrict__ meas,
    ProjDims d, int kpx = 0, int kpy = 0) {
    const int iu = blockIdx.x * blockDim.x + threadIdx.x;
    const int iv0 = (blockIdx.y * blockDim.y + threadIdx.y) * FWD_R;
    const int g = blockIdx.z;
    if (iu >= d.nu || iv0 >= d.nv) return;
    const int t = g / d.views;
    const ColParams c = load_col(col, (size_t)g * d.nu + iu);
    const bool xmaj = c.xmajor != 0.0f;
    const int nmaj = xmaj ? d.nx : d.ny, na = xmaj ? d.ny : d.nx;
    const size_t fs = (size_t)d.nx * d.ny * d.nz;
    const float2* __restrict__ vol = (xmaj ? px : py) + (size_t)t * fs;   // (v(z), v(z+1)) pairs
    const float cmaj = xmaj ? d.cx : d.cy;
    const int zs = nmaj * na;    // z stride of the frame

    RayZ rz[FWD_R];
#pragma unroll
    for (int r = 0; r < FWD_R; ++r) rz[r] = ray_z(c, det_v(min(iv0 + r, d.nv - 1), d), d.cz);

    // planes where some crossing can touch the grid (-1 < f < n on both minor
    // axes, one plane of margin), and the inner planes where all four taps of
    // every ray are inside (0.5 <= f <= n - 1.5)
    float klo = (float)(nmaj - 1), khi = 0.0f;
    float kin_lo = 0.0f, kin_hi = (float)(nmaj - 1);
    planes_within(c.fa_mid, c.ba, 0.5f, (float)na - 1.5f, cmaj, kin_lo, kin_hi);
#pragma unroll
    for (int r = 0; r < FWD_R; ++r) {
        float lo = 0.0f, hi = (float)(nmaj - 1);
        const float fm[2] = {c.fa_mid, rz[r].fz_mid}, bb[2] = {c.ba, rz[r].bz};
        const float top[2] = {(float)na, (float)d.nz};
        for (int a = 0; a < 2; ++a) {
            if (fabsf(bb[a]) > 1e-12f) {
                const float k1 = (-1.0f - fm[a]) / bb[a] + cmaj, k2 = (top[a] - fm[a]) / bb[a] + cmaj;
                lo = fmaxf(lo, floorf(fminf(k1, k2)) - 1.0f);
                hi = fminf(hi, ceilf(fmaxf(k1, k2)) + 1.0f);
            } else if (!(fm[a] > -1.0f && fm[a] < top[a])) {
                hi = -1.0f;
            }
        }
        if (lo <= hi) {
            klo = fminf(klo, lo);
            khi = fmaxf(khi, hi);
        }
        planes_within(rz[r].fz_mid, rz[r].bz, 0.5f, (float)d.nz - 1.5f, cmaj, kin_lo, kin_hi);
    }
    float acc[FWD_R];
#pragma unroll
    for (int r = 0; r < FWD_R; ++r) acc[r] = 0.0f;
    if (klo <= khi) {
        const int K0 = (int)klo, K1 = (int)khi;
        int F0 = (int)fmaxf(kin_lo, klo), F1 = (int)fminf(kin_hi, khi);
        if (F0 > F1) F0 = K1 + 1, F1 = K1;

        // one plane with every tap checked against the grid
        auto checked = [&](int k) {
            const float tk = __fsub_rn((float)k, cmaj);
            const float fa = __fmaf_rn(tk, c.ba, c.fa_mid);
            const float a0f = floorf(fa);
            const float wa1 = __fsub_rn(fa, a0f);
            const int ia = (int)a0f;
            const bool a_in0 = ia >= 0 && ia < na, a_in1 = ia + 1 >= 0 && ia + 1 < na;
#pragma unroll
            for (int r = 0; r < FWD_R; ++r) {
                const float fz = __fmaf_rn(tk, rz[r].bz, rz[r].fz_mid);
                const float z0f = floorf(fz);
                const float wz1 = __fsub_rn(fz, z0f);
                const int iz = (int)z0f;
                // the pair of slice iz holds taps iz and iz + 1 (0 above the
                // grid); below it (iz = -1) only the upper tap, from slice 0
                float v00 = 0.0f, v01 = 0.0f, v10 = 0.0f, v11 = 0.0f;
                if (iz >= 0 && iz < d.nz) {
                    const float2* row = vol + ((ptrdiff_t)iz * nmaj + k) * na;
                    if (a_in0) { const float2 q = __ldg(row + ia); v00 = q.x; v10 = q.y; }
                    if (a_in1) { const float2 q = __ldg(row + ia + 1); v01 = q.x; v11 = q.y; }
                } else if (iz == -1) {
                    const float2* row = vol + (ptrdiff_t)k * na;
                    if (a_in0) v10 = __ldg(row + ia).x;
                    if (a_in1) v11 = __ldg(row + ia + 1).x;
                }
                const float top = __fmaf_rn(wa1, __fsub_rn(v01, v00), v00);
                const float bot = __fmaf_rn(wa1, __fsub_rn(v11, v10), v10);
                acc[r] = __fadd_rn(acc[r], __fmaf_rn(wz1, __fsub_rn(bot, top), top));
            }
        };
        const int kp = xmaj ? kpx : kpy, ka = xmaj ? kpy : kpx;
        for (int k = K0; k < F0; ++k)
            if (!PAR || (k & 1) == kp) checked(k);
        for (int k = PAR ? F0 + ((F0 ^ kp) & 1) : F0; k <= F1; k += PAR ? 2 : 1) {
            const float tk = __fsub_rn((float)k, cmaj);
            const float fa = __fmaf_rn(tk, c.ba, c.fa_mid);
            const float a0f = floorf(fa);
            const float wa1 = __fsub_rn(fa, a0f);
            const float2* pk = vol + k * na + (int)a0f;
            const bool lo = (((int)a0f) & 1) == ka;   // PAR: the tap at a0 has the group's parity
#pragma unroll
            for (int r = 0; r < FWD_R; ++r) {
                const float fz = __fmaf_rn(tk, rz[r].bz, rz[r].fz_mid);
                const float z0f = floorf(fz);
                const float wz1 = __fsub_rn(fz, z0f);
                const float2* p0 = pk + (ptrdiff_t)((int)z0f) * zs;
                const float2 zero = make_float2(0.0f, 0.0f);
                const float2 q0 = (!PAR || lo) ? __ldg(p0) : zero;
                const float2 q1 = (!PAR || !lo) ? __ldg(p0 + 1) : zero;
                const float v00 = q0.x, v10 = q0.y, v01 = q1.x, v11 = q1.y;
                const float top = __fmaf_rn(wa1, __fsub_rn(v01, v00), v00);
                const float bot = __fmaf_rn(wa1, __fsub_rn(v11, v10), v10);
                acc[r] = __fadd_rn(acc[r], __fmaf_rn(wz1, __fsub_rn(bot, top), top));
            }
        }
        for (int k = F1 + 1; k <= K1; ++k)
            if (!PAR || (k & 1) == kp) checked(k);
    }
#pragma unroll
    for (int r = 0; r < FWD_R; ++r) {
        const int iv = iv0 + r;
        if (iv >= d.nv) break;
        const float val = acc[r] * rz[r].step;
        const size_t ray = ((size_t)g * d.nv + iv) * d.nu + iu;
        if (MODE == FWD_PLAIN) out[ray] = val;
        else if (MODE == FWD_LAMBDA) out[ray] = rz[r].step * (lam[ray] * val);
        else out[ray] = rz[r].step * (lam[ray] * (meas[ray] - val));
    }
}

// ------------------------------------------------------------------ adjoint (gather)

enum AdjMode { ADJ_PLAIN = 0, ADJ_CG_INIT = 1, ADJ_CG_Q = 2 };

// Voxels of one z-run handled by one thread of the gather: 8, 16, 32 or 64,
// chosen per plan (default 16).

// Detector u coordinate (in pixels) of the point (x, y, .) for view (cs, sn);
// only used to bound candidate columns, so a fast division is enough.
__device__ __forceinline__ float u_pixel(float x, float y, float cs, float sn, const ProjDims& d) {
    const float lat = -x * sn + y * cs;
    const float depth = d.dso - x * cs - y * sn;
    return __fdividef(d.dsd * lat, depth) / d.du + d.cu;
}

// Adds, for the rays of one view whose major axis is XMAJ, w(ray, voxel) *
// e'(ray) to the ZB accumulators of the voxel run (ix, iy, iz_lo ..
// iz_lo+ZB-1), where e' = step * e is the step-weighted sinogram.
//
// An x-major ray touches column (ix, iy) on plane k = ix when floor(f_y) is
// iy-1 or iy.  Candidate detector columns come from the exact projection of
// the segment {x = x_ix, |y - y_iy| <= voxel} (plus one column of margin); on
// a column that qualifies, the rows whose f_z(k) can fall within one voxel of
// the run follow from f_z(v) = c_z + v (c1 + tk inv_dmaj).  Each ray's f_a is
// recomputed with the forward's own operations (bit for bit); f_z of row 0
// likewise, and of a row iv by one FMA from it (a few 1e-5 voxel from the
// forward's value, so the taps agree except within that distance of a voxel
// boundary, where the weights are continuous; the value depends on the ray
// alone, not on the run length the plan's autotuner picks).
// Every ray-plane crossing of the forward is visited by the two runs that hold
// its a-taps, so the work tracks the forward's.
template <bool XMAJ, int ZB>
__device__ __forceinline__ void gather_runs(const float4* __restrict__ col, const float* __restrict__ e,
                                            int g, int ix, int iy, int iz_lo, float cs, float sn,
                                            const ProjDims& d, float (*acc)[128], int tid) {
    const int kpl = XMAJ ? ix : iy;             // plane index along the major axis
    const int ia = XMAJ ? iy : ix;              // voxel index on the minor axis
    const float cmaj = XMAJ ? d.cx : d.cy;
    const float xc = (ix - d.cx) * d.vox, yc = (iy - d.cy) * d.vox;
    float u1, u2;
    if (XMAJ) {
        u1 = u_pixel(xc, yc - d.vox, cs, sn, d);
        u2 = u_pixel(xc, yc + d.vox, cs, sn, d);
    } else {
        u1 = u_pixel(xc - d.vox, yc, cs, sn, d);
        u2 = u_pixel(xc + d.vox, yc, cs, sn, d);
    }
    const int iu_lo = max(0, (int)floorf(fminf(u1, u2)) - 1);
    const int iu_hi = min(d.nu - 1, (int)ceilf(fmaxf(u1, u2)) + 1);
    const float tk = __fsub_rn((float)kpl, cmaj);
    const float inv_dv = 1.0f / d.dv;
    for (int iu = iu_lo; iu <= iu_hi; ++iu) {
        const ColParams c = load_col(col, (size_t)g * d.nu + iu);
        if ((c.xmajor != 0.0f) != XMAJ) continue;
        const float fa = __fmaf_rn(tk, c.ba, c.fa_mid);
        const float a0f = floorf(fa);
        const int a0 = (int)a0f;
        if (ia != a0 && ia != a0 + 1) continue;
        const float wa1 = __fsub_rn(fa, a0f);
        const float wa = (ia == a0) ? __fsub_rn(1.0f, wa1) : wa1;
        // rows with f_z in (iz_lo - 1, iz_lo + ZB); gz > 0 (planes lie
        // between source and detector)
        const float rgz = __fdividef(1.0f, c.c1 + tk * c.inv_dmaj);
        const float va = (iz_lo - 1 - d.cz) * rgz * inv_dv + d.cv;
        const float vb = (iz_lo + ZB - d.cz) * rgz * inv_dv + d.cv;
        const int iv_lo = max(0, (int)floorf(va) - 1);
        const int iv_hi = min(d.nv - 1, (int)ceilf(vb) + 1);
        const float* erow = e + ((size_t)g * d.nv) * d.nu + iu;
        // f_z is affine in the row: f_z(iv) = f_z(0) + iv dfz, with f_z(0) the
        // forward's crossing of detector row 0 (so a ray's value does not
        // depend on the run that evaluates it; within a few 1e-5 voxel of the
        // forward's own FP32 value)
        const RayZ rzb = ray_z(c, det_v(0, d), d.cz);
        const float fzb = __fmaf_rn(tk, rzb.bz, rzb.fz_mid);
        const float dfz = d.dv * __fmaf_rn(tk, c.inv_dmaj, c.c1);   // > 0
        // rows in [iva, ivb) have both z taps inside the run (f_z in
        // [iz_lo + 0.01, iz_lo + ZB - 1.01]); the others are checked
        const float rdfz = __fdividef(1.0f, dfz);
        const int iva = min(max((int)ceilf(((float)iz_lo + 0.01f - fzb) * rdfz), iv_lo), iv_hi + 1);
        const int ivb = min(max((int)floorf(((float)(iz_lo + ZB) - 1.01f - fzb) * rdfz) + 1, iva), iv_hi + 1);
        // explicit roundings: both loops must form a row's terms identically
        auto checked = [&](int iv) {
            const float fz = __fmaf_rn((float)iv, dfz, fzb);
            const float z0f = floorf(fz);
            const int k0 = (int)z0f - iz_lo;
            if (k0 < -1 || k0 >= ZB) return;
            const float ev = __fmul_rn(wa, __ldg(erow + (size_t)iv * d.nu));
            const float c1 = __fmul_rn(__fsub_rn(fz, z0f), ev);
            if (k0 >= 0) acc[k0][tid] = __fadd_rn(acc[k0][tid], __fsub_rn(ev, c1));
            if (k0 + 1 < ZB) acc[k0 + 1][tid] = __fadd_rn(acc[k0 + 1][tid], c1);
        };
        for (int iv = iv_lo; iv < iva; ++iv) checked(iv);
        for (int iv = iva; iv < ivb; ++iv) {
            const float fz = __fmaf_rn((float)iv, dfz, fzb);
            const float z0f = floorf(fz);
            const int k0 = min(max((int)z0f - iz_lo, 0), ZB - 2);   // in range by the choice of [iva, ivb)
            const float ev = __fmul_rn(wa, __ldg(erow + (size_t)iv * d.nu));
            const float c1 = __fmul_rn(__fsub_rn(fz, z0f), ev);
            acc[k0][tid] = __fadd_rn(acc[k0][tid], __fsub_rn(ev, c1));
            acc[k0 + 1][tid] = __fadd_rn(acc[k0 + 1][tid], c1);
        }
        for (int iv = ivb; iv <= iv_hi; ++iv) checked(iv);
    }
}

// One thread per run of ZB voxels along z; block 32 (x) x 4 (y).
// e is the step-weighted sinogram e' = step * e.
//   ADJ_PLAIN:   out = A^T e
//   ADJ_CG_INIT: r = A^T e + (v - z)/sigma^2, p = r, partial sum r.r
//   ADJ_CG_Q:    q = A^T e + p/sigma^2, partial sum p.q
// (at most 64 registers: eight blocks per SM, no spills)
template <int MODE, int ZB>
__global__ void __launch_bounds__(128, 8) joseph_adj_kernel(
    const float4* __restrict__ col, const float2* __restrict__ trig, const int* __restrict__ vflag,
    const float* __restrict__ e, float* __restrict__ out, const float* __restrict__ a1,
    const float* __restrict__ a2, float* __restrict__ out2, double* __restrict__ partial,
    float inv_s2, ProjDims d) {
    __shared__ float acc[ZB][128];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int ix = blockIdx.x * 32 + threadIdx.x;
    const int iy = blockIdx.y * 4 + threadIdx.y;
    const int nzb = (d.nz + ZB - 1) / ZB;
    const int zb = blockIdx.z % nzb;
    const int t = blockIdx.z / nzb;
    const int iz_lo = zb * ZB;
    const bool inside = ix < d.nx && iy < d.ny;
#pragma unroll
    for (int k = 0; k < ZB; ++k) acc[k][tid] = 0.0f;
    if (inside) {
        for (int j = 0; j < d.views; ++j) {
            const int g = t * d.views + j;
            const float2 cs = __ldg(trig + g);
            const int fl = __ldg(vflag + g);
            if (fl & 1) gather_runs<true, ZB>(col, e, g, ix, iy, iz_lo, cs.x, cs.y, d, acc, tid);
            if (fl & 2) gather_runs<false, ZB>(col, e, g, ix, iy, iz_lo, cs.x, cs.y, d, acc, tid);
        }
    }
    double dot = 0.0;
    for (int k = 0; k < ZB; ++k) {
        const int iz = iz_lo + k;
        if (!inside || iz >= d.nz) break;
        const size_t i = (((size_t)t * d.nz + iz) * d.ny + iy) * d.nx + ix;
        const float s = acc[k][tid];
        if (MODE == ADJ_PLAIN) {
            out[i] = s;
        } else if (MODE == ADJ_CG_INIT) {   // a1 = v, a2 = z
            const float r = s + (a1[i] - a2[i]) * inv_s2;
            out[i] = r;
            out2[i] = r;
            dot += (double)r * (double)r;
        } else {                            // a1 = p
            const float p = a1[i];
            const float q = s + p * inv_s2;
            out[i] = q;
            dot += (double)p * (double)q;
        }
    }
    if (MODE != ADJ_PLAIN) {
        const double sum = block_sum_f64(dot);
        if (tid == 0) {
            const int bpf = gridDim.x * gridDim.y * nzb;   // blocks per frame
            const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zb);
            partial[(size_t)t * bpf + b] = sum;
        }
    }
}

// e' = step * e for every ray (input of the gather for a plain A^T).
__global__ void step_weight_kernel(const float4* __restrict__ col, const float* __restrict__ e,
                                   float* __restrict__ out, ProjDims d) {
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int iv = blockIdx.y * 4 + threadIdx.y;
    const int g = blockIdx.z;
    if (iu >= d.nu || iv >= d.nv) return;
    const ColParams c = load_col(col, (size_t)g * d.nu + iu);
    const RayZ rz = ray_z(c, det_v(iv, d), d.cz);
    const size_t ray = ((size_t)g * d.nv + iv) * d.nu + iu;
    out[ray] = rz.step * e[ray];
}

// ------------------------------------------------------------------ CG scalars

enum FinMode { FIN_RR0 = 0, FIN_ALPHA = 1, FIN_BETA = 2 };

// One block per frame: sums that frame's block partials in a fixed order.
//   FIN_RR0:   rr = sum
//   FIN_ALPHA: alpha = rr / sum (0 when sum == 0)
//   FIN_BETA:  beta = sum / rr (0 when rr == 0); rr = sum
// Any non-finite sum raises the status flag.
template <int MODE>
__global__ void cg_finalize_kernel(const double* __restrict__ partial, int nparts,
                                   double* __restrict__ rr, double* __restrict__ coef,
                                   int* __restrict__ status) {
    const int t = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[(size_t)t * nparts + i];
    s = block_sum_f64(s);
    if (threadIdx.x == 0) {
        if (!isfinite(s)) atomicExch(status, (int)MSF_ERR_NUMERIC);
        if (MODE == FIN_RR0) {
            rr[t] = s;
        } else if (MODE == FIN_ALPHA) {
            coef[t] = (s != 0.0) ? rr[t] / s : 0.0;
        } else {
            coef[t] = (rr[t] != 0.0) ? s / rr[t] : 0.0;
            rr[t] = s;
        }
    }
}

// z += alpha p; r -= alpha q; partial r.r  (grid: blocks_per_frame x nt).
// Each thread adds the squares of runs of 8 of its elements in FP32 before its
// FP64 sum (FP64 arithmetic is a small fraction of the FP32 rate on this GPU);
// the order of every addition is fixed.
__global__ void cg_update_kernel(float* __restrict__ z, float* __restrict__ r,
                                 const float* __restrict__ p, const float* __restrict__ q,
                                 const double* __restrict__ alpha, double* __restrict__ partial,
                                 size_t fs) {
    const int t = blockIdx.y;
    const float a = (float)alpha[t];
    const size_t off = (size_t)t * fs;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    double dot = 0.0;
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    while (i < fs) {
        float run = 0.0f;
        for (int k = 0; k < 8 && i < fs; ++k, i += stride) {
            z[off + i] = __fmaf_rn(a, p[off + i], z[off + i]);
            const float rn = __fmaf_rn(-a, q[off + i], r[off + i]);
            r[off + i] = rn;
            run = __fmaf_rn(rn, rn, run);
        }
        dot += (double)run;
    }
    const double s = block_sum_f64(dot);
    if (threadIdx.x == 0) partial[(size_t)t * gridDim.x + blockIdx.x] = s;
}

// ------------------------------------------------------------------ grouped ICD data agent
//
// The partial update L~ of Sec. III as coordinate descent on the cost of
// Eq. (4).  A sweep visits the eight parity groups (pz*2 + py)*2 + px of the
// voxels in increasing order; inside a group every voxel takes its own Newton
// step against the same step-weighted residual sinogram e' = step*Lambda*(y - Az),
//     delta_s = -theta1_s / theta2_s,
//     theta1_s = -(A^T Lambda e)_s + (z_s - v_s)/sigma^2,
//     theta2_s = sum_r Lambda_r a_rs^2 + 1/sigma^2,
// and the group moves by alpha_t delta (per frame t), alpha_t the exact
// minimiser of the quadratic cost along delta.  A parity group holds at most
// one of the four bilinear taps of any ray-plane crossing.

constexpr int ICD_SINO_BLOCKS = 256;   // blocks per frame of the sinogram passes
constexpr int ICD_ZB = 8;              // group voxels per z-run of the group gather (16 slices)

// Adds, for the rays of one view whose major axis is XMAJ, the gather terms of
// the voxels (ix, iy, base + ZS*j), j < ZB, into acc[j]: w_a w_z e' (SQ false)
// or w_a^2 w_z^2 e' (SQ true, with e' = step^2 Lambda: the diagonal of
// A^T Lambda A).  Candidate columns, the a weight and the affine z crossing per
// row are formed exactly as in gather_runs.
template <bool XMAJ, int ZB, int ZS, bool SQ>
__device__ __forceinline__ void gather_icd(const float4* __restrict__ col, const float* __restrict__ e, int g,
                                           int ix, int iy, int base, float cs, float sn, const ProjDims& d,
                                           float (*acc)[128], int tid) {
    const int kpl = XMAJ ? ix : iy;
    const int ia = XMAJ ? iy : ix;
    const float cmaj = XMAJ ? d.cx : d.cy;
    const float xc = (ix - d.cx) * d.vox, yc = (iy - d.cy) * d.vox;
    float u1, u2;
    if (XMAJ) {
        u1 = u_pixel(xc, yc - d.vox, cs, sn, d);
        u2 = u_pixel(xc, yc + d.vox, cs, sn, d);
    } else {
        u1 = u_pixel(xc - d.vox, yc, cs, sn, d);
        u2 = u_pixel(xc + d.vox, yc, cs, sn, d);
    }
    const int iu_lo = max(0, (int)floorf(fminf(u1, u2)) - 1);
    const int iu_hi = min(d.nu - 1, (int)ceilf(fmaxf(u1, u2)) + 1);
    const float tk = __fsub_rn((float)kpl, cmaj);
    const float inv_dv = 1.0f / d.dv;
    const int zlast = base + ZS * (ZB - 1);
    for (int iu = iu_lo; iu <= iu_hi; ++iu) {
        const ColParams c = load_col(col, (size_t)g * d.nu + iu);
        if ((c.xmajor != 0.0f) != XMAJ) continue;
        const float fa = __fmaf_rn(tk, c.ba, c.fa_mid);
        const float a0f = floorf(fa);
        const int a0 = (int)a0f;
        if (ia != a0 && ia != a0 + 1) continue;
        const float wa1 = __fsub_rn(fa, a0f);
        const float wa = (ia == a0) ? __fsub_rn(1.0f, wa1) : wa1;
        const float wav = SQ ? __fmul_rn(wa, wa) : wa;
        const float rgz = __fdividef(1.0f, c.c1 + tk * c.inv_dmaj);
        const float va = (base - 1 - d.cz) * rgz * inv_dv + d.cv;
        const float vb = (zlast + 1 - d.cz) * rgz * inv_dv + d.cv;
        const int iv_lo = max(0, (int)floorf(va) - 1);
        const int iv_hi = min(d.nv - 1, (int)ceilf(vb) + 1);
        const float* erow = e + ((size_t)g * d.nv) * d.nu + iu;
        const RayZ rzb = ray_z(c, det_v(0, d), d.cz);
        const float fzb = __fmaf_rn(tk, rzb.bz, rzb.fz_mid);
        const float dfz = d.dv * __fmaf_rn(tk, c.inv_dmaj, c.c1);
        for (int iv = iv_lo; iv <= iv_hi; ++iv) {
            const float fz = __fmaf_rn((float)iv, dfz, fzb);
            const float z0f = floorf(fz);
            const int z0 = (int)z0f;
            if (z0 + 1 < base || z0 > zlast) continue;
            const float ev = __fmul_rn(wav, __ldg(erow + (size_t)iv * d.nu));
            const float wz1 = __fsub_rn(fz, z0f);
            const float w1 = SQ ? __fmul_rn(wz1, wz1) : wz1;
            const float w0 = SQ ? __fmul_rn(__fsub_rn(1.0f, wz1), __fsub_rn(1.0f, wz1)) : 0.0f;
            const float c1 = __fmul_rn(w1, ev);
            const float c0 = SQ ? __fmul_rn(w0, ev) : __fsub_rn(ev, c1);
            const int o0 = z0 - base, o1 = z0 + 1 - base;
            if (o0 >= 0 && o0 % ZS == 0 && o0 / ZS < ZB) acc[o0 / ZS][tid] = __fadd_rn(acc[o0 / ZS][tid], c0);
            if (o1 >= 0 && o1 % ZS == 0 && o1 / ZS < ZB) acc[o1 / ZS][tid] = __fadd_rn(acc[o1 / ZS][tid], c1);
        }
    }
}

// theta2 = (A^T Lambda A)_ss + 1/sigma^2 for every voxel: the squared-weight
// gather of e2 = step^2 Lambda.  Grid and runs as joseph_adj_kernel.
template <int ZB>
__global__ void __launch_bounds__(128) icd_theta2_kernel(const float4* __restrict__ col,
                                                         const float2* __restrict__ trig,
                                                         const int* __restrict__ vflag,
                                                         const float* __restrict__ e2, float* __restrict__ theta2,
                                                         float inv_s2, ProjDims d) {
    __shared__ float acc[ZB][128];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int ix = blockIdx.x * 32 + threadIdx.x;
    const int iy = blockIdx.y * 4 + threadIdx.y;
    const int nzb = (d.nz + ZB - 1) / ZB;
    const int zb = blockIdx.z % nzb, t = blockIdx.z / nzb;
    const int base = zb * ZB;
    const bool inside = ix < d.nx && iy < d.ny;
#pragma unroll
    for (int k = 0; k < ZB; ++k) acc[k][tid] = 0.0f;
    if (inside) {
        for (int j = 0; j < d.views; ++j) {
            const int g = t * d.views + j;
            const float2 cs = __ldg(trig + g);
            const int fl = __ldg(vflag + g);
            if (fl & 1) gather_icd<true, ZB, 1, true>(col, e2, g, ix, iy, base, cs.x, cs.y, d, acc, tid);
            if (fl & 2) gather_icd<false, ZB, 1, true>(col, e2, g, ix, iy, base, cs.x, cs.y, d, acc, tid);
        }
        for (int k = 0; k < ZB && base + k < d.nz; ++k)
            theta2[(((size_t)t * d.nz + base + k) * d.ny + iy) * d.nx + ix] = acc[k][tid] + inv_s2;
    }
}

// Group dimensions: voxels of parity p along an axis of n voxels.
__host__ __device__ __forceinline__ int par_count(int n, int p) { return (n - p + 1) / 2; }

struct IcdGroup {
    int px, py, pz;
    int gx, gy, gz;   // group voxels along x, y, z
    int nzb;          // z-runs of ZB group voxels per column
};

// The group step's gather: for every voxel s of the group, delta_s =
// -theta1_s/theta2_s (written to dlt), and per-block partial sums of
// theta1.delta and delta.delta (FP64, fixed order).  A thread owns one group
// column (ix, iy) and a run of ZB group voxels along z (stride 2).
template <int ZB>
__global__ void __launch_bounds__(128) icd_group_kernel(const float4* __restrict__ col,
                                                        const float2* __restrict__ trig,
                                                        const int* __restrict__ vflag, const float* __restrict__ e,
                                                        const float* __restrict__ z, const float* __restrict__ v,
                                                        const float* __restrict__ theta2, float* __restrict__ dlt,
                                                        double* __restrict__ partial, float inv_s2, IcdGroup G,
                                                        ProjDims d) {
    __shared__ float acc[ZB][128];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int jx = blockIdx.x * 32 + threadIdx.x, jy = blockIdx.y * 4 + threadIdx.y;
    const int ix = 2 * jx + G.px, iy = 2 * jy + G.py;
    const int zb = blockIdx.z % G.nzb, t = blockIdx.z / G.nzb;
    const int base = G.pz + 2 * ZB * zb;
    const bool inside = jx < G.gx && jy < G.gy;
#pragma unroll
    for (int k = 0; k < ZB; ++k) acc[k][tid] = 0.0f;
    if (inside) {
        for (int j = 0; j < d.views; ++j) {
            const int g = t * d.views + j;
            const float2 cs = __ldg(trig + g);
            const int fl = __ldg(vflag + g);
            if (fl & 1) gather_icd<true, ZB, 2, false>(col, e, g, ix, iy, base, cs.x, cs.y, d, acc, tid);
            if (fl & 2) gather_icd<false, ZB, 2, false>(col, e, g, ix, iy, base, cs.x, cs.y, d, acc, tid);
        }
    }
    double gd = 0.0, dd = 0.0;
    for (int k = 0; k < ZB; ++k) {
        const int iz = base + 2 * k;
        if (!inside || iz >= d.nz) break;
        const size_t i = (((size_t)t * d.nz + iz) * d.ny + iy) * d.nx + ix;
        const float th1 = __fmaf_rn(__fsub_rn(z[i], v[i]), inv_s2, -acc[k][tid]);
        const float del = -__fdiv_rn(th1, theta2[i]);
        dlt[i] = del;
        gd += (double)th1 * (double)del;
        dd += (double)del * (double)del;
    }
    const double sg = block_sum_f64(gd);
    const double sd = block_sum_f64(dd);
    if (tid == 0) {
        const int bpf = gridDim.x * gridDim.y * G.nzb;
        const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zb);
        partial[2 * ((size_t)t * bpf + b)] = sg;
        partial[2 * ((size_t)t * bpf + b) + 1] = sd;
    }
}

// Sinogram passes of a group step, per frame (grid ICD_SINO_BLOCKS x nt):
//   PASS 0: per-block partial sums of Lambda (A delta)^2
//   PASS 1: e' -= alpha_t step Lambda (A delta)
// ad = A delta (plain forward), lam = Lambda, e' the step-weighted residual.
template <int PASS>
__global__ void __launch_bounds__(256) icd_sino_kernel(const float4* __restrict__ col,
                                                       const float* __restrict__ ad, const float* __restrict__ lam,
                                                       float* __restrict__ e, const double* __restrict__ alpha,
                                                       double* __restrict__ partial, ProjDims d) {
    const int t = blockIdx.y;
    const size_t per_view = (size_t)d.nu * d.nv, mt = per_view * d.views;
    const size_t off = (size_t)t * mt;
    const float a = PASS == 1 ? (float)alpha[t] : 0.0f;
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < mt; i += (size_t)gridDim.x * blockDim.x) {
        const float val = ad[off + i];
        const float l = lam[off + i];
        if (PASS == 0) {
            s += (double)l * (double)val * (double)val;
        } else {
            const int j = (int)(i / per_view);
            const int iv = (int)((i % per_view) / d.nu), iu = (int)(i % d.nu);
            const ColParams c = load_col(col, ((size_t)t * d.views + j) * d.nu + iu);
            const float step = ray_z(c, det_v(iv, d), d.cz).step;
            e[off + i] = __fmaf_rn(-a, __fmul_rn(step, __fmul_rn(l, val)), e[off + i]);
        }
    }
    if (PASS == 0) {
        const double b = block_sum_f64(s);
        if (threadIdx.x == 0) partial[(size_t)t * gridDim.x + blockIdx.x] = b;
    }
}

// alpha_t = -sum(theta1.delta) / (sum Lambda (A delta)^2 + sum(delta.delta)/sigma^2)
// per frame (one block each), from the partials of the group gather (bpf per
// frame) and of sinogram pass 0, summed in a fixed order.
__global__ void icd_alpha_kernel(const double* __restrict__ gpart, int bpf, const double* __restrict__ spart,
                                 double inv_s2, double* __restrict__ alpha, int* __restrict__ status) {
    const int t = blockIdx.x;
    double gd = 0.0, dd = 0.0, sq = 0.0;
    for (int i = threadIdx.x; i < bpf; i += blockDim.x) {
        gd += gpart[2 * ((size_t)t * bpf + i)];
        dd += gpart[2 * ((size_t)t * bpf + i) + 1];
    }
    for (int i = threadIdx.x; i < ICD_SINO_BLOCKS; i += blockDim.x) sq += spart[(size_t)t * ICD_SINO_BLOCKS + i];
    gd = block_sum_f64(gd);
    dd = block_sum_f64(dd);
    sq = block_sum_f64(sq);
    if (threadIdx.x == 0) {
        const double den = sq + dd * inv_s2;
        if (!isfinite(gd) || !isfinite(den)) atomicExch(status, (int)MSF_ERR_NUMERIC);
        alpha[t] = (den > 0.0 && isfinite(den) && isfinite(gd)) ? -gd / den : 0.0;
    }
}

// z_s += alpha_t delta_s and delta_s = 0 for the voxels of the group.
__global__ void icd_update_kernel(float* __restrict__ z, float* __restrict__ dlt, const double* __restrict__ alpha,
                                  IcdGroup G, ProjDims d) {
    const size_t per_frame = (size_t)G.gx * G.gy * G.gz;
    const size_t total = per_frame * d.nt;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(i / per_frame);
        size_t r = i % per_frame;
        const int jz = (int)(r / ((size_t)G.gx * G.gy));
        r %= (size_t)G.gx * G.gy;
        const int jy = (int)(r / G.gx), jx = (int)(r % G.gx);
        const size_t k = (((size_t)t * d.nz + 2 * jz + G.pz) * d.ny + 2 * jy + G.py) * d.nx + 2 * jx + G.px;
        z[k] = __fmaf_rn((float)alpha[t], dlt[k], z[k]);
        dlt[k] = 0.0f;
    }
}

// e2 = step^2 Lambda for every ray (input of the theta2 gather).
__global__ void icd_step2_kernel(const float4* __restrict__ col, const float* __restrict__ lam,
                                 float* __restrict__ out, ProjDims d) {
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int iv = blockIdx.y * 4 + threadIdx.y;
    const int g = blockIdx.z;
    if (iu >= d.nu || iv >= d.nv) return;
    const ColParams c = load_col(col, (size_t)g * d.nu + iu);
    const float step = ray_z(c, det_v(iv, d), d.cz).step;
    const size_t ray = ((size_t)g * d.nv + iv) * d.nu + iu;
    out[ray] = __fmul_rn(__fmul_rn(step, step), lam[ray]);
}

// ------------------------------------------------------------------ phantom (test data)

#define MSF_MAX_ELL_RECORDS 256
__constant__ double c_ell[MSF_MAX_ELL_RECORDS * 16];

__device__ __forceinline__ void ell_local(const double* e, double px, double py, double pz,
                                          double* q) {
    const double tx = px - e[0], ty = py - e[1], tz = pz - e[2];
    for (int k = 0; k < 3; ++k)
        q[k] = (e[6 + 3 * k] * tx + e[7 + 3 * k] * ty + e[8 + 3 * k] * tz) / e[3 + k];
}

__global__ void phantom_voxelize_kernel(float* __restrict__ x, int nx, int ny, int nz, int nt,
                                        double vox, int n_ell, int ss) {
    const size_t fs = (size_t)nx * ny * nz;
    const size_t total = fs * nt;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(i / fs);
        size_t r = i % fs;
        const int iz = (int)(r / ((size_t)nx * ny));
        r %= (size_t)nx * ny;
        const int iy = (int)(r / nx), ix = (int)(r % nx);
        double acc = 0.0;
        for (int e = 0; e < n_ell; ++e) {
            const double* E = c_ell + 16 * ((size_t)t * n_ell + e);
            int inside = 0;
            for (int a = 0; a < ss; ++a)
                for (int b = 0; b < ss; ++b)
                    for (int cc = 0; cc < ss; ++cc) {
                        double q[3];
                        ell_local(E, (ix - 0.5 * (nx - 1) + (cc + 0.5) / ss - 0.5) * vox,
                                  (iy - 0.5 * (ny - 1) + (b + 0.5) / ss - 0.5) * vox,
                                  (iz - 0.5 * (nz - 1) + (a + 0.5) / ss - 0.5) * vox, q);
                        inside += (q[0] * q[0] + q[1] * q[1] + q[2] * q[2] <= 1.0);
                    }
            acc += E[15] * (double)inside / (double)(ss * ss * ss);
        }
        x[i] = (float)acc;
    }
}

__global__ void phantom_project_kernel(const double* __restrict__ angles, float* __restrict__ y,
                                       ProjDims d, double du, double dv, double dso, double dsd,
                                       int n_ell) {
    const size_t per_view = (size_t)d.nu * d.nv;
    const size_t total = per_view * d.views * d.nt;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(i / per_view);
        const int t = g / d.views;
        const int iv = (int)((i % per_view) / d.nu), iu = (int)(i % d.nu);
        const double th = angles[g], c = cos(th), s = sin(th);
        const double u = (iu - 0.5 * (d.nu - 1)) * du, v = (iv - 0.5 * (d.nv - 1)) * dv;
        const double sx = dso * c, sy = dso * s;
        const double dx = -(dsd - dso) * c - u * s - sx, dy = -(dsd - dso) * s + u * c - sy,
                     dz = v;
        const double len = sqrt(dx * dx + dy * dy + dz * dz);
        double acc = 0.0;
        for (int e = 0; e < n_ell; ++e) {
            const double* E = c_ell + 16 * ((size_t)t * n_ell + e);
            double q0[3], q1[3];
            ell_local(E, sx, sy, 0.0, q0);
            for (int k = 0; k < 3; ++k)
                q1[k] = (E[6 + 3 * k] * dx + E[7 + 3 * k] * dy + E[8 + 3 * k] * dz) / E[3 + k];
            const double A = q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2];
            const double B = 2.0 * (q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2]);
            const double C = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] - 1.0;
            const double disc = B * B - 4.0 * A * C;
            if (disc > 0.0) acc += E[15] * len * sqrt(disc) / A;
        }
        y[i] = (float)acc;
    }
}

}  // namespace msf

// ====================================================================== handles

struct msf_projector {
    msf_geom geom;
    msf_vol vol;
    msf::ProjDims dims;
    std::vector<double> angles;
    double* d_angles = nullptr;
    float4* d_col = nullptr;
    float2* d_trig = nullptr;
    int* d_vflag = nullptr;
    float2* d_px = nullptr;    // z-paired volume, [nt][nz][nx][ny] (x-major rays)
    float2* d_py = nullptr;    // z-paired volume, [nt][nz][ny][nx] (y-major rays)
    float* d_sw = nullptr;     // step-weighted sinogram for msf_backproject
    int fwd_bx = 32, fwd_by = 4;   // forward ray block (columns x rows)
    int adj_zb = 16;               // gather z-run length
    uint64_t tuning_gen = 0;       // advanced whenever the launch shapes change
    size_t bytes = 0;
};

struct msf_dataprox {
    msf_projector* p = nullptr;
    float *d_r = nullptr, *d_p = nullptr, *d_p2 = nullptr, *d_q = nullptr, *d_s = nullptr;
    double *d_partial = nullptr, *d_rr = nullptr, *d_alpha = nullptr, *d_beta = nullptr;
    int* d_status = nullptr;
    int parts_adj = 0, parts_upd = 0, parts_max = 0;
    // grouped ICD: a second sinogram (A delta, and step^2 Lambda for theta2),
    // the group gather's partial sums and the sinogram pass's partial sums
    float* d_s2 = nullptr;
    double *d_ipart = nullptr, *d_spart = nullptr;
    int parts_icd = 0;
};

namespace msf {

static size_t frame_size(const msf_vol& v) { return (size_t)v.nx * v.ny * v.nz; }
static size_t vol_size(const msf_vol& v) { return frame_size(v) * v.nt; }
static size_t sino_size(const msf_projector* p) {
    return (size_t)p->geom.nu * p->geom.nv * p->geom.views * p->vol.nt;
}

static msf_status launch_pairs(msf_projector* p, const float* in, cudaStream_t st) {
    const msf_vol& v = p->vol;
    dim3 grid((v.nx + 31) / 32, (v.ny + 31) / 32, v.nz * v.nt);
    MSF_PROF("transpose", st);
    pair_kernel<false><<<grid, dim3(32, 8), 0, st>>>(in, p->d_px, p->d_py, nullptr, nullptr, nullptr, v.nx, v.ny, v.nz);
    MSF_LAUNCH_CHECK();
    return MSF_OK;
}

// Forward grid: blockDim.x columns x FWD_R*blockDim.y rows per block, one z per view.
static dim3 fwd_grid(const ProjDims& d, dim3 block) {
    const unsigned rows = block.y * FWD_R;
    return dim3((d.nu + block.x - 1) / block.x, (d.nv + rows - 1) / rows, d.nt * d.views);
}

static msf_status launch_fwd(msf_projector* p, int mode, const float* x, float* out,
                             const float* lam, const float* meas, cudaStream_t st) {
    MSF_TRY(launch_pairs(p, x, st));
    const ProjDims& d = p->dims;
    dim3 block(p->fwd_bx, p->fwd_by);
    dim3 grid = fwd_grid(d, block);
    MSF_PROF("joseph_fwd", st);
    if (mode == FWD_PLAIN)
        joseph_fwd_kernel<FWD_PLAIN><<<grid, block, 0, st>>>(p->d_px, p->d_py, p->d_col, out, lam, meas, d);
    else if (mode == FWD_LAMBDA)
        joseph_fwd_kernel<FWD_LAMBDA><<<grid, block, 0, st>>>(p->d_px, p->d_py, p->d_col, out, lam, meas, d);
    else
        joseph_fwd_kernel<FWD_RESIDUAL><<<grid, block, 0, st>>>(p->d_px, p->d_py, p->d_col, out, lam, meas, d);
    MSF_LAUNCH_CHECK();
    return MSF_OK;
}

// A x for an x that is zero outside the voxels with x = kpx and y = kpy (mod 2)
// (the ICD agent's group step), visiting only the planes that can touch them.
static msf_status launch_fwd_parity(msf_projector* p, const float* x, float* out, int kpx, int kpy, cudaStream_t st) {
    MSF_TRY(launch_pairs(p, x, st));
    const ProjDims& d = p->dims;
    dim3 block(p->fwd_bx, p->fwd_by);
    dim3 grid = fwd_grid(d, block);
    MSF_PROF("joseph_fwd", st);
    joseph_fwd_kernel<FWD_PLAIN, true><<<grid, block, 0, st>>>(p->d_px, p->d_py, p->d_col, out, nullptr, nullptr, d,
                                                               kpx, kpy);
    MSF_LAUNCH_CHECK();
    return MSF_OK;
}

static int adj_nzb(const ProjDims& d, int zb) { return (d.nz + zb - 1) / zb; }
static dim3 adj_grid(const ProjDims& d, int zb) { return dim3((d.nx + 31) / 32, (d.ny + 3) / 4, adj_nzb(d, zb) * d.nt); }
// partial sums per frame of an adjoint launch
static int adj_parts(const msf_projector* p) {
    const dim3 g = adj_grid(p->dims, p->adj_zb);
    return g.x * g.y * adj_nzb(p->dims, p->adj_zb);
}

template <int MODE>
static void launch_adj_zb(msf_projector* p, const float* e, float* out, const float* a1, const float* a2,
                          float* out2, double* partial, float inv_s2, cudaStream_t st) {
    const ProjDims& d = p->dims;
    const dim3 block(32, 4), grid = adj_grid(d, p->adj_zb);
    if (p->adj_zb == 8)
        joseph_adj_kernel<MODE, 8><<<grid, block, 0, st>>>(p->d_col, p->d_trig, p->d_vflag, e, out, a1, a2, out2, partial, inv_s2, d);
    else if (p->adj_zb == 32)
        joseph_adj_kernel<MODE, 32><<<grid, block, 0, st>>>(p->d_col, p->d_trig, p->d_vflag, e, out, a1, a2, out2, partial, inv_s2, d);
    else if (p->adj_zb == 64)
        joseph_adj_kernel<MODE, 64><<<grid, block, 0, st>>>(p->d_col, p->d_trig, p->d_vflag, e, out, a1, a2, out2, partial, inv_s2, d);
    else
        joseph_adj_kernel<MODE, 16><<<grid, block, 0, st>>>(p->d_col, p->d_trig, p->d_vflag, e, out, a1, a2, out2, partial, inv_s2, d);
}

static msf_status launch_adj(msf_projector* p, int mode, const float* e, float* out,
                             const float* a1, const float* a2, float* out2, double* partial,
                             float inv_s2, cudaStream_t st) {
    MSF_PROF("joseph_adj", st);
    if (mode == ADJ_PLAIN)
        launch_adj_zb<ADJ_PLAIN>(p, e, out, a1, a2, out2, partial, inv_s2, st);
    else if (mode == ADJ_CG_INIT)
        launch_adj_zb<ADJ_CG_INIT>(p, e, out, a1, a2, out2, partial, inv_s2, st);
    else
        launch_adj_zb<ADJ_CG_Q>(p, e, out, a1, a2, out2, partial, inv_s2, st);
    MSF_LAUNCH_CHECK();
    return MSF_OK;
}

}  // namespace msf

using namespace msf;

const msf_vol* msf::projector_volume(const msf_projector* p) { return &p->vol; }
int* msf::dataprox_status(msf_dataprox* d) { return d->d_status; }
size_t msf::projector_sino_size(const msf_projector* p) { return sino_size(p); }
void msf::projector_detector(const msf_projector* p, int* nu, int* nv) {
    *nu = p->geom.nu;
    *nv = p->geom.nv;
}

extern "C" msf_status msf_projector_create(const msf_geom* geom, const msf_vol* vol,
                                           msf_projector** out) {
    MSF_REQUIRE(geom && vol && out, "msf_projector_create: NULL argument");
    *out = nullptr;
    MSF_REQUIRE(vol->nx > 0 && vol->ny > 0 && vol->nz > 0 && vol->nt > 0 && vol->voxel > 0,
                "msf_projector_create: volume sizes and voxel must be positive");
    MSF_REQUIRE(geom->nu > 0 && geom->nv > 0 && geom->views > 0 && geom->du > 0 && geom->dv > 0,
                "msf_projector_create: detector sizes, pitch and views must be positive");
    MSF_REQUIRE(geom->angles != nullptr, "msf_projector_create: angles is NULL");
    const double R = 0.5 * vol->voxel * sqrt((double)vol->nx * vol->nx + (double)vol->ny * vol->ny);
    MSF_REQUIRE(geom->dso > R && geom->dsd - geom->dso > R,
                "msf_projector_create: source (dso=%g) and detector (dsd-dso=%g) must lie outside "
                "the volume's circumscribed cylinder (radius %g)", geom->dso, geom->dsd - geom->dso, R);
    const double vmax = 0.5 * (geom->nv - 1) * geom->dv;
    MSF_REQUIRE(vmax < geom->dsd / sqrt(2.0),
                "msf_projector_create: cone too wide (z-major rays are not modelled)");
    MSF_REQUIRE((size_t)vol->nt * vol->nx * vol->ny * vol->nz < (size_t)1 << 40,
                "msf_projector_create: volume too large");
    MSF_TRY(check_device());

    msf_projector* p = new msf_projector();
    p->geom = *geom;
    p->vol = *vol;
    const int G = vol->nt * geom->views;
    p->angles.assign(geom->angles, geom->angles + G);
    p->geom.angles = p->angles.data();
    ProjDims& d = p->dims;
    d.nx = vol->nx; d.ny = vol->ny; d.nz = vol->nz; d.nt = vol->nt;
    d.nu = geom->nu; d.nv = geom->nv; d.views = geom->views;
    d.cx = 0.5f * (vol->nx - 1); d.cy = 0.5f * (vol->ny - 1); d.cz = 0.5f * (vol->nz - 1);
    d.cu = 0.5f * (geom->nu - 1); d.cv = 0.5f * (geom->nv - 1);
    d.vox = (float)vol->voxel; d.du = (float)geom->du; d.dv = (float)geom->dv;
    d.dso = (float)geom->dso; d.dsd = (float)geom->dsd;

    auto cleanup = [&](msf_status st) { msf_projector_destroy(p); return st; };
    const size_t col_bytes = (size_t)G * geom->nu * 2 * sizeof(float4);
    const size_t vol_bytes = vol_size(*vol) * sizeof(float);
    if (cudaMalloc(&p->d_angles, G * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&p->d_col, col_bytes) != cudaSuccess ||
        cudaMalloc(&p->d_trig, G * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&p->d_vflag, G * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&p->d_px, 2 * vol_bytes) != cudaSuccess || cudaMalloc(&p->d_py, 2 * vol_bytes) != cudaSuccess ||
        cudaMalloc(&p->d_sw, sino_size(p) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(MSF_ERR_NOMEM, "msf_projector_create: out of device memory"));
    }
    p->bytes = G * sizeof(double) + col_bytes + G * (sizeof(float2) + sizeof(int)) + 4 * vol_bytes +
               sino_size(p) * sizeof(float);
    std::vector<float2> trig(G);
    for (int g = 0; g < G; ++g) trig[g] = make_float2((float)cos(p->angles[g]), (float)sin(p->angles[g]));
    int* d_bad = nullptr;
    int h_bad = 0;
    cudaError_t e = cudaMemcpy(p->d_angles, p->angles.data(), G * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_trig, trig.data(), G * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->d_vflag, 0, G * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d_bad, 0, sizeof(int));
    if (e == cudaSuccess) {
        column_table_kernel<<<dim3((geom->nu + 127) / 128, G), 128>>>(p->d_angles, p->d_col, p->d_vflag, d_bad, d, vol->voxel,
                                                                    geom->du, geom->dso, geom->dsd);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (d_bad) cudaFree(d_bad);
    if (e != cudaSuccess) return cleanup(fail(MSF_ERR_CUDA, "msf_projector_create: %s", cudaGetErrorString(e)));
    if (h_bad) return cleanup(fail(MSF_ERR_ARG, "msf_projector_create: a ray's voxel planes are not all "
                                               "between its source and detector"));
    *out = p;
    return MSF_OK;
}

extern "C" void msf_projector_destroy(msf_projector* p) {
    if (!p) return;
    cudaFree(p->d_angles);
    cudaFree(p->d_col);
    cudaFree(p->d_trig);
    cudaFree(p->d_vflag);
    cudaFree(p->d_px);
    cudaFree(p->d_py);
    cudaFree(p->d_sw);
    delete p;
}

extern "C" size_t msf_projector_bytes(const msf_projector* p) { return p ? p->bytes : 0; }

extern "C" msf_status msf_project(msf_projector* p, const float* d_x, float* d_y, void* stream) {
    MSF_REQUIRE(p && d_x && d_y, "msf_project: NULL argument");
    return launch_fwd(p, FWD_PLAIN, d_x, d_y, nullptr, nullptr, as_stream(stream));
}

extern "C" msf_status msf_backproject(msf_projector* p, const float* d_y, float* d_x, void* stream) {
    MSF_REQUIRE(p && d_x && d_y, "msf_backproject: NULL argument");
    cudaStream_t st = as_stream(stream);
    {
        const ProjDims& d = p->dims;
        MSF_PROF("step_weight", st);
        step_weight_kernel<<<dim3((d.nu + 31) / 32, (d.nv + 3) / 4, d.nt * d.views), dim3(32, 4), 0, st>>>(
            p->d_col, d_y, p->d_sw, d);
        MSF_LAUNCH_CHECK();
    }
    return launch_adj(p, ADJ_PLAIN, p->d_sw, d_x, nullptr, nullptr, nullptr, nullptr, 0.0f, st);
}

extern "C" msf_status msf_dataprox_create(msf_projector* p, msf_dataprox** out) {
    MSF_REQUIRE(p && out, "msf_dataprox_create: NULL argument");
    *out = nullptr;
    msf_dataprox* d = new msf_dataprox();
    d->p = p;
    const size_t nv = vol_size(p->vol), ns = sino_size(p);
    const dim3 ga = adj_grid(p->dims, 8);             // the largest block count of any z-run
    d->parts_adj = ga.x * ga.y * adj_nzb(p->dims, 8);
    d->parts_upd = 512;
    d->parts_max = d->parts_adj > d->parts_upd ? d->parts_adj : d->parts_upd;
    const int nt = p->vol.nt;
    {   // the largest group grid (parity 0 along every axis)
        const msf_vol& v = p->vol;
        d->parts_icd = ((par_count(v.nx, 0) + 31) / 32) * ((par_count(v.ny, 0) + 3) / 4) *
                       ((par_count(v.nz, 0) + ICD_ZB - 1) / ICD_ZB);
    }
    if (cudaMalloc(&d->d_s2, ns * 4) != cudaSuccess ||
        cudaMalloc(&d->d_ipart, (size_t)nt * d->parts_icd * 2 * 8) != cudaSuccess ||
        cudaMalloc(&d->d_spart, (size_t)nt * ICD_SINO_BLOCKS * 8) != cudaSuccess ||
        cudaMalloc(&d->d_r, nv * 4) != cudaSuccess || cudaMalloc(&d->d_p, nv * 4) != cudaSuccess ||
        cudaMalloc(&d->d_p2, nv * 4) != cudaSuccess ||
        cudaMalloc(&d->d_q, nv * 4) != cudaSuccess || cudaMalloc(&d->d_s, ns * 4) != cudaSuccess ||
        cudaMalloc(&d->d_partial, (size_t)nt * d->parts_max * 8) != cudaSuccess ||
        cudaMalloc(&d->d_rr, nt * 8) != cudaSuccess || cudaMalloc(&d->d_alpha, nt * 8) != cudaSuccess ||
        cudaMalloc(&d->d_beta, nt * 8) != cudaSuccess || cudaMalloc(&d->d_status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        msf_dataprox_destroy(d);
        return fail(MSF_ERR_NOMEM, "msf_dataprox_create: out of device memory");
    }
    if (cudaMemset(d->d_status, 0, sizeof(int)) != cudaSuccess) {
        msf_dataprox_destroy(d);
        return fail(MSF_ERR_CUDA, "msf_dataprox_create: memset failed");
    }
    *out = d;
    return MSF_OK;
}

extern "C" void msf_dataprox_destroy(msf_dataprox* d) {
    if (!d) return;
    cudaFree(d->d_r); cudaFree(d->d_p); cudaFree(d->d_p2); cudaFree(d->d_q); cudaFree(d->d_s);
    cudaFree(d->d_partial); cudaFree(d->d_rr); cudaFree(d->d_alpha); cudaFree(d->d_beta);
    cudaFree(d->d_status);
    cudaFree(d->d_s2); cudaFree(d->d_ipart); cudaFree(d->d_spart);
    delete d;
}

extern "C" msf_status msf_prox_data(msf_dataprox* dp, const float* d_y, const float* d_lambda,
                                    const float* d_v, float* d_x, double sigma, int n_cg, void* stream) {
    MSF_REQUIRE(dp && d_y && d_lambda && d_v && d_x, "msf_prox_data: NULL argument");
    MSF_REQUIRE(sigma > 0 && isfinite(sigma), "msf_prox_data: sigma must be positive");
    MSF_REQUIRE(n_cg >= 0, "msf_prox_data: n_cg must be >= 0");
    if (n_cg == 0) return MSF_OK;
    msf_projector* p = dp->p;
    cudaStream_t st = as_stream(stream);
    const float inv_s2 = (float)(1.0 / (sigma * sigma));
    const int nt = p->vol.nt;
    const size_t fs = frame_size(p->vol);
    // r = A^T Lambda (y - A z) + (v - z)/sigma^2 ; p = r ; rr = r.r
    MSF_TRY(launch_fwd(p, FWD_RESIDUAL, d_x, dp->d_s, d_lambda, d_y, st));
    MSF_TRY(launch_adj(p, ADJ_CG_INIT, dp->d_s, dp->d_r, d_v, d_x, dp->d_p, dp->d_partial, inv_s2, st));
    {
        MSF_PROF("cg_finalize", st);
        cg_finalize_kernel<FIN_RR0><<<nt, 256, 0, st>>>(dp->d_partial, adj_parts(p), dp->d_rr, nullptr, dp->d_status);
        MSF_LAUNCH_CHECK();
    }
    const msf_vol& v = p->vol;
    const dim3 tgrid((v.nx + 31) / 32, (v.ny + 31) / 32, v.nz * v.nt);
    // the direction p alternates between two buffers: the fused update reads
    // p at slices z and z + 1 while writing the new p
    float* pc = dp->d_p;
    for (int it = 0; it < n_cg; ++it) {
        // z-paired copies of p for the forward pass (fused with p = r + beta p after the first pass)
        if (it == 0) {
            MSF_TRY(launch_pairs(p, pc, st));
        } else {
            float* pn = pc == dp->d_p ? dp->d_p2 : dp->d_p;
            MSF_PROF("transpose_pupdate", st);
            pair_kernel<true><<<tgrid, dim3(32, 8), 0, st>>>(pc, p->d_px, p->d_py, dp->d_r, pn, dp->d_beta, v.nx,
                                                             v.ny, v.nz);
            MSF_LAUNCH_CHECK();
            pc = pn;
        }
        {   // s = Lambda A p  (pairs already built)
            const ProjDims& d = p->dims;
            dim3 block(p->fwd_bx, p->fwd_by);
            dim3 grid = fwd_grid(d, block);
            MSF_PROF("joseph_fwd", st);
            joseph_fwd_kernel<FWD_LAMBDA><<<grid, block, 0, st>>>(p->d_px, p->d_py, p->d_col, dp->d_s, d_lambda, nullptr, d);
            MSF_LAUNCH_CHECK();
        }
        // q = A^T s + p/sigma^2 ; alpha = rr / p.q
        MSF_TRY(launch_adj(p, ADJ_CG_Q, dp->d_s, dp->d_q, pc, nullptr, nullptr, dp->d_partial, inv_s2, st));
        {
            MSF_PROF("cg_finalize", st);
            cg_finalize_kernel<FIN_ALPHA><<<nt, 256, 0, st>>>(dp->d_partial, adj_parts(p), dp->d_rr, dp->d_alpha, dp->d_status);
            MSF_LAUNCH_CHECK();
        }
        {   // z += alpha p ; r -= alpha q ; beta = r.r / rr
            MSF_PROF("cg_update", st);
            cg_update_kernel<<<dim3(dp->parts_upd, nt), 256, 0, st>>>(d_x, dp->d_r, pc, dp->d_q, dp->d_alpha, dp->d_partial, fs);
            MSF_LAUNCH_CHECK();
        }
        {
            MSF_PROF("cg_finalize", st);
            cg_finalize_kernel<FIN_BETA><<<nt, 256, 0, st>>>(dp->d_partial, dp->parts_upd, dp->d_rr, dp->d_beta, dp->d_status);
            MSF_LAUNCH_CHECK();
        }
    }
    return MSF_OK;
}

extern "C" msf_status msf_prox_data_icd(msf_dataprox* dp, const float* d_y, const float* d_lambda,
                                        const float* d_v, float* d_x, double sigma, int n_sweeps, void* stream) {
    MSF_REQUIRE(dp && d_y && d_lambda && d_v && d_x, "msf_prox_data_icd: NULL argument");
    MSF_REQUIRE(sigma > 0 && isfinite(sigma), "msf_prox_data_icd: sigma must be positive");
    MSF_REQUIRE(n_sweeps >= 0, "msf_prox_data_icd: n_sweeps must be >= 0");
    if (n_sweeps == 0) return MSF_OK;
    msf_projector* p = dp->p;
    cudaStream_t st = as_stream(stream);
    const ProjDims& d = p->dims;
    const msf_vol& v = p->vol;
    const int nt = v.nt;
    const float inv_s2 = (float)(1.0 / (sigma * sigma));
    // e' = step Lambda (y - A z)
    MSF_TRY(launch_fwd(p, FWD_RESIDUAL, d_x, dp->d_s, d_lambda, d_y, st));
    {   // theta2 = (A^T Lambda A)_ss + 1/sigma^2
        MSF_PROF("icd_step2", st);
        icd_step2_kernel<<<dim3((d.nu + 31) / 32, (d.nv + 3) / 4, d.nt * d.views), dim3(32, 4), 0, st>>>(
            p->d_col, d_lambda, dp->d_s2, d);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("icd_theta2", st);
        const dim3 grid((d.nx + 31) / 32, (d.ny + 3) / 4, ((d.nz + 15) / 16) * d.nt);
        icd_theta2_kernel<16><<<grid, dim3(32, 4), 0, st>>>(p->d_col, p->d_trig, p->d_vflag, dp->d_s2, dp->d_q,
                                                            inv_s2, d);
        MSF_LAUNCH_CHECK();
    }
    MSF_TRY_CUDA(cudaMemsetAsync(dp->d_p, 0, vol_size(v) * sizeof(float), st));
    for (int sw = 0; sw < n_sweeps; ++sw) {
        for (int grp = 0; grp < 8; ++grp) {
            IcdGroup G;
            G.px = grp & 1; G.py = (grp >> 1) & 1; G.pz = grp >> 2;
            G.gx = par_count(v.nx, G.px); G.gy = par_count(v.ny, G.py); G.gz = par_count(v.nz, G.pz);
            if (G.gx == 0 || G.gy == 0 || G.gz == 0) continue;
            G.nzb = (G.gz + ICD_ZB - 1) / ICD_ZB;
            const dim3 grid((G.gx + 31) / 32, (G.gy + 3) / 4, G.nzb * nt);
            const int bpf = grid.x * grid.y * G.nzb;
            {
                MSF_PROF("icd_group", st);
                icd_group_kernel<ICD_ZB><<<grid, dim3(32, 4), 0, st>>>(p->d_col, p->d_trig, p->d_vflag, dp->d_s,
                                                                      d_x, d_v, dp->d_q, dp->d_p, dp->d_ipart,
                                                                      inv_s2, G, d);
                MSF_LAUNCH_CHECK();
            }
            // A delta: delta is zero outside the group (icd_update clears it)
            MSF_TRY(launch_fwd_parity(p, dp->d_p, dp->d_s2, G.px, G.py, st));
            {
                MSF_PROF("icd_sino", st);
                icd_sino_kernel<0><<<dim3(ICD_SINO_BLOCKS, nt), 256, 0, st>>>(p->d_col, dp->d_s2, d_lambda, dp->d_s,
                                                                              nullptr, dp->d_spart, d);
                MSF_LAUNCH_CHECK();
            }
            {
                MSF_PROF("icd_alpha", st);
                icd_alpha_kernel<<<nt, 256, 0, st>>>(dp->d_ipart, bpf, dp->d_spart, 1.0 / (sigma * sigma), dp->d_alpha,
                                                     dp->d_status);
                MSF_LAUNCH_CHECK();
            }
            {
                MSF_PROF("icd_update", st);
                icd_update_kernel<<<152 * 4, 256, 0, st>>>(d_x, dp->d_p, dp->d_alpha, G, d);
                MSF_LAUNCH_CHECK();
            }
            {
                MSF_PROF("icd_sino", st);
                icd_sino_kernel<1><<<dim3(ICD_SINO_BLOCKS, nt), 256, 0, st>>>(p->d_col, dp->d_s2, d_lambda, dp->d_s,
                                                                              dp->d_alpha, nullptr, d);
                MSF_LAUNCH_CHECK();
            }
        }
    }
    return MSF_OK;
}

extern "C" msf_status msf_phantom_voxelize(const msf_vol* vol, const double* h_ell, int n_ell, int ss,
                                           float* d_x, void* stream) {
    MSF_REQUIRE(vol && h_ell && d_x, "msf_phantom_voxelize: NULL argument");
    MSF_REQUIRE(n_ell > 0 && ss > 0 && (size_t)n_ell * vol->nt <= MSF_MAX_ELL_RECORDS,
                "msf_phantom_voxelize: need 0 < n_ell*nt <= %d and ss > 0", MSF_MAX_ELL_RECORDS);
    cudaStream_t st = as_stream(stream);
    MSF_TRY_CUDA(cudaMemcpyToSymbolAsync(c_ell, h_ell, (size_t)n_ell * vol->nt * 16 * sizeof(double), 0,
                                         cudaMemcpyHostToDevice, st));
    phantom_voxelize_kernel<<<152 * 8, 256, 0, st>>>(d_x, vol->nx, vol->ny, vol->nz, vol->nt, vol->voxel, n_ell, ss);
    MSF_LAUNCH_CHECK();
    MSF_TRY_CUDA(cudaStreamSynchronize(st));   // c_ell is reused by the next call
    return MSF_OK;
}

extern "C" msf_status msf_phantom_project(msf_projector* p, const double* h_ell, int n_ell, float* d_y,
                                          void* stream) {
    MSF_REQUIRE(p && h_ell && d_y, "msf_phantom_project: NULL argument");
    MSF_REQUIRE(n_ell > 0 && (size_t)n_ell * p->vol.nt <= MSF_MAX_ELL_RECORDS,
                "msf_phantom_project: need 0 < n_ell*nt <= %d", MSF_MAX_ELL_RECORDS);
    cudaStream_t st = as_stream(stream);
    MSF_TRY_CUDA(cudaMemcpyToSymbolAsync(c_ell, h_ell, (size_t)n_ell * p->vol.nt * 16 * sizeof(double), 0,
                                         cudaMemcpyHostToDevice, st));
    phantom_project_kernel<<<152 * 8, 256, 0, st>>>(p->d_angles, d_y, p->dims, p->geom.du, p->geom.dv,
                                                    p->geom.dso, p->geom.dsd, n_ell);
    MSF_LAUNCH_CHECK();
    MSF_TRY_CUDA(cudaStreamSynchronize(st));
    return MSF_OK;
}

// ====================================================================== no-allocation forward projection
//
// msf_project_static: the forward projection of msf_project for callers that
// cannot allocate device memory.  The per-column ray table that a projector
// plan would own lives instead in the file-scope device array below, of fixed
// size, which every GPU that loads this library keeps until the process exits.
// The frame is read in its natural layout for both ray families (no transposed
// copy), so the caller's input and output are the only other memory touched.

namespace msf {

constexpr size_t STATIC_SCRATCH_BYTES = (size_t)8 << 20;   // 8 MiB
constexpr int STATIC_MAX_VIEWS = 8192;                      // nt * views
constexpr size_t STATIC_MAX_COLUMNS = 250000;               // nt * views * nu

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Layout inside the array: [angles: G doubles][column table: G*nu*32 B]
// [view flags: G ints][geometry flag: 1 int].
static_assert(STATIC_MAX_VIEWS * 8 + STATIC_MAX_COLUMNS * 32 + STATIC_MAX_VIEWS * 4 + 256 <= STATIC_SCRATCH_BYTES,
              "static scratch too small for its stated limits");

// Joseph forward projection reading the frame [nz][ny][nx] for both ray
// families.  Per crossing it performs the forward's operations with the same
// explicit roundings (the lerp v00 + w_a (v01 - v00) along a, then along z,
// and a round-to-nearest accumulation over increasing planes), and a plane
// whose taps all lie outside the grid adds exactly zero in joseph_fwd_kernel,
// so the result equals msf_project's bit for bit; only the addressing differs
// (x-major rays read x-strided data here instead of the transposed copy).
__global__ void __launch_bounds__(128) joseph_fwd_direct_kernel(const float* __restrict__ x,
                                                                const float4* __restrict__ col,
                                                                float* __restrict__ out, ProjDims d) {
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int iv = blockIdx.y * 4 + threadIdx.y;
    const int g = blockIdx.z;
    if (iu >= d.nu || iv >= d.nv) return;
    const int t = g / d.views;
    const ColParams c = load_col(col, (size_t)g * d.nu + iu);
    const bool xmaj = c.xmajor != 0.0f;
    const int nmaj = xmaj ? d.nx : d.ny, na = xmaj ? d.ny : d.nx;
    const float* __restrict__ vol = x + (size_t)t * d.nx * d.ny * d.nz;
    // element (iz, plane k, minor ia): x-major -> x[iz][ia][k], y-major -> x[iz][k][ia]
    const ptrdiff_t s_maj = xmaj ? 1 : d.nx, s_min = xmaj ? d.nx : 1;
    const ptrdiff_t s_z = (ptrdiff_t)d.nx * d.ny;
    const float cmaj = xmaj ? d.cx : d.cy;
    const RayZ rz = ray_z(c, det_v(iv, d), d.cz);
    float acc = 0.0f;
    for (int k = 0; k < nmaj; ++k) {
        const float tk = __fsub_rn((float)k, cmaj);
        const float fa = __fmaf_rn(tk, c.ba, c.fa_mid);
        const float fz = __fmaf_rn(tk, rz.bz, rz.fz_mid);
        const float a0f = floorf(fa), z0f = floorf(fz);
        if (a0f < -1.0f || a0f > (float)(na - 1) || z0f < -1.0f || z0f > (float)(d.nz - 1)) continue;
        const float wa1 = __fsub_rn(fa, a0f), wz1 = __fsub_rn(fz, z0f);
        const int ia = (int)a0f, iz = (int)z0f;
        const bool a_in0 = ia >= 0, a_in1 = ia + 1 < na;
        const bool z_in0 = iz >= 0, z_in1 = iz + 1 < d.nz;
        const float* p00 = vol + iz * s_z + k * s_maj + ia * s_min;
        const float v00 = (z_in0 && a_in0) ? __ldg(p00) : 0.0f;
        const float v01 = (z_in0 && a_in1) ? __ldg(p00 + s_min) : 0.0f;
        const float v10 = (z_in1 && a_in0) ? __ldg(p00 + s_z) : 0.0f;
        const float v11 = (z_in1 && a_in1) ? __ldg(p00 + s_z + s_min) : 0.0f;
        const float top = __fmaf_rn(wa1, __fsub_rn(v01, v00), v00);
        const float bot = __fmaf_rn(wa1, __fsub_rn(v11, v10), v10);
        acc = __fadd_rn(acc, __fmaf_rn(wz1, __fsub_rn(bot, top), top));
    }
    out[((size_t)g * d.nv + iv) * d.nu + iu] = __fmul_rn(acc, rz.step);
}

// Device address of g_static_scratch for each device, looked up once per
// device (with that device current) on the first call made on it.
static std::mutex g_static_mu;
static void* g_static_ptr[128] = {nullptr};

}  // namespace msf

extern "C" msf_status msf_project_static(const msf_geom* geom, const msf_vol* vol, const float* d_x, float* d_y,
                                         void* stream) {
    MSF_REQUIRE(geom && vol && d_x && d_y && geom->angles, "msf_project_static: NULL argument");
    MSF_REQUIRE(vol->nx > 0 && vol->ny > 0 && vol->nz > 0 && vol->nt > 0 && vol->voxel > 0,
                "msf_project_static: volume sizes and voxel must be positive");
    MSF_REQUIRE(geom->nu > 0 && geom->nv > 0 && geom->views > 0 && geom->du > 0 && geom->dv > 0,
                "msf_project_static: detector sizes, pitch and views must be positive");
    const long long G = (long long)vol->nt * geom->views;
    MSF_REQUIRE(G <= STATIC_MAX_VIEWS && (size_t)G * geom->nu <= STATIC_MAX_COLUMNS,
                "msf_project_static: nt*views = %lld and nt*views*nu = %lld exceed the static table "
                "(at most %d views and %zu view-columns); use msf_projector_create + msf_project",
                G, G * geom->nu, STATIC_MAX_VIEWS, STATIC_MAX_COLUMNS);
    const double R = 0.5 * vol->voxel * sqrt((double)vol->nx * vol->nx + (double)vol->ny * vol->ny);
    MSF_REQUIRE(geom->dso > R && geom->dsd - geom->dso > R,
                "msf_project_static: source and detector must lie outside the volume's circumscribed cylinder");
    MSF_REQUIRE(0.5 * (geom->nv - 1) * geom->dv < geom->dsd / sqrt(2.0),
                "msf_project_static: cone too wide (z-major rays are not modelled)");
    // The voxel planes of every ray must lie between its source and detector.
    // This is checked here in FP64 on the host for every (view, column) -- at
    // most STATIC_MAX_COLUMNS evaluations -- with the formulas of
    // column_table_kernel, so no device flag has to be read back (the table
    // kernel still writes its flag into the array; nothing reads it).  Checking
    // only the end columns would not do: where a view's columns switch between
    // x-major and y-major, the first column of the inner segment can fail alone.
    for (long long g = 0; g < G; ++g) {
        const double th = geom->angles[g], c = cos(th), s = sin(th);
        const double sx = geom->dso * c, sy = geom->dso * s;
        for (int iu = 0; iu < geom->nu; ++iu) {
            const double u = (iu - 0.5 * (geom->nu - 1)) * geom->du;
            const double dx = -(geom->dsd - geom->dso) * c - u * s - sx, dy = -(geom->dsd - geom->dso) * s + u * c - sy;
            const bool xm = fabs(dx) >= fabs(dy);
            const double dmaj = xm ? dx : dy, smaj = xm ? sx : sy;
            const int nmaj = xm ? vol->nx : vol->ny;
            const double l1 = (-0.5 * (nmaj - 1) * vol->voxel - smaj) / dmaj;
            const double l2 = (0.5 * (nmaj - 1) * vol->voxel - smaj) / dmaj;
            MSF_REQUIRE(fmin(l1, l2) > 0.0 && fmax(l1, l2) < 1.0,
                        "msf_project_static: a ray's voxel planes are not all between its source and detector "
                        "(view %lld, column %d)", g, iu);
        }
    }
    int dev = 0;
    MSF_TRY_CUDA(cudaGetDevice(&dev));
    MSF_REQUIRE(dev >= 0 && dev < 128, "msf_project_static: device index %d out of range", dev);
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            MSF_TRY(check_device());
            cudaError_t e = cudaGetSymbolAddress(&g_static_ptr[dev], g_static_scratch);
            if (e != cudaSuccess) {
                g_static_ptr[dev] = nullptr;
                return fail(MSF_ERR_CUDA, "msf_project_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            }
        }
        base = g_static_ptr[dev];
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    double* d_angles = reinterpret_cast<double*>(b);
    float4* d_col = reinterpret_cast<float4*>(b + (size_t)STATIC_MAX_VIEWS * 8);
    int* d_vflag = reinterpret_cast<int*>(b + (size_t)STATIC_MAX_VIEWS * 8 + STATIC_MAX_COLUMNS * 32);
    int* d_bad = d_vflag + STATIC_MAX_VIEWS;
    ProjDims d;
    d.nx = vol->nx; d.ny = vol->ny; d.nz = vol->nz; d.nt = vol->nt;
    d.nu = geom->nu; d.nv = geom->nv; d.views = geom->views;
    d.cx = 0.5f * (vol->nx - 1); d.cy = 0.5f * (vol->ny - 1); d.cz = 0.5f * (vol->nz - 1);
    d.cu = 0.5f * (geom->nu - 1); d.cv = 0.5f * (geom->nv - 1);
    d.vox = (float)vol->voxel; d.du = (float)geom->du; d.dv = (float)geom->dv;
    d.dso = (float)geom->dso; d.dsd = (float)geom->dsd;
    cudaStream_t st = as_stream(stream);
    // the array keeps the previous call's contents: the flags start at zero
    MSF_TRY_CUDA(cudaMemcpyAsync(d_angles, geom->angles, G * sizeof(double), cudaMemcpyHostToDevice, st));
    MSF_TRY_CUDA(cudaMemsetAsync(d_vflag, 0, G * sizeof(int), st));
    MSF_TRY_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    {
        MSF_PROF("column_table", st);
        column_table_kernel<<<dim3((geom->nu + 127) / 128, (unsigned)G), 128, 0, st>>>(
            d_angles, d_col, d_vflag, d_bad, d, vol->voxel, geom->du, geom->dso, geom->dsd);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("joseph_fwd_direct", st);
        joseph_fwd_direct_kernel<<<dim3((d.nu + 31) / 32, (d.nv + 3) / 4, (unsigned)G), dim3(32, 4), 0, st>>>(
            d_x, d_col, d_y, d);
        MSF_LAUNCH_CHECK();
    }
    return MSF_OK;
}

// ====================================================================== autotuning

namespace msf {
uint64_t projector_tuning_gen(const msf_projector* p) { return p ? p->tuning_gen : 0; }
}  // namespace msf

extern "C" msf_status msf_projector_set_tuning(msf_projector* p, int fwd_cols, int fwd_rows, int adj_zrun) {
    MSF_REQUIRE(p, "msf_projector_set_tuning: NULL plan");
    MSF_REQUIRE((fwd_cols == 32 && fwd_rows == 4) || (fwd_cols == 64 && fwd_rows == 2) ||
                    (fwd_cols == 16 && fwd_rows == 8),
                "msf_projector_set_tuning: forward block %dx%d is not 32x4, 64x2 or 16x8", fwd_cols, fwd_rows);
    MSF_REQUIRE(adj_zrun == 8 || adj_zrun == 16 || adj_zrun == 32 || adj_zrun == 64,
                "msf_projector_set_tuning: adjoint z-run %d is not 8, 16, 32 or 64", adj_zrun);
    p->fwd_bx = fwd_cols;
    p->fwd_by = fwd_rows;
    p->adj_zb = adj_zrun;
    ++p->tuning_gen;
    return MSF_OK;
}

extern "C" msf_status msf_projector_autotune(msf_projector* p, void* stream, int* h_choice) {
    MSF_REQUIRE(p, "msf_projector_autotune: NULL plan");
    cudaStream_t st = as_stream(stream);
    const size_t nv = vol_size(p->vol), ns = sino_size(p);
    // inputs: the plan's own scratch (transposed stack and step-weighted sinogram)
    // are overwritten; outputs go to a temporary buffer allocated here
    float* tmp = nullptr;
    MSF_TRY_CUDA(cudaMalloc(&tmp, (nv > ns ? nv : ns) * sizeof(float)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    msf_status st_ = MSF_OK;
    auto time_it = [&](auto&& fn) -> float {
        fn();   // warm
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) fn();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    MSF_TRY_CUDA(cudaMemsetAsync(p->d_px, 0, nv * sizeof(float2), st));
    MSF_TRY_CUDA(cudaMemsetAsync(p->d_py, 0, nv * sizeof(float2), st));
    MSF_TRY_CUDA(cudaMemsetAsync(p->d_sw, 0, ns * sizeof(float), st));
    const int shapes[3][2] = {{32, 4}, {64, 2}, {16, 8}};
    float best = 1e30f;
    int bi = 0;
    for (int i = 0; i < 3; ++i) {
        p->fwd_bx = shapes[i][0];
        p->fwd_by = shapes[i][1];
        const float ms = time_it([&] {
            const ProjDims& d = p->dims;
            dim3 block(p->fwd_bx, p->fwd_by);
            dim3 grid = fwd_grid(d, block);
            joseph_fwd_kernel<FWD_PLAIN><<<grid, block, 0, st>>>(p->d_px, p->d_py, p->d_col, tmp, nullptr, nullptr, d);
        });
        if (ms < best) { best = ms; bi = i; }
    }
    p->fwd_bx = shapes[bi][0];
    p->fwd_by = shapes[bi][1];
    // z-runs of 64 halve the gather's block count; they are tried only while
    // their grid stays at least 24 waves deep (8 blocks per SM), because with a
    // shallower grid, run beside other problems' kernels (a batch), the longer
    // blocks measured slower although they won when timed alone
    const int zbs[4] = {8, 16, 32, 64};
    int nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        nsm = 0;
    const dim3 g64 = adj_grid(p->dims, 64);
    const bool deep64 = nsm > 0 && (double)g64.x * g64.y * g64.z >= 24.0 * 8.0 * nsm;
    best = 1e30f;
    int bz = 1;
    for (int i = 0; i < (deep64 ? 4 : 3); ++i) {
        p->adj_zb = zbs[i];
        const float ms = time_it([&] { launch_adj_zb<ADJ_PLAIN>(p, p->d_sw, tmp, nullptr, nullptr, nullptr, nullptr, 0.0f, st); });
        if (ms < best) { best = ms; bz = i; }
    }
    p->adj_zb = zbs[bz];
    ++p->tuning_gen;
    if (cudaGetLastError() != cudaSuccess) st_ = fail(MSF_ERR_CUDA, "msf_projector_autotune: a trial launch failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tmp);
    if (h_choice) {
        h_choice[0] = p->fwd_bx;
        h_choice[1] = p->fwd_by;
        h_choice[2] = p->adj_zb;
    }
    return st_;
}
