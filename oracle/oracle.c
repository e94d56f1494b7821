/*
 * FP64 CPU oracle for multi-slice fusion (arXiv 2008.01567) -- loop-heavy parts.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA path (paper_2008_01567_gb300/csrc).
 *
 * Contents
 *   or_project            Joseph ray-driven cone-beam projector A_n (forward) and
 *                         its literal transpose A_n^T (same ray loop, scatter-add).
 *                         A_n is the system matrix of Sec. II, Eq. (2); the paper
 *                         leaves its model to its cone-beam reference, so the rules
 *                         below are this project's reading (circular orbit, flat
 *                         detector, Joseph interpolation).
 *                         Mode 2 is the transpose with squared weights,
 *                         x_s = sum_r a_rs^2 y_r, the diagonal of A^T diag(y) A
 *                         (the curvature that ICD divides by, Sec. III).
 *   or_ellipsoid_project  exact line integrals of a sum of uniform ellipsoids
 *                         (measurement simulation, Sec. VII-A: noisy data from the
 *                         projection of a phantom that moves one voxel per frame).
 *   or_ellipsoid_voxelize supersampled voxelisation of the same phantom.
 *   or_qggmrf_*           q-GGMRF potential, its symmetric-bound surrogate
 *                         coefficient, and a 16-colour ICD solver for the prior
 *                         proximal map H(v) of Sec. III, Eq. (5) with the 4D MRF
 *                         prior of Sec. VII (26 spatial + 2 temporal neighbours);
 *                         the surrogate's Laplacian for the direct MAP solve.
 *
 * Geometry (all lengths in the caller's unit):
 *   voxel (ix,iy,iz) centre = ((ix-(nx-1)/2)*vox, (iy-(ny-1)/2)*vox, (iz-(nz-1)/2)*vox)
 *   view angle th: source s = (dso cos th, dso sin th, 0)
 *                  detector centre c = -(dsd-dso)(cos th, sin th, 0)
 *                  u axis (-sin th, cos th, 0), v axis (0,0,1)
 *                  pixel (iu,iv) centre = c + (iu-(nu-1)/2) du u + (iv-(nv-1)/2) dv v
 *   ray direction d = pixel - s.  Major axis: x when |d_x| >= |d_y|, else y.
 *   For every voxel-centre plane of the major axis, the volume slice is sampled
 *   bilinearly (taps outside the volume count as zero) at the ray's crossing
 *   point, and the sample is weighted by vox*|d|/|d_major| (chord per plane).
 * Layouts: volume [nz][ny][nx] (x fastest), sinogram [nviews][nv][nu] (u fastest).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- geometry */

typedef struct {
    double sx, sy, sz;   /* source */
    double dx, dy, dz;   /* direction to the detector pixel centre (not normalised) */
} or_ray;

static or_ray ray_of(double th, int iu, int iv, int nu, int nv, double du, double dv,
                     double dso, double dsd)
{
    or_ray r;
    double c = cos(th), s = sin(th);
    double u = (iu - 0.5 * (nu - 1)) * du;
    double v = (iv - 0.5 * (nv - 1)) * dv;
    double px = -(dsd - dso) * c + u * (-s);
    double py = -(dsd - dso) * s + u * c;
    double pz = v;
    r.sx = dso * c; r.sy = dso * s; r.sz = 0.0;
    r.dx = px - r.sx; r.dy = py - r.sy; r.dz = pz - r.sz;
    return r;
}

/* Joseph sampling of one ray: visits every (voxel, weight) pair of the ray and
 * either gathers (adjoint == 0: returns sum w*x[v]) or scatters (adjoint == 1:
 * x[v] += w*val; adjoint == 2: x[v] += w*w*val).  One routine for both
 * directions makes A^T the literal transpose of A.  A ray meets a voxel on one
 * plane only (the plane of the voxel's major-axis index), so w is the whole
 * matrix entry a_rv and w*w its square. */
static double joseph_ray(const or_ray* r, double* x, int nx, int ny, int nz, double vox,
                         int adjoint, double val)
{
    double len = sqrt(r->dx * r->dx + r->dy * r->dy + r->dz * r->dz);
    double acc = 0.0;
    int xmajor = fabs(r->dx) >= fabs(r->dy);
    int nmaj = xmajor ? nx : ny;       /* planes along the major axis */
    int na = xmajor ? ny : nx;         /* first minor axis (the other in-plane axis) */
    double dmaj = xmajor ? r->dx : r->dy;
    double smaj = xmajor ? r->sx : r->sy;
    double da = xmajor ? r->dy : r->dx;
    double sa = xmajor ? r->sy : r->sx;
    double step = vox * len / fabs(dmaj);
    for (int k = 0; k < nmaj; ++k) {
        double pc = (k - 0.5 * (nmaj - 1)) * vox;     /* plane coordinate */
        double lam = (pc - smaj) / dmaj;
        double a = sa + lam * da;                      /* in-plane minor coordinate */
        double z = r->sz + lam * r->dz;
        double fa = a / vox + 0.5 * (na - 1);          /* fractional voxel index */
        double fz = z / vox + 0.5 * (nz - 1);
        double a0f = floor(fa), z0f = floor(fz);
        if (a0f < -1.0 || a0f > na - 1 || z0f < -1.0 || z0f > nz - 1) continue;
        int a0 = (int)a0f, z0 = (int)z0f;
        double wa1 = fa - a0f, wz1 = fz - z0f;
        double wa[2] = {1.0 - wa1, wa1}, wz[2] = {1.0 - wz1, wz1};
        for (int jz = 0; jz < 2; ++jz) {
            int iz = z0 + jz;
            if (iz < 0 || iz >= nz) continue;
            for (int ja = 0; ja < 2; ++ja) {
                int ia = a0 + ja;
                if (ia < 0 || ia >= na) continue;
                size_t idx = xmajor ? ((size_t)iz * ny + ia) * nx + k
                                    : ((size_t)iz * ny + k) * nx + ia;
                double w = step * wa[ja] * wz[jz];
                if (adjoint == 2) x[idx] += w * w * val;
                else if (adjoint) x[idx] += w * val;
                else acc += w * x[idx];
            }
        }
    }
    return acc;
}

/* Forward (adjoint == 0): y[view][iv][iu] = (A x).  Adjoint (adjoint == 1):
 * x = A^T y; adjoint == 2: x = (A.^2)^T y (x is overwritten in both).  Angles
 * in radians, one per view. */
void or_project(double* x, double* y, int nx, int ny, int nz, double vox,
                int nu, int nv, double du, double dv, double dso, double dsd,
                const double* angles, int nviews, int adjoint)
{
    if (adjoint) {
        memset(x, 0, sizeof(double) * (size_t)nx * ny * nz);
        for (int j = 0; j < nviews; ++j)
            for (int iv = 0; iv < nv; ++iv)
                for (int iu = 0; iu < nu; ++iu) {
                    or_ray r = ray_of(angles[j], iu, iv, nu, nv, du, dv, dso, dsd);
                    double val = y[((size_t)j * nv + iv) * nu + iu];
                    if (val != 0.0) joseph_ray(&r, x, nx, ny, nz, vox, adjoint, val);
                }
        return;
    }
    #pragma omp parallel for schedule(dynamic) collapse(2)
    for (int j = 0; j < nviews; ++j)
        for (int iv = 0; iv < nv; ++iv)
            for (int iu = 0; iu < nu; ++iu) {
                or_ray r = ray_of(angles[j], iu, iv, nu, nv, du, dv, dso, dsd);
                y[((size_t)j * nv + iv) * nu + iu] = joseph_ray(&r, x, nx, ny, nz, vox, 0, 0.0);
            }
}

/* ----------------------------------------------------------------- phantom */
/* Ellipsoid record: 16 doubles = centre(3), semi-axes(3), rotation R(9, row-major;
 * row k is the k-th ellipsoid axis in world coordinates), attenuation mu(1).
 * A point P is inside when sum_k ((R (P-c))_k / a_k)^2 <= 1.  Overlaps add. */

static void ell_local(const double* e, const double* p, double* q)
{
    const double* c = e; const double* ax = e + 3; const double* R = e + 6;
    double t[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
    for (int k = 0; k < 3; ++k)
        q[k] = (R[3 * k] * t[0] + R[3 * k + 1] * t[1] + R[3 * k + 2] * t[2]) / ax[k];
}

static void ell_local_dir(const double* e, const double* d, double* q)
{
    const double* ax = e + 3; const double* R = e + 6;
    for (int k = 0; k < 3; ++k)
        q[k] = (R[3 * k] * d[0] + R[3 * k + 1] * d[1] + R[3 * k + 2] * d[2]) / ax[k];
}

/* Exact line integral through the ellipsoids along the infinite line s + lam d:
 * chord length = |d| * (lam2 - lam1) where lam1,2 solve |q0 + lam q1|^2 = 1. */
void or_ellipsoid_project(const double* ell, int nell, double* y,
                          int nu, int nv, double du, double dv, double dso, double dsd,
                          const double* angles, int nviews)
{
    #pragma omp parallel for schedule(static) collapse(2)
    for (int j = 0; j < nviews; ++j)
        for (int iv = 0; iv < nv; ++iv)
            for (int iu = 0; iu < nu; ++iu) {
                or_ray r = ray_of(angles[j], iu, iv, nu, nv, du, dv, dso, dsd);
                double s[3] = {r.sx, r.sy, r.sz}, d[3] = {r.dx, r.dy, r.dz};
                double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                double acc = 0.0;
                for (int e = 0; e < nell; ++e) {
                    const double* E = ell + 16 * e;
                    double q0[3], q1[3];
                    ell_local(E, s, q0);
                    ell_local_dir(E, d, q1);
                    double A = q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2];
                    double B = 2.0 * (q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2]);
                    double C = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] - 1.0;
                    double disc = B * B - 4.0 * A * C;
                    if (disc > 0.0) acc += E[15] * len * sqrt(disc) / A;
                }
                y[((size_t)j * nv + iv) * nu + iu] = acc;
            }
}

/* Voxel value = sum_e mu_e * (fraction of the ss^3 sub-sample points inside e). */
void or_ellipsoid_voxelize(const double* ell, int nell, double* x, int nx, int ny, int nz,
                           double vox, int ss)
{
    #pragma omp parallel for schedule(static) collapse(2)
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                double acc = 0.0;
                for (int e = 0; e < nell; ++e) {
                    const double* E = ell + 16 * e;
                    int inside = 0;
                    for (int a = 0; a < ss; ++a)
                        for (int b = 0; b < ss; ++b)
                            for (int c = 0; c < ss; ++c) {
                                double p[3] = {
                                    (ix - 0.5 * (nx - 1) + (c + 0.5) / ss - 0.5) * vox,
                                    (iy - 0.5 * (ny - 1) + (b + 0.5) / ss - 0.5) * vox,
                                    (iz - 0.5 * (nz - 1) + (a + 0.5) / ss - 0.5) * vox};
                                double q[3];
                                ell_local(E, p, q);
                                if (q[0] * q[0] + q[1] * q[1] + q[2] * q[2] <= 1.0) ++inside;
                            }
                    acc += E[15] * (double)inside / (double)(ss * ss * ss);
                }
                x[((size_t)iz * ny + iy) * nx + ix] = acc;
            }
}

/* ----------------------------------------------------------------- q-GGMRF */
/* Potential (Thibault et al., Med. Phys. 2007):
 *   rho(D) = |D|^p / (p sx^p) * u/(1+u),   u = |D/(T sx)|^(q-p),   1 <= q <= p.
 * Surrogate coefficient a(D) = rho'(D)/(2D), written with r = 1/u = |D/(T sx)|^(p-q):
 *   a(D) = |D|^(p-2)/(2 sx^p) * (1 + (q/p) r)/(1 + r)^2,
 * which is finite at D = 0 for p = 2 (the case this project supports). */
double or_qggmrf_rho(double D, double p, double q, double T, double sx)
{
    double ad = fabs(D);
    if (ad == 0.0) return 0.0;
    double u = pow(ad / (T * sx), q - p);
    return pow(ad, p) / (p * pow(sx, p)) * u / (1.0 + u);
}

double or_qggmrf_coef(double D, double p, double q, double T, double sx)
{
    double ad = fabs(D);
    double r = pow(ad / (T * sx), p - q);
    return pow(ad, p - 2.0) / (2.0 * pow(sx, p)) * (1.0 + (q / p) * r) / ((1.0 + r) * (1.0 + r));
}

/* Neighbour weights: 26 spatial neighbours with b proportional to 1/distance,
 * normalised to sum to 1; 2 temporal neighbours with weight bt each. */
static void nb_weights(double* bface, double* bedge, double* bcorner)
{
    double s = 6.0 + 12.0 / sqrt(2.0) + 8.0 / sqrt(3.0);
    *bface = 1.0 / s; *bedge = 1.0 / (sqrt(2.0) * s); *bcorner = 1.0 / (sqrt(3.0) * s);
}

/* Prior cost h(z) = sum over unordered neighbour pairs {s,r} of b_sr rho(z_s - z_r)
 * on a 4D volume [nt][nz][ny][nx] with free boundaries. */
double or_qggmrf_cost(const double* z, int nx, int ny, int nz, int nt,
                      double p, double q, double T, double sx, double bt)
{
    double bf, be, bc;
    nb_weights(&bf, &be, &bc);
    double h = 0.0;
    for (int t = 0; t < nt; ++t)
        for (int iz = 0; iz < nz; ++iz)
            for (int iy = 0; iy < ny; ++iy)
                for (int ix = 0; ix < nx; ++ix) {
                    size_t s = (((size_t)t * nz + iz) * ny + iy) * nx + ix;
                    /* each unordered pair once: take neighbours with a positive
                     * lexicographic offset (dt,dz,dy,dx) */
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int pos = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
                                if (!pos) continue;
                                int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                                if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                                int m = abs(dx) + abs(dy) + abs(dz);
                                double b = m == 1 ? bf : (m == 2 ? be : bc);
                                size_t r = (((size_t)t * nz + jz) * ny + jy) * nx + jx;
                                h += b * or_qggmrf_rho(z[s] - z[r], p, q, T, sx);
                            }
                    if (t + 1 < nt) {
                        size_t r = s + (size_t)nz * ny * nx;
                        h += bt * or_qggmrf_rho(z[s] - z[r], p, q, T, sx);
                    }
                }
    return h;
}

/* ICD for H(v) = argmin_z ||v - z||^2/(2 sigma^2) + h(z)  (Sec. III, Eq. (5)).
 * One sweep visits the 16 colours c = ((pt*2+pz)*2+py)*2+px in increasing order,
 * where (px,py,pz,pt) are the parities of (ix,iy,iz,t); no two voxels of one
 * colour are neighbours.  Each voxel takes the minimiser of the symmetric-bound
 * quadratic surrogate built at the current values:
 *   z_s <- (v_s/sigma^2 + 2 sum_r b_sr a_sr z_r) / (1/sigma^2 + 2 sum_r b_sr a_sr),
 *   a_sr = a(z_s - z_r).
 * z holds the starting point on entry and the result on exit. */
void or_qggmrf_icd(const double* v, double* z, int nx, int ny, int nz, int nt,
                   double sigma, double p, double q, double T, double sx, double bt,
                   int nsweeps)
{
    double bf, be, bc;
    nb_weights(&bf, &be, &bc);
    double is2 = 1.0 / (sigma * sigma);
    size_t fs = (size_t)nz * ny * nx;
    for (int sw = 0; sw < nsweeps; ++sw)
        for (int col = 0; col < 16; ++col) {
            int px = col & 1, py = (col >> 1) & 1, pz = (col >> 2) & 1, pt = (col >> 3) & 1;
            for (int t = pt; t < nt; t += 2)
                for (int iz = pz; iz < nz; iz += 2)
                    for (int iy = py; iy < ny; iy += 2)
                        for (int ix = px; ix < nx; ix += 2) {
                            size_t s = (((size_t)t * nz + iz) * ny + iy) * nx + ix;
                            double zs = z[s], num = v[s] * is2, den = is2;
                            for (int dz = -1; dz <= 1; ++dz)
                                for (int dy = -1; dy <= 1; ++dy)
                                    for (int dx = -1; dx <= 1; ++dx) {
                                        if (!dx && !dy && !dz) continue;
                                        int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                                        if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                                        int m = abs(dx) + abs(dy) + abs(dz);
                                        double b = m == 1 ? bf : (m == 2 ? be : bc);
                                        double zr = z[(((size_t)t * nz + jz) * ny + jy) * nx + jx];
                                        double ba = b * or_qggmrf_coef(zs - zr, p, q, T, sx);
                                        num += 2.0 * ba * zr; den += 2.0 * ba;
                                    }
                            for (int dt = -1; dt <= 1; dt += 2) {
                                int tt = t + dt;
                                if (tt < 0 || tt >= nt) continue;
                                double zr = z[s + (ptrdiff_t)dt * (ptrdiff_t)fs];
                                double ba = bt * or_qggmrf_coef(zs - zr, p, q, T, sx);
                                num += 2.0 * ba * zr; den += 2.0 * ba;
                            }
                            z[s] = num / den;
                        }
        }
}

/* The Laplacian of the symmetric-bound surrogate of h built at `anchor`:
 *   out_s = sum_{r in N(s)} b_sr a(anchor_s - anchor_r) (x_s - x_r),
 * over the 26 spatial and 2 temporal neighbours (free boundaries).  The
 * surrogate Q(x) = sum over pairs b_sr a_sr (x_s - x_r)^2 majorises h up to a
 * constant and touches it at the anchor; its gradient is 2 * out. */
void or_qggmrf_surrogate_lap(const double* anchor, const double* x, double* out, int nx, int ny, int nz,
                             int nt, double p, double q, double T, double sx, double bt)
{
    double bf, be, bc;
    nb_weights(&bf, &be, &bc);
    size_t fs = (size_t)nz * ny * nx;
    for (int t = 0; t < nt; ++t)
        for (int iz = 0; iz < nz; ++iz)
            for (int iy = 0; iy < ny; ++iy)
                for (int ix = 0; ix < nx; ++ix) {
                    size_t s = (size_t)t * fs + ((size_t)iz * ny + iy) * nx + ix;
                    double acc = 0.0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                if (!dx && !dy && !dz) continue;
                                int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                                if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                                int m = abs(dx) + abs(dy) + abs(dz);
                                double b = m == 1 ? bf : (m == 2 ? be : bc);
                                size_t r = (size_t)t * fs + ((size_t)jz * ny + jy) * nx + jx;
                                acc += b * or_qggmrf_coef(anchor[s] - anchor[r], p, q, T, sx) * (x[s] - x[r]);
                            }
                    for (int dt = -1; dt <= 1; dt += 2) {
                        int tt = t + dt;
                        if (tt < 0 || tt >= nt) continue;
                        size_t r = s + (ptrdiff_t)dt * (ptrdiff_t)fs;
                        acc += bt * or_qggmrf_coef(anchor[s] - anchor[r], p, q, T, sx) * (x[s] - x[r]);
                    }
                    out[s] = acc;
                }
}
