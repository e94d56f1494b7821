"""FP64 CPU oracle for multi-slice fusion (arXiv 2008.01567).

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA library is
checked against.  Only tests/, the smoke check and the benchmark's CPU-baseline
leg may import it.  It shares no code with the CUDA path; the loop-heavy parts
(projector, phantom, q-GGMRF ICD) are plain C in oracle.c, the rest is numpy in
float64 written in the paper's order and notation.

Every function names the passage it follows, and states in its docstring the
reading it takes where the paper leaves a point open (projector model, CNN
depth and width, temporal edges, ...).  All functions here are pinned by tests
under tests/ against closed forms, invariants, brute force or library routines;
none is marked unpinned.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.or_project.argtypes = [P, P, I, I, I, D, I, I, D, D, D, D, P, I, I]
        lib.or_ellipsoid_project.argtypes = [P, I, P, I, I, D, D, D, D, P, I]
        lib.or_ellipsoid_voxelize.argtypes = [P, I, P, I, I, I, D, I]
        lib.or_qggmrf_rho.argtypes = [D, D, D, D, D]
        lib.or_qggmrf_rho.restype = D
        lib.or_qggmrf_coef.argtypes = [D, D, D, D, D]
        lib.or_qggmrf_coef.restype = D
        lib.or_qggmrf_cost.argtypes = [P, I, I, I, I, D, D, D, D, D]
        lib.or_qggmrf_cost.restype = D
        lib.or_qggmrf_icd.argtypes = [P, P, I, I, I, I, D, D, D, D, D, D, I]
        lib.or_qggmrf_surrogate_lap.argtypes = [P, P, P, I, I, I, I, D, D, D, D, D]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


# ====================================================================== Sec. II
# Measurement model: y_n = A_n x_n + noise, l(x) = 1/2 sum_n ||y_n - A_n x_n||^2_Lambda_n.


def project(x3: np.ndarray, scan, angles: np.ndarray) -> np.ndarray:
    """y = A_n x_n for one frame (Sec. II, Eq. (2)); x3 [nz,ny,nx] -> y [views,nv,nu]."""
    x3 = np.ascontiguousarray(x3, dtype=np.float64)
    angles = np.ascontiguousarray(angles, dtype=np.float64)
    y = np.zeros((len(angles), scan.nv, scan.nu))
    nz, ny, nx = x3.shape
    _L().or_project(_p(x3), _p(y), nx, ny, nz, scan.vox, scan.nu, scan.nv, scan.pitch,
                    scan.pitch, scan.dso, scan.dsd, _p(angles), len(angles), 0)
    return y


def backproject(y3: np.ndarray, scan, angles: np.ndarray, shape=None) -> np.ndarray:
    """x = A_n^T y_n for one frame: the literal transpose (scatter) of `project`."""
    y3 = np.ascontiguousarray(y3, dtype=np.float64)
    angles = np.ascontiguousarray(angles, dtype=np.float64)
    nz, ny, nx = shape if shape is not None else (scan.n, scan.n, scan.n)
    x = np.zeros((nz, ny, nx))
    _L().or_project(_p(x), _p(y3), nx, ny, nz, scan.vox, scan.nu, scan.nv, scan.pitch,
                    scan.pitch, scan.dso, scan.dsd, _p(angles), len(angles), 1)
    return x


def project4d(x4: np.ndarray, scan) -> np.ndarray:
    """A x for the whole 4D volume: frames are independent (Eq. (2) is separable)."""
    ang = scan.angles()
    return np.stack([project(x4[t], scan, ang[t]) for t in range(x4.shape[0])])


def backproject4d(y4: np.ndarray, scan, shape3=None) -> np.ndarray:
    ang = scan.angles()
    return np.stack([backproject(y4[t], scan, ang[t], shape3) for t in range(y4.shape[0])])


def ellipsoid_sinogram(ell4: np.ndarray, scan) -> np.ndarray:
    """Exact line integrals of the ellipsoid phantom, frame by frame -> [nt,V,nv,nu]."""
    ang = scan.angles()
    out = np.zeros((scan.nt, scan.views, scan.nv, scan.nu))
    for t in range(scan.nt):
        e = np.ascontiguousarray(ell4[t], dtype=np.float64)
        a = np.ascontiguousarray(ang[t])
        _L().or_ellipsoid_project(_p(e), e.shape[0], _p(out[t]), scan.nu, scan.nv, scan.pitch,
                                  scan.pitch, scan.dso, scan.dsd, _p(a), scan.views)
    return out


def ellipsoid_volume(ell4: np.ndarray, scan, ss: int = 4) -> np.ndarray:
    """Supersampled voxelisation of the phantom -> [nt,n,n,n]."""
    out = np.zeros((scan.nt, scan.n, scan.n, scan.n))
    for t in range(scan.nt):
        e = np.ascontiguousarray(ell4[t], dtype=np.float64)
        _L().or_ellipsoid_voxelize(_p(e), e.shape[0], _p(out[t]), scan.n, scan.n, scan.n, scan.vox, ss)
    return out


def expected_counts(p: np.ndarray, I0: float) -> np.ndarray:
    """Beer-Lambert mean photon count I0 exp(-p) for line integrals p."""
    return I0 * np.exp(-p)


def log_measurement(counts: np.ndarray, I0: float) -> np.ndarray:
    """y = -ln(max(n,1)/I0): zero counts are clamped to one photon."""
    return -np.log(np.maximum(counts, 1.0) / I0)


def weights(y: np.ndarray, c: float) -> np.ndarray:
    """Lambda_n = diag{c exp(-y_n)} (Sec. II, below Eq. (2))."""
    return c * np.exp(-y)


# ====================================================================== Sec. III
# Data proximal map L(x) = argmin_z l(z) + ||x - z||^2 / (2 sigma^2)   (Eq. (4)).


def normal_op(z3, lam3, scan, angles, sigma):
    """(A^T Lambda A + I/sigma^2) z for one frame: the Hessian of the cost in Eq. (4)."""
    return backproject(lam3 * project(z3, scan, angles), scan, angles, z3.shape) + z3 / sigma ** 2


def prox_data_frame(y3, lam3, v3, z3, scan, angles, sigma, n_cg):
    """Partial update L~(v; z) of Eq. (13): n_cg conjugate-gradient iterations on
    (A^T Lambda A + I/sigma^2) z = A^T Lambda y + v/sigma^2, warm-started at z.
    Textbook Hestenes-Stiefel CG; the scalars are kept per frame."""
    z = np.array(z3, dtype=np.float64)
    r = backproject(lam3 * (y3 - project(z, scan, angles)), scan, angles, z.shape) + (v3 - z) / sigma ** 2
    p = r.copy()
    rr = float(np.vdot(r, r))
    for _ in range(n_cg):
        q = normal_op(p, lam3, scan, angles, sigma)
        pq = float(np.vdot(p, q))
        if pq == 0.0:
            break
        alpha = rr / pq
        z += alpha * p
        r -= alpha * q
        rr_new = float(np.vdot(r, r))
        beta = rr_new / rr if rr != 0.0 else 0.0
        p = r + beta * p
        rr = rr_new
    return z


def prox_data(y4, lam4, v4, z4, scan, sigma, n_cg):
    """L~ for the 4D volume: one independent CG per time-point (Eq. (2) separable, Sec. VI)."""
    ang = scan.angles()
    return np.stack([prox_data_frame(y4[t], lam4[t], v4[t], z4[t], scan, ang[t], sigma, n_cg)
                     for t in range(v4.shape[0])])


def backproject_sq(y3: np.ndarray, scan, angles: np.ndarray, shape=None) -> np.ndarray:
    """x_s = sum_r a_rs^2 y_r for one frame: the transpose of `project` with each
    matrix entry squared (with y = Lambda, the diagonal of A^T Lambda A)."""
    y3 = np.ascontiguousarray(y3, dtype=np.float64)
    angles = np.ascontiguousarray(angles, dtype=np.float64)
    nz, ny, nx = shape if shape is not None else (scan.n, scan.n, scan.n)
    x = np.zeros((nz, ny, nx))
    _L().or_project(_p(x), _p(y3), nx, ny, nz, scan.vox, scan.nu, scan.nv, scan.pitch,
                    scan.pitch, scan.dso, scan.dsd, _p(angles), len(angles), 2)
    return x


def parity_groups(shape3) -> list:
    """The eight voxel groups of the grouped ICD sweep: voxel (z, y, x) belongs to
    group (pz*2 + py)*2 + px with (pz, py, px) = (z, y, x) mod 2; groups are
    visited in increasing order.  Returned as boolean masks."""
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape3], indexing="ij")
    key = ((z % 2) * 2 + (y % 2)) * 2 + (x % 2)
    return [key == g for g in range(8)]


def data_cost(y3, lam3, v3, z3, scan, angles, sigma) -> float:
    """The cost of Eq. (4) with l of Eq. (2) for one frame:
    1/2 ||y - A z||^2_Lambda + ||z - v||^2 / (2 sigma^2)."""
    e = y3 - project(z3, scan, angles)
    return 0.5 * float(np.sum(lam3 * e * e)) + float(np.sum((z3 - v3) ** 2)) / (2.0 * sigma ** 2)


def prox_data_icd_frame(y3, lam3, v3, z3, scan, angles, sigma, n_sweeps, groups=None):
    """Partial update L~(v; z) of Eq. (13) by iterative coordinate descent
    (Sec. III takes L~ as a few ICD iterations), in a grouped order that a GPU
    can run in parallel: each sweep visits the voxel groups in order; within a
    group every voxel takes its own one-dimensional Newton step against the
    same error sinogram,
        theta1_s = -(A^T Lambda e)_s + (z_s - v_s)/sigma^2,
        theta2_s = (A^T Lambda A)_ss + 1/sigma^2,     delta_s = -theta1_s/theta2_s,
    (e = y - A z), and the group moves by alpha * delta, with alpha the exact
    minimiser of the quadratic cost along delta,
        alpha = -theta1.delta / (||A delta||^2_Lambda + ||delta||^2/sigma^2),
    before e is updated and the next group is visited.  With one voxel per
    group alpha = 1 and this is plain sequential ICD; with several it is a
    descent step of the cost in every group.  groups: list of boolean masks
    (default: the eight parity groups)."""
    z = np.array(z3, dtype=np.float64)
    if groups is None:
        groups = parity_groups(z.shape)
    e = y3 - project(z, scan, angles)
    theta2 = backproject_sq(lam3, scan, angles, z.shape) + 1.0 / sigma ** 2
    for _ in range(n_sweeps):
        for g in groups:
            theta1 = -backproject(lam3 * e, scan, angles, z.shape) + (z - v3) / sigma ** 2
            delta = np.where(g, -theta1 / theta2, 0.0)
            Ad = project(delta, scan, angles)
            den = float(np.sum(lam3 * Ad * Ad)) + float(np.sum(delta * delta)) / sigma ** 2
            if den <= 0.0:
                continue
            alpha = -float(np.sum(theta1 * delta)) / den
            z += alpha * delta
            e -= alpha * Ad
    return z


def prox_data_icd(y4, lam4, v4, z4, scan, sigma, n_sweeps):
    """The grouped-ICD L~ for the 4D volume: one independent solve per time-point."""
    ang = scan.angles()
    return np.stack([prox_data_icd_frame(y4[t], lam4[t], v4[t], z4[t], scan, ang[t], sigma, n_sweeps)
                     for t in range(v4.shape[0])])


# Prior proximal map H(x) = argmin_z ||x - z||^2/(2 sigma^2) + h(z)   (Eq. (5)),
# with h the 4D q-GGMRF MRF of Sec. VII (26 spatial + 2 temporal neighbours).


def qggmrf_rho(d, p, q, T, sx):
    return _L().or_qggmrf_rho(float(d), p, q, T, sx)


def qggmrf_coef(d, p, q, T, sx):
    return _L().or_qggmrf_coef(float(d), p, q, T, sx)


def qggmrf_cost(z4, p, q, T, sx, bt):
    z4 = np.ascontiguousarray(z4, dtype=np.float64)
    nt, nz, ny, nx = z4.shape
    return _L().or_qggmrf_cost(_p(z4), nx, ny, nz, nt, p, q, T, sx, bt)


def prox_qggmrf(v4, z4, sigma, p, q, T, sx, bt, n_sweeps):
    """n_sweeps 16-colour ICD sweeps for H(v), starting from z4 (see oracle.c)."""
    v4 = np.ascontiguousarray(v4, dtype=np.float64)
    z = np.array(z4, dtype=np.float64, order="C")
    nt, nz, ny, nx = v4.shape
    _L().or_qggmrf_icd(_p(v4), _p(z), nx, ny, nz, nt, sigma, p, q, T, sx, bt, n_sweeps)
    return z


# The MBIR + 4D-MRF comparison of Sec. VI solved directly: the MAP estimate of
# Eq. (3) with the q-GGMRF prior, without the MACE split.


def surrogate_lap(anchor4, x4, p, q, T, sx, bt):
    """(L_a x)_s = sum_r b_sr a(anchor_s - anchor_r) (x_s - x_r); 2 L_a x is the
    gradient of the prior's quadratic surrogate built at `anchor` (see oracle.c)."""
    a = np.ascontiguousarray(anchor4, dtype=np.float64)
    x = np.ascontiguousarray(x4, dtype=np.float64)
    out = np.zeros_like(x)
    nt, nz, ny, nx = x.shape
    _L().or_qggmrf_surrogate_lap(_p(a), _p(x), _p(out), nx, ny, nz, nt, p, q, T, sx, bt)
    return out


def map_cost(y4, lam4, x4, scan, p, q, T, sx, bt, beta) -> float:
    """Phi(x) = l(x) + beta h(x) = 1/2 sum_t ||y_t - A x_t||^2_Lambda + beta h(x), the
    MAP cost of Eq. (3) with the 4D q-GGMRF prior h of Sec. VII."""
    e = y4 - project4d(x4, scan)
    return 0.5 * float(np.sum(lam4 * e * e)) + beta * qggmrf_cost(x4, p, q, T, sx, bt)


def map_mm(y4, lam4, x4, scan, p, q, T, sx, bt, beta, n_outer, n_cg):
    """Direct MAP solve of Eq. (3), l(x) + beta h(x), by majorise-minimise: each
    outer iteration replaces h by its symmetric-bound quadratic surrogate built
    at the current x (equal to h there, above it elsewhere), and takes n_cg
    conjugate-gradient steps, warm-started at x, on the surrogate problem
        (A^T Lambda A + 2 beta L_a) x = A^T Lambda y
    over the whole 4D volume (the prior couples the time-points, so the CG
    scalars are global).  With MACE weights mu = (mu_0, mu_1) and exact agents
    the consensus equilibrium of Sec. III is this MAP point with beta = mu_1/mu_0."""
    x = np.array(x4, dtype=np.float64)
    ang = scan.angles()
    nt = x.shape[0]

    def data_normal(v):
        return np.stack([backproject(lam4[t] * project(v[t], scan, ang[t]), scan, ang[t], v[t].shape)
                         for t in range(nt)])

    for _ in range(n_outer):
        anchor = x.copy()
        r = np.stack([backproject(lam4[t] * (y4[t] - project(x[t], scan, ang[t])), scan, ang[t], x[t].shape)
                      for t in range(nt)]) - 2.0 * beta * surrogate_lap(anchor, x, p, q, T, sx, bt)
        d = r.copy()
        rr = float(np.vdot(r, r))
        for _ in range(n_cg):
            qv = data_normal(d) + 2.0 * beta * surrogate_lap(anchor, d, p, q, T, sx, bt)
            dq = float(np.vdot(d, qv))
            if dq == 0.0:
                break
            alpha = rr / dq
            x += alpha * d
            r -= alpha * qv
            rr_new = float(np.vdot(r, r))
            d = r + (rr_new / rr if rr != 0.0 else 0.0) * d
            rr = rr_new
    return x


# Blind correction of fixtures outside the field of view (Appendix A, Algorithm 2).


def cylinder_mask(shape3, vox, r_mask) -> np.ndarray:
    """1 for voxels whose centre lies within r_mask of the rotation axis (z), else 0."""
    nz, ny, nx = shape3
    yc = (np.arange(ny) - 0.5 * (ny - 1)) * vox
    xc = (np.arange(nx) - 0.5 * (nx - 1)) * vox
    inside = (xc[None, :] ** 2 + yc[:, None] ** 2) <= r_mask ** 2
    return np.broadcast_to(inside[None], (nz, ny, nx)).astype(np.float64)


def gaussian_taps(sigma_px: float) -> np.ndarray:
    """Normalised Gaussian taps g_k ~ exp(-k^2 / (2 sigma^2)), |k| <= ceil(3 sigma)."""
    R = int(math.ceil(3.0 * sigma_px))
    k = np.arange(-R, R + 1, dtype=np.float64)
    g = np.exp(-k * k / (2.0 * sigma_px * sigma_px))
    return g / g.sum()


def blur_sinogram(e4, sigma_px):
    """Separable Gaussian blur of every view of a sinogram [..., nv, nu] along u
    then v, detector pixels outside the detector counting as zero."""
    g = gaussian_taps(sigma_px)
    R = (len(g) - 1) // 2
    out = np.array(e4, dtype=np.float64)
    for axis in (-1, -2):
        n = out.shape[axis]
        pad = [(0, 0)] * out.ndim
        pad[axis] = (R, R)
        ep = np.pad(out, pad)
        acc = np.zeros_like(out)
        for j, gj in enumerate(g):
            acc += gj * np.take(ep, np.arange(j, j + n), axis=axis)
        out = acc
    return out


def fixture_correct(y4, x4, scan, r_mask, sigma_px):
    """Algorithm 2 given the reconstruction x = recon(y, A):
        x^m = mask(x)                  (cylinder of radius r_mask)
        e   = y - A x^m
        p   = blur(e)                  (separable Gaussian, sigma_px detector pixels)
        c   = argmin_c ||e - c p||^2 = <e, p> / <p, p>   (one scalar for the scan)
        y^corr = y - c p.
    Returns (y_corr, c)."""
    m = cylinder_mask(x4.shape[1:], scan.vox, r_mask)
    e = y4 - project4d(x4 * m[None], scan)
    p = blur_sinogram(e, sigma_px)
    pp = float(np.sum(p * p))
    c = float(np.sum(e * p)) / pp if pp > 0 else 0.0
    return y4 - c * p, c


# MACE operators.


def mu_from_beta(beta: float, K: int) -> np.ndarray:
    """Agent weights of the average in Eq. (9): mu_0 = 1/(1+beta), mu_k = beta/((1+beta)K)."""
    return np.array([1.0 / (1.0 + beta)] + [beta / ((1.0 + beta) * K)] * K)


def average(W, mu):
    """W-bar of Eq. (9) as the weighted sum sum_i mu_i W_i."""
    return sum(m * w for m, w in zip(mu, W))


def G(W, mu):
    """Averaging operator of Eq. (8): every block becomes W-bar."""
    wb = average(W, mu)
    return [wb.copy() for _ in W]


def mann_step_direct(W, FW, mu, rho):
    """Eq. (12): W <- (1-rho) W + rho T W with T = (2G - I)(2F - I), given F(W)."""
    V = [2.0 * f - w for f, w in zip(FW, W)]
    GV = G(V, mu)
    TW = [2.0 * g - v for g, v in zip(GV, V)]
    return [(1.0 - rho) * w + rho * t for w, t in zip(W, TW)]


def mace_iteration(W, X, agents, mu, rho):
    """One pass of Algorithm 1: X <- F~(W; X); Z <- G(2X - W); W <- W + 2 rho (Z - X).

    agents[i](W_i, X_i) returns the new X_i (agent 0 is the partial-update data
    prox L~, the others the prior agents H_k).  Returns (W, X, residual)."""
    X = [agents[i](W[i], X[i]) for i in range(len(W))]
    zbar = average([2.0 * x - w for x, w in zip(X, W)], mu)
    W = [w + 2.0 * rho * (zbar - x) for w, x in zip(W, X)]
    return W, X, consensus_residual(X, mu)


def consensus_residual(X, mu):
    """sqrt(sum_i mu_i ||X_i - X-bar||^2) / ||X-bar||: the spread between the agents'
    states that the stopping rule of Sec. III compares with a threshold."""
    xb = average(X, mu)
    num = sum(m * float(np.vdot(x - xb, x - xb)) for m, x in zip(mu, X))
    den = float(np.vdot(xb, xb))
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)


def mace(x0, agents, mu, rho, n_iter):
    """Algorithm 1 from X = W = [x0; ...; x0]; returns (X_0, W, X, residuals)."""
    W = [np.array(x0, dtype=np.float64) for _ in agents]
    X = [np.array(x0, dtype=np.float64) for _ in agents]
    res = []
    for _ in range(n_iter):
        W, X, r = mace_iteration(W, X, agents, mu, rho)
        res.append(r)
    return X[0], W, X, res


# Metrics (Sec. VII-A).


def nrmse(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def psnr(x, ref):
    """20 log10(Range(ref)/RMSE), Range = 99.9th minus 0.1st percentile of ref."""
    rng = np.percentile(ref, 99.9) - np.percentile(ref, 0.1)
    return 20.0 * math.log10(rng / math.sqrt(float(np.mean((x - ref) ** 2))))


def ssim_map2d(a, b, L, win=11, sd=1.5, k1=0.01, k2=0.03):
    """SSIM map of two 2D images (Wang et al.): local means, variances and
    covariance under a normalised win x win Gaussian window (standard deviation
    sd), at every window position wholly inside the image, combined as
    (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
    C1 = (k1 L)^2, C2 = (k2 L)^2.  Written as the windowed sums themselves."""
    r = np.arange(win) - (win - 1) / 2.0
    g1 = np.exp(-r * r / (2.0 * sd * sd))
    w = np.outer(g1, g1)
    w /= w.sum()
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    H, W = a.shape
    out = np.empty((H - win + 1, W - win + 1))
    c1, c2 = (k1 * L) ** 2, (k2 * L) ** 2
    for i in range(H - win + 1):
        for j in range(W - win + 1):
            pa = a[i:i + win, j:j + win]
            pb = b[i:i + win, j:j + win]
            mx, my = float((w * pa).sum()), float((w * pb).sum())
            sxx = float((w * (pa - mx) ** 2).sum())
            syy = float((w * (pb - my) ** 2).sum())
            sxy = float((w * (pa - mx) * (pb - my)).sum())
            out[i, j] = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return out


def ssim(x, ref, L=None):
    """Mean SSIM over every 2D slice of the last two axes (xy-slices of each
    time-point of a 4D volume); L defaults to the PSNR's percentile range of ref."""
    if L is None:
        L = np.percentile(ref, 99.9) - np.percentile(ref, 0.1)
    H, W = ref.shape[-2:]
    xs = np.asarray(x, dtype=np.float64).reshape(-1, H, W)
    rs = np.asarray(ref, dtype=np.float64).reshape(-1, H, W)
    maps = [ssim_map2d(a, b, L) for a, b in zip(xs, rs)]
    return float(np.mean(np.stack(maps)))


# ====================================================================== Sec. IV-V
# 2.5D CNN denoiser: five adjacent time-points of a 2D slice enter as channels and
# the denoised centre slice comes out, with a residual connection through the
# centre channel.  Depth 10, 3x3 kernels, 64 channels, ReLU, BatchNorm in the
# hidden layers (residual learning as in DnCNN).

ORIENTS = ("xy", "yz", "zx")


def orient_slices(v4: np.ndarray, orient: str) -> np.ndarray:
    """4D [nt,nz,ny,nx] -> images [nt, S, H, W] in the plane of the agent:
    xy-t: slice z, image (y, x); yz-t: slice x, image (z, y); zx-t: slice y, image (x, z)."""
    if orient == "xy":
        return v4
    if orient == "yz":
        return v4.transpose(0, 3, 1, 2)
    if orient == "zx":
        return v4.transpose(0, 2, 3, 1)
    raise ValueError(orient)


def orient_volume(s4: np.ndarray, orient: str) -> np.ndarray:
    """Inverse of orient_slices."""
    if orient == "xy":
        return s4
    if orient == "yz":
        return s4.transpose(0, 2, 3, 1)
    if orient == "zx":
        return s4.transpose(0, 3, 1, 2)
    raise ValueError(orient)


def window5(s4: np.ndarray) -> np.ndarray:
    """[nt,S,H,W] -> network input [nt*S, 5, H, W]: channels are time-points
    t-2..t+2 of the same slice, clamped at the first and last time-point."""
    nt = s4.shape[0]
    idx = np.clip(np.arange(nt)[:, None] + np.arange(-2, 3)[None, :], 0, nt - 1)
    x = s4[idx]                              # [nt, 5, S, H, W]
    x = x.transpose(0, 2, 1, 3, 4)           # [nt, S, 5, H, W]
    return np.ascontiguousarray(x.reshape(nt * s4.shape[1], 5, s4.shape[2], s4.shape[3]))


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, w, b=None):
    """y[n,o,i,j] = b[o] + sum_{c,ky,kx} w[o,c,ky,kx] x[n,c,i+ky-1,j+kx-1], zero padding."""
    n, c, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((n, w.shape[0], h, wd))
    for ky in range(3):
        for kx in range(3):
            y += np.tensordot(w[:, :, ky, kx], xp[:, :, ky:ky + h, kx:kx + wd], axes=([1], [1])).transpose(1, 0, 2, 3)
    if b is not None:
        y += b[None, :, None, None]
    return y


def conv3x3_dgrad(dy, w):
    """Input gradient of conv3x3: correlation of dy with the flipped, transposed kernel."""
    return conv3x3(dy, np.ascontiguousarray(w.transpose(1, 0, 2, 3)[:, :, ::-1, ::-1]))


def conv3x3_wgrad(dy, x):
    """Weight gradient of conv3x3: dw[o,c,ky,kx] = sum_{n,i,j} dy[n,o,i,j] x[n,c,i+ky-1,j+kx-1]."""
    n, c, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dw = np.zeros((dy.shape[1], c, 3, 3))
    for ky in range(3):
        for kx in range(3):
            dw[:, :, ky, kx] = np.tensordot(dy, xp[:, :, ky:ky + h, kx:kx + wd], axes=([0, 2, 3], [0, 2, 3]))
    return dw


BN_EPS = 1e-5


def fold_bn(convs, bns, stats):
    """Inference network with BatchNorm folded into the hidden convolutions:
    w' = w * g/sqrt(var+eps), b' = (b - mean) g/sqrt(var+eps) + beta."""
    out = [convs[0]]
    for l in range(1, len(convs) - 1):
        w, b = convs[l]
        g, be = bns[l - 1]
        mean, var = stats[l - 1]
        s = g / np.sqrt(var + BN_EPS)
        out.append((w * s[:, None, None, None], (b - mean) * s + be))
    out.append(convs[-1])
    return out


def cnn_forward(x, layers, emulate_bf16=False):
    """Inference forward of the 2.5D residual CNN with folded layers [(w, b)] on
    x [B,5,H,W]; returns the denoised centre slice [B,H,W] = centre - R(x).
    With emulate_bf16 the weights, the network input and every stored hidden
    activation are rounded to bfloat16 (the accumulations stay FP64)."""
    r = bf16 if emulate_bf16 else (lambda a: a)
    a = r(x)
    for l, (w, b) in enumerate(layers):
        z = conv3x3(a, r(w), b)
        if l < len(layers) - 1:
            a = r(np.maximum(z, 0.0))
        else:
            a = z
    return x[:, 2] - a[:, 0]


def denoise(v4, layers, orient, emulate_bf16=False):
    """Agent H_{orient,t} of Eq. (14) on a 4D volume [nt,nz,ny,nx]."""
    s4 = orient_slices(v4, orient)
    x = window5(s4)
    out = cnn_forward(x, layers, emulate_bf16)
    return np.ascontiguousarray(orient_volume(out.reshape(s4.shape), orient))


# ---- training (Sec. V): MSE on (noisy, clean) pairs, BatchNorm in training mode, Adam.


def bn_relu_forward(z, gamma, beta):
    """BatchNorm in training mode (batch statistics over (n, i, j), biased
    variance, eps = 1e-5) followed by ReLU on z [N,C,H,W].
    Returns (a, y, xhat, istd, mean, var) with y = gamma xhat + beta, a = max(y, 0)."""
    mean = z.mean(axis=(0, 2, 3))
    var = z.var(axis=(0, 2, 3))
    istd = 1.0 / np.sqrt(var + BN_EPS)
    xhat = (z - mean[None, :, None, None]) * istd[None, :, None, None]
    y = gamma[None, :, None, None] * xhat + beta[None, :, None, None]
    return np.maximum(y, 0.0), y, xhat, istd, mean, var


def bn_relu_backward(da, y, xhat, istd, gamma):
    """Gradients through ReLU and training-mode BatchNorm: from the gradient da
    of a = max(y, 0) to dz (the conv output), d gamma and d beta.  With
    dy = da [y > 0] and m the mean over (n, i, j):
        dz = istd (gamma dy - m(gamma dy) - xhat m(gamma dy xhat)),
        d gamma = sum dy xhat,  d beta = sum dy."""
    dy = da * (y > 0)
    dgamma, dbeta = (dy * xhat).sum(axis=(0, 2, 3)), dy.sum(axis=(0, 2, 3))
    dxh = dy * gamma[None, :, None, None]
    m1 = dxh.mean(axis=(0, 2, 3))[None, :, None, None]
    m2 = (dxh * xhat).mean(axis=(0, 2, 3))[None, :, None, None]
    return istd[None, :, None, None] * (dxh - m1 - xhat * m2), dgamma, dbeta



def train_forward(x, convs, bns, emulate_bf16=False):
    """Training forward; returns (out, cache).  Hidden layers: conv (+bias),
    BatchNorm with batch statistics (biased variance), ReLU.
    With emulate_bf16, the points where a BF16 implementation stores values are
    rounded to BF16: the network input, every conv weight, and every
    activation after ReLU; pre-BatchNorm outputs and the last layer's output
    stay unrounded (FP64 here)."""
    r = bf16 if emulate_bf16 else (lambda t: t)
    cache = {"a": [r(x)], "z": [], "xhat": [], "istd": [], "y": [], "stats": [], "emulate": emulate_bf16}
    a = r(x)
    L = len(convs)
    for l in range(L):
        w, b = convs[l]
        z = conv3x3(a, r(w), b)
        cache["z"].append(z)
        if l == 0:
            a = r(np.maximum(z, 0.0))
        elif l < L - 1:
            g, be = bns[l - 1]
            a, yv, xhat, istd, mean, var = bn_relu_forward(z, g, be)
            cache["xhat"].append(xhat)
            cache["istd"].append(istd)
            cache["y"].append(yv)
            cache["stats"].append((mean, var))
            a = r(a)
        else:
            a = z
        if l < L - 1:
            cache["a"].append(a)
    out = x[:, 2] - a[:, 0]
    return out, cache


def train_loss_grad(x, clean, convs, bns, emulate_bf16=False):
    """MSE loss mean((out - clean)^2) and its gradients w.r.t. every conv weight,
    conv bias and BatchNorm gamma/beta.  Returns (loss, gconvs, gbns, stats).
    With emulate_bf16, besides the forward's rounding (train_forward), the
    gradients that a BF16 implementation stores between layers are rounded:
    the input gradient of every layer below the last, and the pre-activation
    gradient dz of every layer below the last; the last layer's input
    gradient is formed with FP32 weights, the others with the rounded ones."""
    r = bf16 if emulate_bf16 else (lambda t: t)
    out, c = train_forward(x, convs, bns, emulate_bf16)
    L = len(convs)
    npx = out.size
    loss = float(np.mean((out - clean) ** 2))
    dout = 2.0 * (out - clean) / npx
    da = -dout[:, None]                       # d/dR of out = centre - R
    gconvs = [None] * L
    gbns = [None] * (L - 2)
    for l in range(L - 1, -1, -1):
        if l == L - 1:
            dz = da
        elif l == 0:
            dz = r(da * (c["z"][0] > 0))
        else:
            dz, dg, db = bn_relu_backward(da, c["y"][l - 1], c["xhat"][l - 1], c["istd"][l - 1], bns[l - 1][0])
            gbns[l - 1] = (dg, db)
            dz = r(dz)
        a_in = c["a"][l]
        gconvs[l] = (conv3x3_wgrad(dz, a_in), dz.sum(axis=(0, 2, 3)))
        if l > 0:
            w = convs[l][0] if l == L - 1 else r(convs[l][0])
            da = r(conv3x3_dgrad(dz, w))
    return loss, gconvs, gbns, c["stats"]


def adam_update(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; t counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
