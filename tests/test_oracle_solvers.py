"""Pins of the oracle's proximal agents and MACE loop (Sec. III, Eqs. (4)-(13),
Algorithm 1) against dense brute-force solves, identities and finite differences."""
import math

import numpy as np
import pytest

from paper_2008_01567_gb300 import synth


def _dense_A(oracle, sc, ang, shape):
    n = int(np.prod(shape))
    cols = []
    for i in range(n):
        e = np.zeros(n); e[i] = 1.0
        cols.append(oracle.project(e.reshape(shape), sc, ang).ravel())
    return np.stack(cols, axis=1)


def _tiny_problem(oracle, n=4, nt=1, seed=0):
    sc = synth.Scan(n=n, nt=nt, nu=7, nv=6, views=3)
    rng = np.random.default_rng(seed)
    y = rng.uniform(0.1, 1.0, (nt, sc.views, sc.nv, sc.nu))
    lam = oracle.weights(y, 50.0)
    return sc, y, lam


def test_cg_prox_equals_dense_solve(oracle):
    # With as many CG steps as unknowns, L~(v; z) equals the exact proximal map of
    # Eq. (4): (A^T Lambda A + I/sigma^2) z = A^T Lambda y + v/sigma^2.
    sc, y, lam = _tiny_problem(oracle)
    ang = sc.angles()[0]
    shape = (4, 4, 4)
    A = _dense_A(oracle, sc, ang, shape)
    sigma = 0.3
    v = synth.normal(1, shape)
    z0 = synth.normal(2, shape)
    H = A.T @ (lam[0].ravel()[:, None] * A) + np.eye(64) / sigma ** 2
    rhs = A.T @ (lam[0].ravel() * y[0].ravel()) + v.ravel() / sigma ** 2
    exact = np.linalg.solve(H, rhs)
    z = oracle.prox_data_frame(y[0], lam[0], v, z0, sc, ang, sigma, 64)
    np.testing.assert_allclose(z.ravel(), exact, rtol=1e-8, atol=1e-10)


def test_cg_energy_error_decreases(oracle):
    # CG minimises the H-norm of the error over growing Krylov spaces, so that
    # norm cannot increase from one iteration count to the next.
    sc, y, lam = _tiny_problem(oracle, seed=3)
    ang = sc.angles()[0]
    shape = (4, 4, 4)
    A = _dense_A(oracle, sc, ang, shape)
    sigma = 1.0
    v = synth.normal(4, shape)
    H = A.T @ (lam[0].ravel()[:, None] * A) + np.eye(64) / sigma ** 2
    exact = np.linalg.solve(H, A.T @ (lam[0].ravel() * y[0].ravel()) + v.ravel() / sigma ** 2)
    prev = math.inf
    for k in range(0, 12):
        e = oracle.prox_data_frame(y[0], lam[0], v, np.zeros(shape), sc, ang, sigma, k).ravel() - exact
        en = float(e @ H @ e)
        assert en <= prev * (1 + 1e-12)
        prev = en


def test_backproject_sq_is_squared_transpose(oracle):
    # (A.^2)^T y from the squared-weight scatter equals the dense columns squared
    sc, y, lam = _tiny_problem(oracle, seed=5)
    ang = sc.angles()[0]
    shape = (4, 4, 4)
    A = _dense_A(oracle, sc, ang, shape)
    got = oracle.backproject_sq(lam[0], sc, ang, shape).ravel()
    np.testing.assert_allclose(got, (A * A).T @ lam[0].ravel(), rtol=1e-12, atol=1e-14)


def _icd_sequential(A, lam, y, v, z0, sigma, order, sweeps):
    # textbook ICD on a dense system matrix: one voxel at a time, exact
    # minimisation of the quadratic cost of Eq. (4) along that coordinate
    z = z0.ravel().copy()
    e = y.ravel() - A @ z
    L = lam.ravel()
    for _ in range(sweeps):
        for s in order:
            a = A[:, s]
            t1 = -a @ (L * e) + (z[s] - v.ravel()[s]) / sigma ** 2
            t2 = a @ (L * a) + 1.0 / sigma ** 2
            d = -t1 / t2
            z[s] += d
            e -= a * d
    return z


def test_grouped_icd_with_single_voxel_groups_is_sequential_icd(oracle):
    sc, y, lam = _tiny_problem(oracle, seed=6)
    ang = sc.angles()[0]
    shape = (4, 4, 4)
    A = _dense_A(oracle, sc, ang, shape)
    sigma = 0.4
    v, z0 = synth.normal(7, shape), synth.normal(8, shape)
    order = list(np.random.default_rng(9).permutation(64))
    groups = []
    for s_ in order:
        m = np.zeros(64, bool); m[s_] = True
        groups.append(m.reshape(shape))
    got = oracle.prox_data_icd_frame(y[0], lam[0], v, z0, sc, ang, sigma, 2, groups)
    ref = _icd_sequential(A, lam[0], y[0], v, z0, sigma, order, 2)
    np.testing.assert_allclose(got.ravel(), ref, rtol=1e-10, atol=1e-12)


def test_grouped_icd_descends_and_converges_to_dense_solve(oracle):
    # parity groups: the cost of Eq. (4) never increases from sweep to sweep and
    # the iterates reach the exact proximal map
    sc, y, lam = _tiny_problem(oracle, seed=10)
    ang = sc.angles()[0]
    shape = (4, 4, 4)
    A = _dense_A(oracle, sc, ang, shape)
    sigma = 0.5
    v = synth.normal(11, shape)
    H = A.T @ (lam[0].ravel()[:, None] * A) + np.eye(64) / sigma ** 2
    exact = np.linalg.solve(H, A.T @ (lam[0].ravel() * y[0].ravel()) + v.ravel() / sigma ** 2)
    z = np.zeros(shape)
    prev = oracle.data_cost(y[0], lam[0], v, z, sc, ang, sigma)
    for _ in range(40):
        z = oracle.prox_data_icd_frame(y[0], lam[0], v, z, sc, ang, sigma, 1)
        c = oracle.data_cost(y[0], lam[0], v, z, sc, ang, sigma)
        assert c <= prev * (1 + 1e-12)
        prev = c
    z = oracle.prox_data_icd_frame(y[0], lam[0], v, z, sc, ang, sigma, 400)
    np.testing.assert_allclose(z.ravel(), exact, rtol=1e-7, atol=1e-9)


def test_parity_groups_partition_the_volume(oracle):
    g = oracle.parity_groups((3, 5, 4))
    assert len(g) == 8
    total = np.sum(g, axis=0)
    assert np.all(total == 1)
    # no two voxels of one group are neighbours along any axis
    for m in g:
        for ax in range(3):
            assert not np.any(m & np.roll(m, 1, axis=ax)[...] & (np.indices(m.shape)[ax] > 0))


def _gmrf_Q(shape4, sx, bt):
    # Hessian of h(z) = sum_{pairs} b rho(z_s - z_r) with p = q = 2, where
    # rho(D) = D^2/(4 sx^2): each pair adds b/(2 sx^2) [[1,-1],[-1,1]].
    nt, nz, ny, nx = shape4
    N = nt * nz * ny * nx
    Q = np.zeros((N, N))
    s = 6 + 12 / math.sqrt(2) + 8 / math.sqrt(3)
    idx = np.arange(N).reshape(shape4)
    for t in range(nt):
        for z in range(nz):
            for yy in range(ny):
                for x in range(nx):
                    i = idx[t, z, yy, x]
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                if (dz, dy, dx) == (0, 0, 0):
                                    continue
                                z2, y2, x2 = z + dz, yy + dy, x + dx
                                if not (0 <= z2 < nz and 0 <= y2 < ny and 0 <= x2 < nx):
                                    continue
                                b = 1.0 / (math.sqrt(abs(dz) + abs(dy) + abs(dx)) * s)
                                j = idx[t, z2, y2, x2]
                                c = b / (2 * sx ** 2) / 2  # each ordered pair visited twice
                                Q[i, i] += c; Q[j, j] += c; Q[i, j] -= c; Q[j, i] -= c
                    if t + 1 < nt:
                        j = idx[t + 1, z, yy, x]
                        c = bt / (2 * sx ** 2)
                        Q[i, i] += c; Q[j, j] += c; Q[i, j] -= c; Q[j, i] -= c
    return Q


def test_qggmrf_quadratic_case_equals_linear_solve(oracle):
    # p = q = 2 makes the q-GGMRF a Gaussian MRF: H(v) = (I/sigma^2 + Q)^-1 v/sigma^2.
    shape = (3, 3, 4, 3)
    v = synth.normal(5, shape)
    sigma, sx, bt = 0.7, 0.5, 0.5
    Q = _gmrf_Q(shape, sx, bt)
    exact = np.linalg.solve(np.eye(v.size) / sigma ** 2 + Q, v.ravel() / sigma ** 2)
    z = oracle.prox_qggmrf(v, np.zeros(shape), sigma, 2.0, 2.0, 1.0, sx, bt, 400)
    np.testing.assert_allclose(z.ravel(), exact, rtol=1e-9, atol=1e-11)
    # the cost function agrees with the quadratic form
    assert oracle.qggmrf_cost(z, 2.0, 2.0, 1.0, sx, bt) == pytest.approx(0.5 * z.ravel() @ Q @ z.ravel(), rel=1e-12)


def test_qggmrf_potential_and_surrogate(oracle):
    p, q, T, sx = 2.0, 1.2, 1.0, 0.3
    # rho ~ D^2/(2 sx^2) near 0 and ~ |D|^q (T sx)^(p-q)/(p sx^p) for large |D|
    d = 1e-6
    assert oracle.qggmrf_rho(d, p, q, T, sx) == pytest.approx(d * d / (2 * sx * sx), rel=1e-4)
    d = 1e6
    assert oracle.qggmrf_rho(d, p, q, T, sx) == pytest.approx(d ** q * (T * sx) ** (p - q) / (p * sx ** p), rel=1e-4)
    # a(D) = rho'(D) / (2 D), with rho' from central differences
    for d in (-2.0, -0.3, 0.01, 0.2, 1.7):
        h = 1e-6 * max(1.0, abs(d))
        drho = (oracle.qggmrf_rho(d + h, p, q, T, sx) - oracle.qggmrf_rho(d - h, p, q, T, sx)) / (2 * h)
        assert oracle.qggmrf_coef(d, p, q, T, sx) == pytest.approx(drho / (2 * d), rel=1e-6)
    assert oracle.qggmrf_coef(0.0, p, q, T, sx) == pytest.approx(1.0 / (2 * sx * sx), rel=1e-15)


def test_qggmrf_icd_reaches_stationary_point(oracle):
    # Converged ICD satisfies the first-order condition of Eq. (5):
    # (z - v)/sigma^2 + grad h(z) = 0, with grad h from differences of the cost.
    shape = (2, 3, 3, 3)
    v = synth.uniform(6, shape, 0.0, 2.0)
    sigma, p, q, T, sx, bt = 0.5, 2.0, 1.2, 1.0, 0.4, 0.5
    z = oracle.prox_qggmrf(v, v.copy(), sigma, p, q, T, sx, bt, 3000)
    g = np.zeros(z.size)
    zf = z.ravel()
    for i in range(z.size):
        h = 1e-6
        zp = zf.copy(); zp[i] += h
        zm = zf.copy(); zm[i] -= h
        g[i] = (oracle.qggmrf_cost(zp.reshape(shape), p, q, T, sx, bt)
                - oracle.qggmrf_cost(zm.reshape(shape), p, q, T, sx, bt)) / (2 * h)
    kkt = (zf - v.ravel()) / sigma ** 2 + g
    assert np.abs(kkt).max() < 1e-6 * np.abs(v.ravel() / sigma ** 2).max()


def test_qggmrf_icd_is_monotone(oracle):
    # Each ICD update minimises a majoriser of the prox cost, so the cost never rises.
    shape = (3, 4, 4, 4)
    v = synth.uniform(7, shape, 0.0, 2.0)
    sigma, p, q, T, sx, bt = 0.2, 2.0, 1.2, 1.0, 0.1, 0.5
    z = np.zeros(shape)
    cost = lambda z: float(((z - v) ** 2).sum() / (2 * sigma ** 2)) + oracle.qggmrf_cost(z, p, q, T, sx, bt)
    prev = cost(z)
    for _ in range(6):
        z = oracle.prox_qggmrf(v, z, sigma, p, q, T, sx, bt, 1)
        c = cost(z)
        assert c <= prev + 1e-12
        prev = c


def test_G_involution_and_mann_forms(oracle):
    # (2G - I)(2G - I) = I (Sec. III) and Algorithm 1 equals the Mann update of Eq. (12).
    rng = np.random.default_rng(8)
    K = 3
    mu = oracle.mu_from_beta(3.0, K)
    assert mu.sum() == pytest.approx(1.0) and np.allclose(mu, 0.25)
    W = [rng.standard_normal((2, 3, 4)) for _ in range(K + 1)]
    V = [2 * g - w for g, w in zip(oracle.G(W, mu), W)]
    VV = [2 * g - v for g, v in zip(oracle.G(V, mu), V)]
    for a, b in zip(VV, W):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13)
    mats = [rng.standard_normal((24, 24)) * 0.3 for _ in range(K + 1)]
    agents = [lambda w, x, M=M: (M @ w.ravel()).reshape(w.shape) for M in mats]
    X = [np.zeros_like(w) for w in W]
    rho = 0.8
    W1, X1, _ = oracle.mace_iteration(W, X, agents, mu, rho)
    W2 = oracle.mann_step_direct(W, [a(w, None) for a, w in zip(agents, W)], mu, rho)
    for a, b in zip(W1, W2):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_mace_fixed_point_is_map_solution(oracle):
    # With proximal agents, the consensus solves Eq. (3):
    # (A^T Lambda A + (beta/K) sum_k Q_k) x = A^T Lambda y.  Agents here: the
    # oracle's CG prox (run to convergence) and two quadratic-MRF ICD proxes.
    n, nt = 4, 2
    sc, y, lam = _tiny_problem(oracle, n=n, nt=nt, seed=9)
    shape4 = (nt, n, n, n)
    sigma, beta, K = 0.5, 1.0, 2
    mu = oracle.mu_from_beta(beta, K)
    prm = [(0.6, 0.5), (0.3, 1.0)]  # (sigma_x, b_temporal) of the two priors
    agents = [lambda w, x: oracle.prox_data(y, lam, w, x, sc, sigma, 64)]
    for sx, bt in prm:
        agents.append(lambda w, x, sx=sx, bt=bt: oracle.prox_qggmrf(w, x, sigma, 2.0, 2.0, 1.0, sx, bt, 300))
    x0 = np.zeros(shape4)
    xhat, W, X, res = oracle.mace(x0, agents, mu, 0.5, 150)
    ang = sc.angles()
    N3 = n ** 3
    H = np.zeros((nt * N3, nt * N3))
    b = np.zeros(nt * N3)
    for t in range(nt):
        A = _dense_A(oracle, sc, ang[t], (n, n, n))
        H[t * N3:(t + 1) * N3, t * N3:(t + 1) * N3] = A.T @ (lam[t].ravel()[:, None] * A)
        b[t * N3:(t + 1) * N3] = A.T @ (lam[t].ravel() * y[t].ravel())
    for sx, bt in prm:
        H += beta / K * _gmrf_Q(shape4, sx, bt)
    exact = np.linalg.solve(H, b)
    np.testing.assert_allclose(xhat.ravel(), exact, rtol=1e-7, atol=1e-9 * np.abs(exact).max())
    np.testing.assert_allclose(oracle.average(X, mu).ravel(), exact, rtol=1e-7, atol=1e-9 * np.abs(exact).max())
    assert res[-1] < 1e-7 < res[0]


def test_consensus_residual_closed_forms(oracle):
    # Sec. III stopping quantity r = sqrt(sum_i mu_i ||X_i - Xbar||^2) / ||Xbar||.
    # Two agents, equal weights, constant fields a and b: Xbar = (a + b) / 2 and
    # each deviation is |a - b| / 2, so r = |a - b| / |a + b|.
    shape = (2, 3, 4, 5)
    a, b = 1.25, 0.5
    r = oracle.consensus_residual([np.full(shape, a), np.full(shape, b)], [0.5, 0.5])
    assert r == pytest.approx(abs(a - b) / abs(a + b), rel=1e-14)
    # agreeing agents: zero up to the rounding of Xbar; the residual does not
    # change with the overall scale
    x = synth.uniform(91, shape, 0.5, 1.5)
    assert oracle.consensus_residual([x, x, x], [0.2, 0.3, 0.5]) <= 1e-15
    y = synth.uniform(92, shape, 0.5, 1.5)
    mu = [0.25, 0.75]
    r1 = oracle.consensus_residual([x, y], mu)
    assert oracle.consensus_residual([7.0 * x, 7.0 * y], mu) == pytest.approx(r1, rel=1e-13)
    # unequal weights, worked by hand on scalars 1 and 0 with mu = (1/4, 3/4):
    # Xbar = 1/4, deviations 3/4 and 1/4, r = sqrt(1/4 * 9/16 + 3/4 * 1/16) / (1/4) = sqrt(3)
    r2 = oracle.consensus_residual([np.ones(1), np.zeros(1)], mu)
    assert r2 == pytest.approx(math.sqrt(3.0), rel=1e-14)


# ---------------------------------------------------------------- direct MAP (MBIR + 4D-MRF, Sec. VI)


def _dense_system(oracle, sc, y, lam, n, nt):
    ang = sc.angles()
    N3 = n ** 3
    H = np.zeros((nt * N3, nt * N3))
    b = np.zeros(nt * N3)
    for t in range(nt):
        A = _dense_A(oracle, sc, ang[t], (n, n, n))
        H[t * N3:(t + 1) * N3, t * N3:(t + 1) * N3] = A.T @ (lam[t].ravel()[:, None] * A)
        b[t * N3:(t + 1) * N3] = A.T @ (lam[t].ravel() * y[t].ravel())
    return H, b


def test_map_quadratic_prior_equals_dense_solve(oracle):
    # p = q = 2: the surrogate equals the prior, so one outer iteration with as
    # many CG steps as unknowns solves (A^T Lambda A + beta Q) x = A^T Lambda y
    n, nt = 4, 2
    sc, y, lam = _tiny_problem(oracle, n=n, nt=nt, seed=12)
    sx, bt, beta = 0.4, 0.5, 2.0
    H, b = _dense_system(oracle, sc, y, lam, n, nt)
    exact = np.linalg.solve(H + beta * _gmrf_Q((nt, n, n, n), sx, bt), b)
    x = oracle.map_mm(y, lam, np.zeros((nt, n, n, n)), sc, 2.0, 2.0, 1.0, sx, bt, beta, 1, nt * n ** 3)
    np.testing.assert_allclose(x.ravel(), exact, rtol=1e-8, atol=1e-10 * np.abs(exact).max())


def test_surrogate_lap_is_half_the_surrogate_gradient(oracle):
    # 2 L_a x is the gradient of Q(x) = sum_pairs b a(anchor) (x_s - x_r)^2, and
    # at x = anchor it equals the gradient of h itself (the surrogate touches h
    # there): both against central finite differences of the oracle's h
    shape = (2, 3, 4, 3)
    p, q, T, sx, bt = 2.0, 1.2, 1.0, 0.3, 0.5
    anchor = synth.uniform(13, shape)
    g = 2.0 * oracle.surrogate_lap(anchor, anchor, p, q, T, sx, bt)
    fd = np.zeros(anchor.size)
    h = 1e-6
    for i in range(anchor.size):
        e = np.zeros(anchor.size); e[i] = h
        fd[i] = (oracle.qggmrf_cost(anchor + e.reshape(shape), p, q, T, sx, bt) -
                 oracle.qggmrf_cost(anchor - e.reshape(shape), p, q, T, sx, bt)) / (2 * h)
    np.testing.assert_allclose(g.ravel(), fd, rtol=1e-6, atol=1e-8)
    # L_a is linear in x
    x1, x2 = synth.normal(14, shape), synth.normal(15, shape)
    np.testing.assert_allclose(oracle.surrogate_lap(anchor, 2 * x1 - x2, p, q, T, sx, bt),
                               2 * oracle.surrogate_lap(anchor, x1, p, q, T, sx, bt)
                               - oracle.surrogate_lap(anchor, x2, p, q, T, sx, bt), rtol=1e-12, atol=1e-12)


def test_map_descends_and_reaches_a_stationary_point(oracle):
    n, nt = 4, 2
    sc, y, lam = _tiny_problem(oracle, n=n, nt=nt, seed=16)
    p, q, T, sx, bt, beta = 2.0, 1.2, 1.0, 0.3, 0.5, 3.0
    x = np.zeros((nt, n, n, n))
    prev = oracle.map_cost(y, lam, x, sc, p, q, T, sx, bt, beta)
    for _ in range(15):
        x = oracle.map_mm(y, lam, x, sc, p, q, T, sx, bt, beta, 1, 4)
        c = oracle.map_cost(y, lam, x, sc, p, q, T, sx, bt, beta)
        assert c <= prev * (1 + 1e-12)
        prev = c
    x = oracle.map_mm(y, lam, x, sc, p, q, T, sx, bt, beta, 200, 30)
    # gradient of Phi by central differences of the cost
    fd = np.zeros(x.size)
    h = 1e-6
    for i in range(x.size):
        e = np.zeros(x.size); e[i] = h
        fd[i] = (oracle.map_cost(y, lam, x + e.reshape(x.shape), sc, p, q, T, sx, bt, beta) -
                 oracle.map_cost(y, lam, x - e.reshape(x.shape), sc, p, q, T, sx, bt, beta)) / (2 * h)
    H, b = _dense_system(oracle, sc, y, lam, n, nt)
    assert np.linalg.norm(fd) <= 1e-6 * np.linalg.norm(b)


def test_mace_with_exact_agents_reaches_the_map_point(oracle):
    # Sec. III: with proximal agents the consensus equilibrium is the MAP point
    # of l + (mu_1/mu_0) h; here the non-quadratic q-GGMRF prior (q = 1.2)
    n, nt = 4, 2
    sc, y, lam = _tiny_problem(oracle, n=n, nt=nt, seed=17)
    p, q, T, sx, bt = 2.0, 1.2, 1.0, 0.3, 0.5
    mu, sigma = [0.25, 0.75], 0.5
    agents = [lambda w, x: oracle.prox_data(y, lam, w, x, sc, sigma, 64),
              lambda w, x: oracle.prox_qggmrf(w, x, sigma, p, q, T, sx, bt, 200)]
    xhat, W, X, res = oracle.mace(np.zeros((nt, n, n, n)), agents, mu, 0.5, 200)
    xmap = oracle.map_mm(y, lam, np.zeros((nt, n, n, n)), sc, p, q, T, sx, bt, mu[1] / mu[0], 300, 30)
    np.testing.assert_allclose(oracle.average(X, mu), xmap, rtol=1e-6, atol=1e-8 * np.abs(xmap).max())


# ---------------------------------------------------------------- blind fixture correction (Appendix A)


def test_blur_taps_and_impulse_response(oracle):
    g = oracle.gaussian_taps(1.7)
    assert g.sum() == pytest.approx(1.0, abs=1e-15) and len(g) == 2 * 6 + 1
    np.testing.assert_allclose(g, g[::-1])
    # an interior impulse spreads into the outer product of the taps
    e = np.zeros((1, 1, 31, 37))
    e[0, 0, 15, 18] = 1.0
    b = oracle.blur_sinogram(e, 1.7)
    np.testing.assert_allclose(b[0, 0, 15 - 6:15 + 7, 18 - 6:18 + 7], np.outer(g, g), rtol=1e-14, atol=1e-17)
    assert b.sum() == pytest.approx(1.0, rel=1e-14)
    # a constant field keeps its value away from the detector edges
    c = oracle.blur_sinogram(np.full((2, 1, 30, 40), 2.5), 2.0)
    np.testing.assert_allclose(c[:, :, 6:-6, 6:-6], 2.5, rtol=1e-14)
    assert c[0, 0, 0, 0] < 2.5


def test_fixture_correction_least_squares_and_recovery(oracle):
    sc = synth.Scan(n=16, nt=2, nu=28, nv=24, views=5)
    ell = synth.ellipsoids(21, 2, sc, axis_range=(0.08, 0.15))
    ell[:, :, 0:2] *= 0.4                      # keep the object well inside the mask
    x = oracle.ellipsoid_volume(ell, sc, ss=2)
    y_obj = oracle.project4d(x, sc)
    # no fixture and an exact reconstruction: nothing to correct
    yc, c = oracle.fixture_correct(y_obj, x, sc, 0.45, 2.0)
    assert abs(c) < 1e-12
    np.testing.assert_allclose(yc, y_obj, atol=1e-12)
    # a smooth fixture shadow (a broad bump drifting across the views) is removed
    vv, uu = np.meshgrid(np.arange(sc.nv), np.arange(sc.nu), indexing="ij")
    f = np.zeros_like(y_obj)
    for t in range(sc.nt):
        for j in range(sc.views):
            f[t, j] = 0.6 * np.exp(-((uu - 4 - 3 * j) ** 2) / 40.0 - ((vv - 12) ** 2) / 200.0)
    y = y_obj + f
    yc, c = oracle.fixture_correct(y, x, sc, 0.45, 2.0)
    assert np.linalg.norm(yc - y_obj) < 0.1 * np.linalg.norm(f)
    assert 0.8 < c < 1.25
    # c minimises ||e - c p||^2
    m = oracle.cylinder_mask(x.shape[1:], sc.vox, 0.45)
    e = y - oracle.project4d(x * m[None], sc)
    p = oracle.blur_sinogram(e, 2.0)
    r = lambda cc: float(np.sum((e - cc * p) ** 2))
    assert r(c) <= min(r(c + 1e-3), r(c - 1e-3))


def test_cylinder_mask(oracle):
    m = oracle.cylinder_mask((3, 8, 8), 1.0 / 8, 0.3)
    assert m.shape == (3, 8, 8) and set(np.unique(m)) <= {0.0, 1.0}
    assert m[0, 3, 3] == 1.0 and m[0, 0, 0] == 0.0
    np.testing.assert_array_equal(m, m[:, ::-1, :])
    np.testing.assert_array_equal(m[0], m[0].T)
