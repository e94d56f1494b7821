"""Pins of the oracle's cone-beam Joseph projector A_n (Sec. II, Eq. (2)) and of the
analytic phantom projector, against closed forms, invariants and brute force."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2008_01567_gb300 import synth


def _scan(n, nu, nv, views=1, **kw):
    return synth.Scan(n=n, nt=1, nu=nu, nv=nv, views=views, **kw)


def test_central_ray_is_column_sum(oracle):
    # Odd grid and odd detector at th = 0: the central ray runs along -x through
    # y = z = 0, hits every plane at a voxel centre, so A x = vox * sum_ix x.
    sc = _scan(9, 11, 11)
    x = synth.uniform(1, (9, 9, 9))
    y = oracle.project(x, sc, np.array([0.0]))
    assert y[0, 5, 5] == pytest.approx(sc.vox * x[4, 4, :].sum(), rel=1e-13)
    # th = pi/2: the source sits on +y and the central ray runs along -y.
    y = oracle.project(x, sc, np.array([math.pi / 2]))
    assert y[0, 5, 5] == pytest.approx(sc.vox * x[4, :, 4].sum(), rel=1e-13)


def _ray(sc, th, iu, iv):
    # The documented scanner: source (dso cos, dso sin, 0); detector centre
    # -(dsd-dso)(cos, sin, 0); u axis (-sin, cos, 0); v axis (0,0,1).
    c, s = math.cos(th), math.sin(th)
    u = (iu - 0.5 * (sc.nu - 1)) * sc.pitch
    v = (iv - 0.5 * (sc.nv - 1)) * sc.pitch
    src = np.array([sc.dso * c, sc.dso * s, 0.0])
    pix = np.array([-(sc.dsd - sc.dso) * c - u * s, -(sc.dsd - sc.dso) * s + u * c, v])
    return src, pix - src


def test_affine_volume_gives_exact_midpoint_rule(oracle):
    # Bilinear interpolation reproduces an affine function exactly.  For a ray
    # whose crossing points stay inside the volume at every plane, Joseph's sum
    # is step * sum_k f(P_k) over N equally spaced points, i.e. (chord through
    # the slab of planes) * f(midpoint) for affine f: a closed form.
    n = 16
    sc = _scan(n, 21, 21)
    coord = (np.arange(n) - 0.5 * (n - 1)) * sc.vox
    zz, yy, xx = np.meshgrid(coord, coord, coord, indexing="ij")
    a, b, c, d = 0.7, 0.3, -0.45, 0.2
    x = a + b * xx + c * yy + d * zz
    for th in (0.1, 0.3, math.pi / 2 + 0.2):
        y = oracle.project(x, sc, np.array([th]))
        for iu, iv in ((10, 10), (9, 11), (11, 8)):
            src, dvec = _ray(sc, th, iu, iv)
            k = 0 if abs(dvec[0]) >= abs(dvec[1]) else 1
            # slab of the N planes along the major axis: centres from -W/2+vox/2
            # to W/2-vox/2; N steps of vox along the major axis
            lam_mid = (0.0 - src[k]) / dvec[k]
            pm = src + lam_mid * dvec
            # the minor coordinates must stay within the grid at every plane
            for pc in coord:
                lam = (pc - src[k]) / dvec[k]
                p = src + lam * dvec
                assert abs(p[1 - k]) < coord[-1] and abs(p[2]) < coord[-1]
            step = sc.vox * np.linalg.norm(dvec) / abs(dvec[k])
            expected = n * step * (a + b * pm[0] + c * pm[1] + d * pm[2])
            assert y[0, iv, iu] == pytest.approx(expected, rel=1e-12)


def test_quarter_turn_equivariance(oracle):
    # Turning the scanner by +90 deg equals turning the object by -90 deg:
    # A(th + pi/2) f == A(th) g with g[z, a, b] = f[z, b, n-1-a].
    n = 12
    sc = _scan(n, 17, 13, views=3)
    f = synth.uniform(2, (n, n, n))
    g = np.ascontiguousarray(np.flip(f, axis=2).transpose(0, 2, 1))
    th = np.array([0.13, 1.1, 2.9])
    y1 = oracle.project(f, sc, th + math.pi / 2)
    y2 = oracle.project(g, sc, th)
    np.testing.assert_allclose(y1, y2, rtol=1e-11, atol=1e-13)


def test_adjoint_identity(oracle):
    sc = _scan(10, 14, 12, views=5)
    ang = np.linspace(0.05, 6.0, 5)
    x = synth.normal(3, (10, 10, 10))
    y = synth.normal(4, (5, 12, 14))
    lhs = np.vdot(oracle.project(x, sc, ang), y)
    rhs = np.vdot(x, oracle.backproject(y, sc, ang))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_adjoint_is_transpose_brute_force(oracle):
    # Dense A column by column vs dense A^T row by row on a tiny problem.
    sc = _scan(4, 6, 5, views=2)
    ang = np.array([0.4, 2.0])
    cols = []
    for i in range(64):
        e = np.zeros(64); e[i] = 1.0
        cols.append(oracle.project(e.reshape(4, 4, 4), sc, ang).ravel())
    A = np.stack(cols, axis=1)
    rows = []
    for j in range(A.shape[0]):
        e = np.zeros(A.shape[0]); e[j] = 1.0
        rows.append(oracle.backproject(e.reshape(2, 5, 6), sc, ang, (4, 4, 4)).ravel())
    At = np.stack(rows, axis=0)
    np.testing.assert_allclose(At, A, rtol=0, atol=1e-15)
    assert (A >= 0).all() and A.sum() > 0


def test_sphere_chord_and_magnification(oracle):
    # A sphere of radius r: the ray through its centre has chord 2r (closed form);
    # at th = 0 a sphere at (0, y0, 0) projects to u = y0 * dsd / dso.
    sc = _scan(8, 41, 41)
    r, mu = 0.1, 1.5
    ell = np.zeros((1, 1, 16))
    ell[0, 0, 3:6] = r
    ell[0, 0, 6:15] = np.eye(3).ravel()
    ell[0, 0, 15] = mu
    s1 = dataclasses.replace(sc, views=1)
    y = oracle.ellipsoid_sinogram(ell, s1)  # angles() of sparse360 with 1 view = [0]
    assert y[0, 0, 20, 20] == pytest.approx(2 * r * mu, rel=1e-12)
    y0 = 0.15
    ell[0, 0, 1] = y0
    y = oracle.ellipsoid_sinogram(ell, s1)[0, 0]
    u = (np.arange(sc.nu) - 0.5 * (sc.nu - 1)) * sc.pitch
    prof = y.sum(axis=0)
    # a sphere's silhouette centre: the tangent cone is symmetric about the
    # source-centre line, whose detector hit is y0 * dsd/dso
    peak_u = u[np.argmax(prof)]
    assert abs(peak_u - y0 * sc.dsd / sc.dso) <= sc.pitch


def test_joseph_converges_to_analytic_chords(oracle):
    # Joseph projection of the voxelised phantom approaches the exact line
    # integrals as the grid is refined.
    errs = []
    for n in (16, 32, 64):
        sc = synth.Scan(n=n, nt=1, nu=48, nv=40, views=4)
        ell = synth.ellipsoids(7, 3, sc)
        exact = oracle.ellipsoid_sinogram(ell, sc)
        vol = oracle.ellipsoid_volume(ell, sc, ss=4)
        approx = oracle.project4d(vol, sc)
        errs.append(np.linalg.norm(approx - exact) / np.linalg.norm(exact))
    # a discontinuous object sampled on a grid of spacing h converges in L2 like
    # h^(1/2): each halving of h must cut the error by well over a quarter
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1]
    assert errs[2] < 0.06


def test_voxelizer_volume(oracle):
    # Sum of voxel values * vox^3 approaches mu * (4/3) pi abc.
    sc = synth.Scan(n=48, nt=1, nu=8, nv=8, views=1)
    ell = synth.ellipsoids(11, 1, sc)
    vol = oracle.ellipsoid_volume(ell, sc, ss=4)
    e = ell[0, 0]
    exact = e[15] * 4.0 / 3.0 * math.pi * e[3] * e[4] * e[5]
    assert vol.sum() * sc.vox ** 3 == pytest.approx(exact, rel=0.02)


def test_measurement_model(oracle):
    # y = -ln(max(n,1)/I0) and Lambda = c exp(-y) (Sec. II); Poisson counts have
    # mean and variance I0 exp(-p).
    p = np.full(200000, 1.3)
    counts = synth.poisson(5, oracle.expected_counts(p, 1e4))
    m = 1e4 * math.exp(-1.3)
    assert counts.mean() == pytest.approx(m, rel=2e-3)
    assert counts.var() == pytest.approx(m, rel=2e-2)
    y = oracle.log_measurement(np.array([0.0, 1.0, 1e4]), 1e4)
    np.testing.assert_allclose(y, [math.log(1e4), math.log(1e4), 0.0])
    np.testing.assert_allclose(oracle.weights(y, 1e4), [1.0, 1.0, 1e4])
