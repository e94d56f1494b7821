"""The stored fixtures of tests/golden/ (written by tests/golden/make_golden.py,
which calls only the oracle and the seeded generators).

CPU: the oracle as it stands reproduces every fixture (a change to its
arithmetic shows up here and has to be justified), and the stored values obey
what the paper and the mathematics fix independently of the oracle: the
hand-worked weights of Eq. (9), the adjoint identity <A x, e> = <x, A^T e> of
Eq. (2), descent of the prox objective of Eq. (4) under the CG partial update
of Eq. (13), the prox optimality bounds of Eq. (5), and the averaging of the
consensus state in Algorithm 1.

GPU: the CUDA path reproduces the stored projections and the stored Mann
residuals through the C ABI, at the tolerances stated for the projector
(1e-5 relative L2) and for three plain MACE iterations (1e-3 relative)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2008_01567_gb300 import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLD, name + ".json")) as f:
        return json.load(f)


def _scan(d):
    return synth.Scan(n=d["n"], nt=d["nt"], nu=d["nu"], nv=d["nv"], views=d["views"], mode=d["mode"])


def _a(v, shape=None):
    a = np.asarray(v, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def gen():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLD, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    oracle.build()
    return mod


# ---------------------------------------------------------------- CPU pins --

@pytest.mark.parametrize("name", ["mu_weights", "joseph_8cube", "cg_prox_6cube", "qggmrf_prox",
                                  "mace_plain_tiny"])
def test_oracle_reproduces_fixture(gen, name):
    stored = _load(name)
    fresh = json.loads(json.dumps(gen.FIXTURES[name]()))
    assert stored.keys() == fresh.keys()
    assert stored["cite"]
    for k, v in stored.items():
        if isinstance(v, list) and v and isinstance(v[0], float):
            np.testing.assert_allclose(fresh[k], v, rtol=1e-12, atol=1e-12, err_msg=k)
        elif k == "cases":
            for a, b in zip(v, fresh[k]):
                np.testing.assert_allclose(a["mu"], b["mu"], rtol=1e-15)
        else:
            assert fresh[k] == v, k


def test_mu_weights_hand_worked():
    # Eq. (9) worked by hand: beta = 1 balances forward and prior models.
    cases = {(c["beta"], c["K"]): c["mu"] for c in _load("mu_weights")["cases"]}
    np.testing.assert_allclose(cases[(1.0, 1)], [0.5, 0.5], rtol=1e-15)
    np.testing.assert_allclose(cases[(1.0, 3)], [0.5, 1 / 6, 1 / 6, 1 / 6], rtol=1e-15)
    np.testing.assert_allclose(cases[(3.0, 3)], [0.25, 0.25, 0.25, 0.25], rtol=1e-15)


def test_joseph_fixture_adjoint_identity():
    g = _load("joseph_8cube")
    sc = _scan(g["scan"])
    x = _a(g["x"])
    e = _a(g["e"])
    lhs, rhs = float(np.dot(_a(g["Ax"]), e)), float(np.dot(x, _a(g["ATe"])))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))
    assert len(g["Ax"]) == sc.nt * sc.views * sc.nv * sc.nu
    # a nonnegative volume has nonnegative line integrals, and some rays hit it
    assert min(g["Ax"]) >= 0.0 and max(g["Ax"]) > 0.0


def test_cg_fixture_descends_the_prox_objective():
    g = _load("cg_prox_6cube")
    sc = _scan(g["scan"])
    counts = _a(g["counts"], (sc.nt, sc.views, sc.nv, sc.nu))
    y = _f32(oracle.log_measurement(counts, g["I0"]))
    lam = _f32(oracle.weights(y, g["I0"]))
    shp = (sc.nt, sc.n, sc.n, sc.n)
    v, z0, z = _a(g["v"], shp), _a(g["z0"], shp), _a(g["z"], shp)

    def objective(x):        # Eq. (4): (1/2)||y - A x||^2_Lambda + ||x - v||^2 / (2 sigma^2)
        r = y - oracle.project4d(x, sc)
        return 0.5 * float(np.sum(lam * r * r)) + float(np.sum((x - v) ** 2)) / (2 * g["sigma"] ** 2)

    assert objective(z) < objective(z0)
    assert objective(z) < objective(v)


def test_qggmrf_fixture_within_range():
    # The q-GGMRF potential is even and increasing in |difference|: the prox of
    # Eq. (5) stays inside [min v, max v] and moves every voxel towards its
    # neighbours, so the result is smoother than v.
    g = _load("qggmrf_prox")
    v, z = _a(g["v"], g["shape"]), _a(g["z"], g["shape"])
    assert v.min() - 1e-12 <= z.min() and z.max() <= v.max() + 1e-12
    tv = lambda a: float(sum(np.abs(np.diff(a, axis=d)).sum() for d in range(4)))
    assert tv(z) < tv(v)


def test_mace_fixture_residuals_and_average():
    g = _load("mace_plain_tiny")
    res = g["residuals"]
    assert len(res) == g["iters"] and all(r > 0 for r in res)
    assert res[-1] < res[0]
    sc = _scan(g["scan"])
    assert len(g["X0"]) == sc.nt * sc.n ** 3
    assert sum(g["mu"]) == pytest.approx(1.0, abs=1e-15)


# ------------------------------------------------------------ GPU against it --

@pytest.fixture(scope="module")
def M():
    import torch
    from paper_2008_01567_gb300 import build, msf
    build.build()
    assert torch.cuda.is_available()
    return msf


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.gpu
def test_gpu_projector_matches_fixture(M):
    import torch
    g = _load("joseph_8cube")
    sc = _scan(g["scan"])
    P = M.Projector(sc)
    y = torch.empty((sc.nt, sc.views, sc.nv, sc.nu), device="cuda")
    M.msf_project(P, _t(_a(g["x"], (sc.nt, sc.n, sc.n, sc.n))), y)
    x = torch.empty((sc.nt, sc.n, sc.n, sc.n), device="cuda")
    M.msf_backproject(P, _t(_a(g["e"], (sc.nt, sc.views, sc.nv, sc.nu))), x)
    torch.cuda.synchronize()
    assert _rel(y.cpu().numpy().ravel(), _a(g["Ax"])) <= 1e-5
    assert _rel(x.cpu().numpy().ravel(), _a(g["ATe"])) <= 1e-5


@pytest.mark.gpu
def test_gpu_plain_mace_matches_fixture(M):
    import torch
    g = _load("mace_plain_tiny")
    sc = _scan(g["scan"])
    P = M.Projector(sc)
    c = _t(_a(g["counts"], (sc.nt, sc.views, sc.nv, sc.nu)))
    yg, lg = torch.empty_like(c), torch.empty_like(c)
    M.msf_weights(c, yg, lg, g["I0"], g["I0"])
    shape = (2, sc.nt, sc.n, sc.n, sc.n)
    W = torch.zeros(shape, device="cuda")
    X = torch.zeros(shape, device="cuda")
    m = g["mrf"]
    mace = M.Mace(P, W, X, yg, lg, M.MSF_PRIOR_QGGMRF, mrf=M.msf_mrf(m["p"], m["q"], m["T"], m["sx"], m["bt"]))
    res = [M.msf_mace_step(mace, g["rho"], g["sigma"], g["mu"], g["n_cg"], g["n_sweeps"])
           for _ in range(g["iters"])]
    np.testing.assert_allclose(res, g["residuals"], rtol=1e-3)
    assert _rel(X[0].cpu().numpy().ravel(), _a(g["X0"])) <= 1e-3
