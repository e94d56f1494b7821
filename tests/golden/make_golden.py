"""Writes the small expected-value fixtures of tests/golden/ from the FP64
oracle alone (plus the seeded input generators of synth).  Each fixture keeps
its inputs, its expected outputs and the passage of the paper it follows.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2008_01567_gb300 import synth  # noqa: E402

I0 = 1e4


def _scan(d):
    return synth.Scan(n=d["n"], nt=d["nt"], nu=d["nu"], nv=d["nv"], views=d["views"], mode=d["mode"])


def _lst(a):
    return [float(v) for v in np.asarray(a, dtype=np.float64).ravel()]


def mu_weights():
    rows = [{"beta": b, "K": k, "mu": _lst(oracle.mu_from_beta(b, k))} for b, k in ((1.0, 1), (1.0, 3), (3.0, 3))]
    return {"cite": "Sec. III, Eq. (9): agent weights mu_0 = 1/(1+beta), mu_k = beta/((1+beta)K)", "cases": rows}


def joseph_8cube():
    sd = dict(n=8, nt=1, nu=10, nv=9, views=3, mode="sparse360")
    sc = _scan(sd)
    x = synth.uniform(701, (sc.nt, sc.n, sc.n, sc.n), 0.0, 2.0)
    e = synth.normal(702, (sc.nt, sc.views, sc.nv, sc.nu))
    return {"cite": "Sec. II, Eq. (2): the system matrix A_n, modelled as a Joseph ray-driven projector; "
                    "its transpose A_n^T",
            "scan": sd, "x": _lst(x), "e": _lst(e),
            "Ax": _lst(oracle.project4d(x, sc)), "ATe": _lst(oracle.backproject4d(e, sc))}


def _measure(sd, seed):
    sc = _scan(sd)
    ell = synth.ellipsoids(seed, 2, sc)
    p = oracle.ellipsoid_sinogram(ell, sc)
    counts = synth.poisson(seed + 1, oracle.expected_counts(p, I0))
    y = oracle.log_measurement(counts, I0)
    return sc, counts, y, oracle.weights(y, I0)


def cg_prox_6cube():
    sd = dict(n=6, nt=1, nu=8, nv=8, views=4, mode="sparse360")
    sc, counts, y, lam = _measure(sd, 711)
    y32 = np.asarray(y, np.float32).astype(np.float64)
    lam32 = np.asarray(lam, np.float32).astype(np.float64)
    v = synth.uniform(713, (1, 6, 6, 6), 0.0, 1.5)
    z0 = synth.uniform(714, (1, 6, 6, 6), 0.0, 1.5)
    sigma, n_cg = 0.2, 4
    return {"cite": "Sec. III, Eqs. (4) and (13): the data proximal map, here n_cg warm-started CG "
                    "iterations on (A^T Lambda A + I/sigma^2) z = A^T Lambda y + v/sigma^2",
            "scan": sd, "I0": I0, "counts": _lst(counts), "v": _lst(v), "z0": _lst(z0), "sigma": sigma,
            "n_cg": n_cg, "z": _lst(oracle.prox_data(y32, lam32, v, z0, sc, sigma, n_cg))}


def qggmrf_prox():
    shape = (2, 4, 4, 4)
    v = synth.uniform(721, shape, 0.0, 1.0)
    prm = dict(p=2.0, q=1.2, T=1.0, sx=0.1, bt=0.5)
    sigma, sweeps = 0.2, 2
    z = oracle.prox_qggmrf(v, v, sigma, prm["p"], prm["q"], prm["T"], prm["sx"], prm["bt"], sweeps)
    return {"cite": "Sec. III, Eq. (5): the prior proximal map, with the 4D q-GGMRF prior of Sec. VII "
                    "(26 spatial + 2 temporal neighbours), n_sweeps ICD sweeps started from v",
            "shape": list(shape), "v": _lst(v), "mrf": prm, "sigma": sigma, "n_sweeps": sweeps, "z": _lst(z)}


def mace_plain_tiny():
    sd = dict(n=8, nt=2, nu=10, nv=9, views=4, mode="sparse360")
    sc, counts, y, lam = _measure(sd, 731)
    y32 = np.asarray(y, np.float32).astype(np.float64)
    lam32 = np.asarray(lam, np.float32).astype(np.float64)
    prm = dict(p=2.0, q=1.2, T=1.0, sx=0.1, bt=0.5)
    rho, sigma, mu, n_cg, sweeps, iters = 0.8, 0.2, [0.25, 0.75], 5, 2, 3
    agents = [lambda w, x: oracle.prox_data(y32, lam32, w, x, sc, sigma, n_cg),
              lambda w, x: oracle.prox_qggmrf(w, x, sigma, prm["p"], prm["q"], prm["T"], prm["sx"], prm["bt"],
                                              sweeps)]
    x0, W, X, res = oracle.mace(np.zeros((sc.nt, sc.n, sc.n, sc.n)), agents, mu, rho, iters)
    return {"cite": "Algorithm 1 (Sec. III) with the Mann update of Eq. (12): the data agent and one "
                    "q-GGMRF prior agent, weights mu of Eq. (9), from W = X = 0",
            "scan": sd, "I0": I0, "counts": _lst(counts), "mrf": prm, "rho": rho, "sigma": sigma, "mu": mu,
            "n_cg": n_cg, "n_sweeps": sweeps, "iters": iters, "residuals": _lst(res), "X0": _lst(x0)}


FIXTURES = {"mu_weights": mu_weights, "joseph_8cube": joseph_8cube, "cg_prox_6cube": cg_prox_6cube,
            "qggmrf_prox": qggmrf_prox, "mace_plain_tiny": mace_plain_tiny}


def main():
    oracle.build()
    for name, fn in FIXTURES.items():
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(fn(), f, indent=1)
        print("wrote", name)


if __name__ == "__main__":
    main()
