"""Seeded test problems built from synth (inputs) and the oracle (measurements
for the oracle side).  Both sides receive the same photon counts."""
import numpy as np

import oracle
from paper_2008_01567_gb300 import synth

I0 = 1e4


def measurement(scan, seed, n_ell=3):
    """(phantom4d, counts, y, lambda) with the oracle's analytic line integrals
    and Poisson counts at I0 photons; y and lambda in float64."""
    ell = synth.ellipsoids(seed, n_ell, scan)
    x0 = oracle.ellipsoid_volume(ell, scan, ss=2)
    p = oracle.ellipsoid_sinogram(ell, scan)
    counts = synth.poisson(seed + 1, oracle.expected_counts(p, I0))
    y = oracle.log_measurement(counts, I0)
    lam = oracle.weights(y, I0)
    return x0, counts, y, lam


def f32(a):
    """Round to float32 and back: the values the GPU side actually receives."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))
