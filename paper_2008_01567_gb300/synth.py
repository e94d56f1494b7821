"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws random numbers and fixes scan protocols; it holds none of the
method's arithmetic (no projection, no proximal map, no network).  Both the CUDA
path and the FP64 oracle receive what it returns as plain arrays.

The paper's phantoms and scans (bottle/screw-cap CT volume, vial and injector-pen
scans, Sec. VII) are not available, so seeded moving-ellipsoid phantoms stand in
for them: a 3D phantom translated vertically by one voxel per time-point, as in
Sec. VII-A, observed by a circular-orbit flat-detector cone beam with a sparse set
of views per time-point spanning 360 deg (Sec. VII-A) or a 90 deg wedge (Sec. VII-B).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20200804

# ------------------------------------------------------------------ protocols


@dataclasses.dataclass(frozen=True)
class Scan:
    """One 4D problem: an isotropic cube of n^3 voxels per frame, nt frames, a
    flat detector of nu x nv square pixels and `views` views per frame.

    Lengths are in volume-width units (the volume is 1 wide), so that
    attenuations of 0.5..2 give line integrals of a few units at every size.
    """

    n: int
    nt: int
    nu: int
    nv: int
    views: int
    mode: str = "sparse360"  # or "wedge<D>", e.g. "wedge90"
    dso: float = 4.0          # source to rotation axis
    dsd: float = 8.0          # source to detector (magnification 2)

    @property
    def vox(self) -> float:
        return 1.0 / self.n

    @property
    def pitch(self) -> float:
        """Square detector pitch: 5% margin around the larger of the projected
        circumscribed cylinder (u) and the projected near edge of the volume (v)."""
        half_w = 0.5
        r_cyl = half_w * math.sqrt(2.0)
        u_half = self.dsd * math.tan(math.asin(r_cyl / self.dso))
        v_half = half_w * self.dsd / (self.dso - r_cyl)
        return 1.05 * max(2.0 * u_half / self.nu, 2.0 * v_half / self.nv)

    def angles(self) -> np.ndarray:
        """View angles [nt, views] in radians.

        sparse360: each frame's views span 360 deg and are interlaced across
        frames, th = 2 pi (j + t/nt) / views.
        wedge<D> (e.g. wedge90, wedge180, wedge360): the object turns
        continuously and frame t covers the D-degree wedge [t W, (t+1) W),
        W = D pi / 180, with th = W (t + j/views).
        """
        t = np.arange(self.nt, dtype=np.float64)[:, None]
        j = np.arange(self.views, dtype=np.float64)[None, :]
        if self.mode == "sparse360":
            return 2.0 * math.pi * (j + t / self.nt) / self.views
        if self.mode.startswith("wedge"):
            deg = float(self.mode[len("wedge"):])
            if not 0.0 < deg <= 360.0:
                raise ValueError(self.mode)
            return math.radians(deg) * (t + j / self.views)
        raise ValueError(self.mode)


# The five workloads of the project (sizes as stated in the project's scope):
TINY = Scan(n=24, nt=4, nu=32, nv=32, views=12)                     # plain method, tiny
PROJ = Scan(n=128, nt=8, nu=192, nv=160, views=32)                  # projector / data prox
PROJ_WEDGE = dataclasses.replace(PROJ, mode="wedge90")
FULL = Scan(n=384, nt=16, nu=512, nv=384, views=24)                 # full multi-slice fusion


def batch_scans() -> list[Scan]:
    """The queue of 12 uneven 4D problems: volumes 64^3x4 .. 192^3x12, detectors
    96x96 .. 288x224, 16..48 views; even entries 360 deg sparse, odd 90 deg wedge."""
    out = []
    for i in range(12):
        n = 64 + int(round(128 * i / 11 / 8.0)) * 8
        nt = 4 + int(round(8 * i / 11))
        nu = 96 + int(round(192 * i / 11))
        nv = 96 + int(round(128 * i / 11))
        views = 16 + int(round(32 * i / 11))
        out.append(Scan(n=n, nt=nt, nu=nu, nv=nv, views=views,
                        mode="sparse360" if i % 2 == 0 else "wedge90"))
    return out


# ------------------------------------------------------------------ phantoms


def _rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ellipsoids(seed: int, n_ell: int, scan: Scan, mu_range=(0.5, 2.0),
               axis_range=(0.08, 0.3)) -> np.ndarray:
    """Ellipsoid records for every frame: array [nt, n_ell, 16] of
    centre(3), semi-axes(3), rotation(9, row k = k-th axis), attenuation(1).
    Centres are uniform in the inner 50% of the volume; frame t is frame 0
    shifted by t voxels along +z (one voxel per time-point)."""
    rng = np.random.default_rng(seed)
    base = np.zeros((n_ell, 16))
    for e in range(n_ell):
        base[e, 0:3] = rng.uniform(-0.25, 0.25, 3)
        base[e, 3:6] = rng.uniform(axis_range[0], axis_range[1], 3)
        base[e, 6:15] = _rotation(rng).T.reshape(-1)
        base[e, 15] = rng.uniform(mu_range[0], mu_range[1])
    out = np.repeat(base[None], scan.nt, axis=0)
    out[:, :, 2] += np.arange(scan.nt)[:, None] * scan.vox
    return out


# ------------------------------------------------------------------ noise


def poisson(seed: int, mean: np.ndarray) -> np.ndarray:
    """Photon counts ~ Poisson(mean), as float64."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.asarray(mean, dtype=np.float64)).astype(np.float64)


def normal(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape) * scale


def uniform(seed: int, shape, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, shape)


# ------------------------------------------------------------------ networks


def cnn_weights(seed: int, channels: int = 64, in_frames: int = 5, layers: int = 10):
    """He-normal initial weights of the 2.5D residual CNN: a list of
    (weight [Cout, Cin, 3, 3], bias [Cout]) per layer, plus BatchNorm (gamma, beta)
    for the hidden layers 2..layers-1 (gamma = 1, beta = 0)."""
    rng = np.random.default_rng(seed)
    convs, bns = [], []
    for l in range(layers):
        cin = in_frames if l == 0 else channels
        cout = 1 if l == layers - 1 else channels
        w = rng.standard_normal((cout, cin, 3, 3)) * math.sqrt(2.0 / (9 * cin))
        if l == layers - 1:
            w *= 0.1
        convs.append((w, np.zeros(cout)))
        if 0 < l < layers - 1:
            bns.append((np.ones(channels), np.zeros(channels)))
    return convs, bns
