"""Image-quality figures of a 4D reconstruction against its phantom (Sec. VI):
NRMSE, the percentile-range PSNR the paper defines, and SSIM (Wang et al.).

These are reporting helpers over device tensors (PyTorch arithmetic); they are
not part of the reconstruction path.

SSIM reading: the paper cites SSIM without saying how it extends to 4D; here
it is the mean, over every xy-slice of every time-point, of the standard SSIM
map of Wang et al. (11 x 11 Gaussian window of standard deviation 1.5,
K1 = 0.01, K2 = 0.03, windows wholly inside the slice), with the dynamic range
L taken as the phantom's percentile range used by the PSNR.
"""
from __future__ import annotations

import math

WIN, WIN_SIGMA, K1, K2 = 11, 1.5, 0.01, 0.03


def nrmse(x, ref) -> float:
    """||x - ref||_2 / ||ref||_2 over the whole array."""
    import torch
    return (torch.linalg.vector_norm((x - ref).double()) / torch.linalg.vector_norm(ref.double())).item()


def percentile(a, q: float) -> float:
    """The q-th percentile of all entries, linear between the closest ranks
    (the usual definition: position q/100 * (n - 1) in sorted order)."""
    import torch
    v = torch.sort(a.reshape(-1)).values
    pos = q / 100.0 * (v.numel() - 1)
    lo = int(math.floor(pos))
    hi = min(lo + 1, v.numel() - 1)
    f = pos - lo
    return float(v[lo].item()) * (1.0 - f) + float(v[hi].item()) * f


def value_range(ref) -> float:
    """Range(x0): the 99.9th minus the 0.1st percentile of the phantom."""
    return percentile(ref, 99.9) - percentile(ref, 0.1)


def psnr(x, ref) -> float:
    """20 log10(Range(ref) / RMSE(x, ref)), Sec. VI."""
    import torch
    rmse = math.sqrt(torch.mean((x.double() - ref.double()) ** 2).item())
    return 20.0 * math.log10(value_range(ref) / rmse)


def _gauss(device, dtype):
    import torch
    r = torch.arange(WIN, device=device, dtype=dtype) - (WIN - 1) / 2.0
    g = torch.exp(-(r * r) / (2.0 * WIN_SIGMA * WIN_SIGMA))
    return g / g.sum()


def ssim(x, ref, L: float | None = None, chunk: int = 256) -> float:
    """Mean SSIM over all 2D slices of the last two axes (xy-slices of every
    time-point for a [nt][nz][ny][nx] volume); L defaults to value_range(ref)."""
    import torch
    if L is None:
        L = value_range(ref)
    c1, c2 = (K1 * L) ** 2, (K2 * L) ** 2
    H, W = x.shape[-2], x.shape[-1]
    if H < WIN or W < WIN:
        raise ValueError(f"slices of {H} x {W} are smaller than the {WIN} x {WIN} window")
    xs = x.reshape(-1, 1, H, W)
    rs = ref.reshape(-1, 1, H, W)
    dtype = torch.float64 if x.device.type == "cpu" else torch.float32
    g = _gauss(x.device, dtype)
    gr, gc = g.view(1, 1, WIN, 1), g.view(1, 1, 1, WIN)

    def filt(a):
        return torch.nn.functional.conv2d(torch.nn.functional.conv2d(a, gr), gc)

    total, count = 0.0, 0
    for i in range(0, xs.shape[0], chunk):
        a = xs[i:i + chunk].to(dtype)
        b = rs[i:i + chunk].to(dtype)
        mx, my = filt(a), filt(b)
        sxx = filt(a * a) - mx * mx
        syy = filt(b * b) - my * my
        sxy = filt(a * b) - mx * my
        m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
        total += float(m.double().sum().item())
        count += m.numel()
    return total / count
