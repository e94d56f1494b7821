"""One 4D MACE problem split by time-point over ranks.

The data term separates over time-points (Sec. II, Eq. (2)): rank r keeps the
frames [lo, hi) of every state and runs the data agent on them alone.  The CNN
agents of Sec. IV read the five time-points t-2 .. t+2 of a slice (clamped at
the first and last time-point), so before them every rank receives a halo of
HALO = 2 frames of each prior agent's input W_k from each time neighbour.  The
consensus and Mann update of Algorithm 1 are per voxel; only the consensus
spread (the stopping quantity of Sec. III) sums over all frames, one allreduce
of two FP64 numbers per iteration.

The q-GGMRF prior of the plain method couples time-points inside every ICD
sweep and is not split here.

The module is host logic only.  The agents and the consensus are callables, so
the same step runs the CUDA path (GpuRank: msf_prox_data on the rank's frames,
msf_denoise on the halo-extended block, msf_mace_consensus) and, in the tests,
the FP64 oracle.  TorchComm carries the halos and the sum over
torch.distributed: gloo for CPU tensors, NCCL for CUDA tensors.
"""
from __future__ import annotations

import math

HALO = 2


def frame_blocks(nt: int, world: int) -> list[tuple[int, int]]:
    """Contiguous blocks [lo, hi) of time-points, one per rank, sizes differing
    by at most one.  With more than one rank every block must hold at least
    HALO frames, so that a halo comes from the neighbouring rank alone."""
    if nt < 1 or world < 1:
        raise ValueError(f"need nt >= 1 and world >= 1, got nt={nt}, world={world}")
    base, extra = divmod(nt, world)
    if world > 1 and base < HALO:
        raise ValueError(f"{nt} time-points over {world} ranks leaves a rank fewer than {HALO} frames")
    blocks, lo = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        blocks.append((lo, lo + n))
        lo += n
    return blocks


def halo_widths(lo: int, hi: int, nt: int) -> tuple[int, int]:
    """Frames a rank holding [lo, hi) receives before and after its own."""
    return min(HALO, lo), min(HALO, nt - hi)


def extend(local, before, after):
    """The halo-extended block: frames received from the previous rank, the
    rank's own frames, frames received from the next rank (along dim 0)."""
    import torch
    parts = [p for p in (before, local, after) if p is not None and p.shape[0] > 0]
    return torch.cat(parts, dim=0)


class TorchComm:
    """Halo exchange between time neighbours and the FP64 sum, over the default
    torch.distributed process group."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()

    def exchange(self, to_prev, to_next, n_prev: int, n_next: int, like):
        """Sends to_prev to rank - 1 and to_next to rank + 1, receives n_prev
        frames from rank - 1 and n_next from rank + 1 (frames shaped like
        like[0]).  Returns (from_prev, from_next), None where there is no
        neighbour."""
        import torch
        dist = self.dist
        reqs = []
        from_prev = from_next = None
        if self.rank > 0 and n_prev > 0:
            from_prev = torch.empty((n_prev,) + tuple(like.shape[1:]), dtype=like.dtype, device=like.device)
            reqs.append(dist.irecv(from_prev, self.rank - 1))
        if self.rank < self.world - 1 and n_next > 0:
            from_next = torch.empty((n_next,) + tuple(like.shape[1:]), dtype=like.dtype, device=like.device)
            reqs.append(dist.irecv(from_next, self.rank + 1))
        if to_prev is not None:
            reqs.append(dist.isend(to_prev.contiguous(), self.rank - 1))
        if to_next is not None:
            reqs.append(dist.isend(to_next.contiguous(), self.rank + 1))
        for r in reqs:
            r.wait()
        return from_prev, from_next

    def allreduce_sum(self, t):
        self.dist.all_reduce(t)
        return t


def split_step(W, X, data_agent, prior_agents, consensus, mu, rho, lo: int, hi: int, nt: int, comm) -> float:
    """One pass of Algorithm 1 on this rank's frames [lo, hi) of one problem.

    W, X: stacked states [K + 1, hi - lo, ...] of this rank, updated in place.
    data_agent(w0, x0) -> new X_0 frames (the partial update of Eq. (13)).
    prior_agents[k - 1](w_ext, n_before) -> new X_k frames, from the
        halo-extended input W_k and the number of halo frames before the
        rank's own.
    consensus(W, X, mu, rho) -> (num, den): the Mann update of W in place and
        this rank's sums of sum_i mu_i (X_i - Xbar)^2 and Xbar^2.
    Returns the consensus spread over all ranks, sqrt(num / den)."""
    import torch
    n_prev, n_next = halo_widths(lo, hi, nt)
    first, last = comm.rank == 0, comm.rank == comm.world - 1
    # halos of the prior agents' inputs, taken before anything changes W
    ext = []
    for k in range(1, len(prior_agents) + 1):
        to_prev = None if first else W[k, :HALO]
        to_next = None if last else W[k, W.shape[1] - HALO:]
        before, after = comm.exchange(to_prev, to_next, n_prev, n_next, W[k])
        ext.append(extend(W[k], before, after))
    X[0].copy_(data_agent(W[0], X[0]))
    for k, agent in enumerate(prior_agents, start=1):
        X[k].copy_(agent(ext[k - 1], n_prev))
    num, den = consensus(W, X, mu, rho)
    s = comm.allreduce_sum(torch.tensor([num, den], dtype=torch.float64, device=W.device))
    num, den = float(s[0]), float(s[1])
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)


class GpuRank:
    """This rank's agents for split_step on its GPU, through the C ABI: the
    data agent on frames [lo, hi) with a projector plan for those frames'
    views, the three CNN agents (xy-t, yz-t, zx-t) on the halo-extended
    blocks, and the consensus of msf_mace_consensus.

    msf: the binding module; scan: the whole problem's scan (synth.Scan-like);
    y, lam: this rank's measurements [hi - lo, views, nv, nu] on the device;
    cnn: this rank's msf.Cnn handle (its workspace must not be shared with
    another rank that runs at the same time)."""

    def __init__(self, msf, scan, lo: int, hi: int, y, lam, cnn, sigma: float, n_cg: int, angles=None):
        import dataclasses

        import numpy as np
        import torch
        ang = np.asarray(scan.angles() if angles is None else angles, dtype=np.float64)
        self.msf, self.lo, self.hi = msf, lo, hi
        self.proj = msf.Projector(dataclasses.replace(scan, nt=hi - lo), angles=ang[lo:hi])
        self.dp = msf.DataProx(self.proj)
        self.y, self.lam, self.cnn = y, lam, cnn
        self.sigma, self.n_cg = sigma, n_cg
        v = self.proj.vol
        self.shape = (v.nx, v.ny, v.nz, v.voxel)
        self.work = torch.zeros(msf.MSF_CONSENSUS_WORK, dtype=torch.float64, device="cuda")

    def data_agent(self, w0, x0):
        self.msf.msf_prox_data(self.dp, self.y, self.lam, w0, x0, self.sigma, self.n_cg)
        return x0

    def prior_agents(self):
        return [self._cnn_agent(o) for o in (0, 1, 2)]

    def _cnn_agent(self, orient: int):
        import torch
        nx, ny, nz, voxel = self.shape

        def agent(w_ext, n_before):
            out = torch.empty_like(w_ext)
            self.msf.msf_denoise(self.cnn, orient, self.msf.msf_vol(nx, ny, nz, w_ext.shape[0], voxel), w_ext, out)
            return out[n_before:n_before + (self.hi - self.lo)]
        return agent

    def consensus(self, W, X, mu, rho):
        self.msf.msf_mace_consensus(W, X, mu, rho, self.work)
        s = self.work[self.msf.MSF_CONSENSUS_SUMS:self.msf.MSF_CONSENSUS_SUMS + 2].cpu()
        return float(s[0]), float(s[1])
