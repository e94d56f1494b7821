"""The time-point split on the GPU: two ranks emulated in one process run the
agents through the C ABI on their own frames -- msf_prox_data with a projector
for their frames' views, msf_denoise on the halo-extended block,
msf_mace_consensus -- and must reproduce msf_mace_step on the whole problem.
Every per-frame computation is the same deterministic kernel on the same data
(the adjoint gathers without atomics, the CG keeps its scalars per frame, the
convolutions work image by image, the consensus is per voxel), so the states
are bit-identical."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2008_01567_gb300 import synth, timesplit
from tests._problems import I0, measurement

pytestmark = pytest.mark.gpu
SIGMA, RHO, N_CG, ITERS = 0.1, 0.8, 5, 3
MU = [0.25, 0.25, 0.25, 0.25]


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


def test_emulated_ranks_match_the_whole_problem(M):
    import torch
    scan = synth.Scan(n=24, nt=5, nu=32, nv=32, views=12)
    n, nt = scan.n, scan.nt
    _, counts, _, _ = measurement(scan, 71)
    convs, bns = synth.cnn_weights(72)
    rng = np.random.default_rng(73)
    convs = [(w, rng.normal(0, 0.05, b.shape)) for w, b in convs]
    stats = [(rng.normal(0, 0.1, 64), rng.uniform(0.5, 2.0, 64)) for _ in bns]
    cnn = M.Cnn(n ** 3 * nt)
    cnn.set_params(M.pack_params(convs, bns, stats))
    c = _t(counts)
    y, lam = torch.empty_like(c), torch.empty_like(c)
    M.msf_weights(c, y, lam, I0, I0)
    # the whole problem
    P = M.Projector(scan)
    W = torch.zeros((4, nt, n, n, n), device="cuda")
    X = torch.zeros_like(W)
    m = M.Mace(P, W, X, y, lam, M.MSF_PRIOR_CNN, cnn=cnn)
    res = [M.msf_mace_step(m, RHO, SIGMA, MU, N_CG) for _ in range(ITERS)]
    # two ranks
    ang = scan.angles()
    ranks = []
    for lo, hi in timesplit.frame_blocks(nt, 2):
        Pr = M.Projector(dataclasses.replace(scan, nt=hi - lo), angles=ang[lo:hi])
        ranks.append(dict(lo=lo, hi=hi, P=Pr, dp=M.DataProx(Pr), y=y[lo:hi].contiguous(),
                          lam=lam[lo:hi].contiguous(), W=torch.zeros((4, hi - lo, n, n, n), device="cuda"),
                          X=torch.zeros((4, hi - lo, n, n, n), device="cuda"),
                          work=torch.zeros(M.MSF_CONSENSUS_WORK, dtype=torch.float64, device="cuda")))
    res_split = []
    for _ in range(ITERS):
        # halos of every prior agent's input, before any rank changes W
        for i, r in enumerate(ranks):
            r["ext"] = []
            for k in range(1, 4):
                before = ranks[i - 1]["W"][k, -timesplit.HALO:] if i > 0 else None
                after = ranks[i + 1]["W"][k, :timesplit.HALO] if i + 1 < len(ranks) else None
                r["ext"].append(timesplit.extend(r["W"][k], before, after))
        num = den = 0.0
        for r in ranks:
            nloc = r["hi"] - r["lo"]
            n_prev, _ = timesplit.halo_widths(r["lo"], r["hi"], nt)
            M.msf_prox_data(r["dp"], r["y"], r["lam"], r["W"][0], r["X"][0], SIGMA, N_CG)
            for k in range(1, 4):
                w_ext = r["ext"][k - 1]
                out = torch.empty_like(w_ext)
                M.msf_denoise(cnn, k - 1, M.msf_vol(n, n, n, w_ext.shape[0], 1.0), w_ext, out)
                r["X"][k].copy_(out[n_prev:n_prev + nloc])
            M.msf_mace_consensus(r["W"], r["X"], MU, RHO, r["work"])
            s = r["work"][M.MSF_CONSENSUS_SUMS:M.MSF_CONSENSUS_SUMS + 2].cpu().numpy()
            num, den = num + s[0], den + s[1]
        res_split.append(math.sqrt(num / den))
    torch.cuda.synchronize()
    Ws = torch.cat([r["W"] for r in ranks], dim=1).cpu().numpy().astype(np.float64)
    Xs = torch.cat([r["X"] for r in ranks], dim=1).cpu().numpy().astype(np.float64)
    Wf, Xf = W.cpu().numpy().astype(np.float64), X.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(Ws, Wf)
    np.testing.assert_array_equal(Xs, Xf)
    # the spread's FP64 sums are grouped by rank
    np.testing.assert_allclose(res_split, res, rtol=1e-12)


def test_consensus_arguments(M):
    import torch
    W = torch.zeros((3, 8), device="cuda")
    work = torch.zeros(M.MSF_CONSENSUS_WORK, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MsfError):
        M.msf_mace_consensus(W, W.clone(), [0.5, 0.25, 0.25], 0.5, work)       # K + 1 = 3
    W = torch.zeros((2, 8), device="cuda")
    with pytest.raises(M.MsfError):
        M.msf_mace_consensus(W, W.clone(), [0.5, 0.5], 1.0, work)              # rho outside (0, 1)
    with pytest.raises(M.MsfError):
        M.msf_mace_consensus(W, W.clone(), [0.75, 0.5], 0.5, work)             # weights do not sum to 1
    with pytest.raises(ValueError):
        M.msf_mace_consensus(W, W.clone(), [0.5, 0.5], 0.5, work[:10])         # workspace too small


class _ThreadComm:
    """Two emulated ranks as threads of one process: halos through queues
    (cloned when sent, so later kernels of the sender cannot change them) and
    the sum through a barrier."""

    def __init__(self, rank, world, mail, barrier, sums):
        self.rank, self.world = rank, world
        self.mail, self.barrier, self.sums = mail, barrier, sums

    def exchange(self, to_prev, to_next, n_prev, n_next, like):
        if to_prev is not None:
            self.mail[(self.rank, self.rank - 1)].put(to_prev.clone())
        if to_next is not None:
            self.mail[(self.rank, self.rank + 1)].put(to_next.clone())
        before = self.mail[(self.rank - 1, self.rank)].get(timeout=60) if self.rank > 0 and n_prev else None
        after = self.mail[(self.rank + 1, self.rank)].get(timeout=60) if self.rank + 1 < self.world and n_next else None
        return before, after

    def allreduce_sum(self, t):
        self.sums[self.rank] = t.clone()
        self.barrier.wait(timeout=60)
        total = sum(self.sums[r] for r in range(self.world))
        self.barrier.wait(timeout=60)
        return total


def test_gpu_rank_agents_in_split_step(M):
    # timesplit.GpuRank + split_step, the two ranks as threads, against
    # msf_mace_step on the whole problem: bit-identical states
    import queue
    import threading

    import torch
    scan = synth.Scan(n=24, nt=4, nu=32, nv=32, views=12)
    n, nt = scan.n, scan.nt
    _, counts, _, _ = measurement(scan, 81)
    convs, bns = synth.cnn_weights(82)
    flat = M.pack_params(convs, bns)
    c = _t(counts)
    y, lam = torch.empty_like(c), torch.empty_like(c)
    M.msf_weights(c, y, lam, I0, I0)
    cnn = M.Cnn(n ** 3 * nt)
    cnn.set_params(flat)
    P = M.Projector(scan)
    W = torch.zeros((4, nt, n, n, n), device="cuda")
    X = torch.zeros_like(W)
    m = M.Mace(P, W, X, y, lam, M.MSF_PRIOR_CNN, cnn=cnn)
    res = [M.msf_mace_step(m, RHO, SIGMA, MU, N_CG) for _ in range(ITERS)]
    torch.cuda.synchronize()
    world = 2
    blocks = timesplit.frame_blocks(nt, world)
    mail = {(a, b): queue.Queue() for a in range(world) for b in range(world)}
    barrier, sums = threading.Barrier(world), {}
    states, results, errors = {}, {}, []
    ranks = []
    for r, (lo, hi) in enumerate(blocks):
        cr = M.Cnn(n ** 3 * nt)           # one workspace per rank
        cr.set_params(flat)
        ranks.append(timesplit.GpuRank(M, scan, lo, hi, y[lo:hi].contiguous(), lam[lo:hi].contiguous(), cr,
                                       SIGMA, N_CG))

    def run(r):
        try:
            lo, hi = blocks[r]
            g = ranks[r]
            Wr = torch.zeros((4, hi - lo, n, n, n), device="cuda")
            Xr = torch.zeros_like(Wr)
            comm = _ThreadComm(r, world, mail, barrier, sums)
            results[r] = [timesplit.split_step(Wr, Xr, g.data_agent, g.prior_agents(), g.consensus, MU, RHO, lo, hi,
                                               nt, comm) for _ in range(ITERS)]
            torch.cuda.synchronize()
            states[r] = (Wr, Xr)
        except Exception as e:            # reported below, with the barrier released
            errors.append(e)
            barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=90)
    assert not errors, errors
    Ws = torch.cat([states[r][0] for r in range(world)], dim=1)
    Xs = torch.cat([states[r][1] for r in range(world)], dim=1)
    assert torch.equal(Ws, W) and torch.equal(Xs, X)
    for r in range(world):
        np.testing.assert_allclose(results[r], res, rtol=1e-12)
