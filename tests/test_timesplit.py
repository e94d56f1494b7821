"""One problem split by time-point over ranks (paper_2008_01567_gb300.timesplit):
the partition and halo arithmetic, and two or three gloo ranks on CPU running Algorithm 1
with the FP64 oracle's agents on their own frames, against the oracle's MACE on
the whole problem.  Every per-frame computation is the same on both sides, so
the states agree to rounding (1e-12 relative)."""
import os
import socket

import numpy as np
import pytest

from paper_2008_01567_gb300 import timesplit

SCAN = dict(n=8, nt=5, nu=10, nv=9, views=4, mode="sparse360")
SIGMA, RHO, N_CG, ITERS = 0.2, 0.8, 3, 3
MU = [0.25, 0.25, 0.25, 0.25]
ORIENTS = ("xy", "yz", "zx")


def test_frame_blocks_partition():
    for nt in range(1, 40):
        for world in range(1, 9):
            if world > 1 and nt // world < timesplit.HALO:
                with pytest.raises(ValueError):
                    timesplit.frame_blocks(nt, world)
                continue
            b = timesplit.frame_blocks(nt, world)
            assert len(b) == world and b[0][0] == 0 and b[-1][1] == nt
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        timesplit.frame_blocks(0, 1)


def test_halo_widths_at_the_ends():
    assert timesplit.halo_widths(0, 3, 5) == (0, 2)
    assert timesplit.halo_widths(3, 5, 5) == (2, 0)
    assert timesplit.halo_widths(4, 8, 16) == (2, 2)
    assert timesplit.halo_widths(0, 16, 16) == (0, 0)


def _problem(nt):
    import oracle
    from paper_2008_01567_gb300 import synth
    from tests._problems import measurement
    scan = synth.Scan(**dict(SCAN, nt=nt))
    _, _, y, lam = measurement(scan, 97)
    convs, bns = synth.cnn_weights(98, channels=16)
    rng = np.random.default_rng(99)
    convs = [(w, rng.normal(0, 0.05, b.shape)) for w, b in convs]
    stats = [(rng.normal(0, 0.1, 16), rng.uniform(0.5, 2.0, 16)) for _ in bns]
    layers = oracle.fold_bn(convs, bns, stats)
    return scan, y, lam, layers


def _consensus(oracle):
    def cons(W, X, mu, rho):
        Wn, Xn = W.numpy(), X.numpy()
        K1 = Wn.shape[0]
        zbar = oracle.average([2.0 * Xn[i] - Wn[i] for i in range(K1)], mu)
        for i in range(K1):
            Wn[i] += 2.0 * rho * (zbar - Xn[i])
        xb = oracle.average(list(Xn), mu)
        num = sum(mu[i] * float(np.vdot(Xn[i] - xb, Xn[i] - xb)) for i in range(K1))
        return num, float(np.vdot(xb, xb))
    return cons


def _worker(rank, world, nt, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        scan, y, lam, layers = _problem(nt)
        ang = scan.angles()
        lo, hi = timesplit.frame_blocks(scan.nt, world)[rank]
        n = scan.n
        W = torch.zeros((4, hi - lo, n, n, n), dtype=torch.float64)
        X = torch.zeros_like(W)

        def data_agent(w0, x0):
            return torch.from_numpy(np.stack([
                oracle.prox_data_frame(y[t], lam[t], w0[i].numpy(), x0[i].numpy(), scan, ang[t], SIGMA, N_CG)
                for i, t in enumerate(range(lo, hi))]))

        def prior(o):
            def agent(w_ext, n_before):
                out_ext = oracle.denoise(w_ext.numpy(), layers, o)
                return torch.from_numpy(out_ext[n_before:n_before + (hi - lo)].copy())
            return agent

        comm = timesplit.TorchComm()
        res = [timesplit.split_step(W, X, data_agent, [prior(o) for o in ORIENTS], _consensus(oracle), MU, RHO,
                                    lo, hi, scan.nt, comm) for _ in range(ITERS)]
        out.put((rank, W.numpy(), X.numpy(), res))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


# two ranks: ragged blocks of 3 and 2 frames, each rank with one neighbour;
# three ranks: blocks of 2, the middle rank receiving halos from both sides
@pytest.mark.parametrize("world,nt", [(2, 5), (3, 6)])
def test_gloo_ranks_match_the_whole_problem(world, nt):
    import multiprocessing as mp

    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, nt, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=600) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # the whole problem in one process
    scan, y, lam, layers = _problem(nt)
    n = scan.n
    agents = [lambda w, x: oracle.prox_data(y, lam, w, x, scan, SIGMA, N_CG)]
    agents += [lambda w, x, o=o: oracle.denoise(w, layers, o) for o in ORIENTS]
    _, Wo, Xo, res = oracle.mace(np.zeros((scan.nt, n, n, n)), agents, MU, RHO, ITERS)
    W = np.concatenate([g[1] for g in got], axis=1)
    X = np.concatenate([g[2] for g in got], axis=1)
    ref_W, ref_X = np.stack(Wo), np.stack(Xo)
    assert np.linalg.norm(W - ref_W) <= 1e-12 * np.linalg.norm(ref_W)
    assert np.linalg.norm(X - ref_X) <= 1e-12 * np.linalg.norm(ref_X)
    for g in got:                       # every rank reports the global spread
        np.testing.assert_allclose(g[3], res, rtol=1e-12)
    # the halo matters: without it the second block's first frame would see
    # its own frame clamped in place of time-points 1 and 2
    v = np.random.default_rng(5).uniform(0.0, 1.5, (scan.nt, n, n, n))
    with_halo = oracle.denoise(v[1:], layers, "xy")[2:]
    without = oracle.denoise(v[3:], layers, "xy")
    assert np.linalg.norm(with_halo[0] - without[0]) > 1e-3 * np.linalg.norm(with_halo[0])
    np.testing.assert_allclose(with_halo, oracle.denoise(v, layers, "xy")[3:], rtol=1e-12, atol=1e-14)
