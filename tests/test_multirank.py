"""The N > 1 path of the benchmark on two CPU ranks (gloo): each rank draws its own
symbols and channels, the timing is the maximum over ranks and the value counts the
whole job's symbols; the oracle's SER counts of two ranks add up to those of one process
over both ranks' symbols; a data-parallel training step (gradients summed over the
ranks, the same averaged step on every rank) equals one process's step over the union
of the ranks' symbols.  No GPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    import oracle
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.rank_env()
    cfg = bench.rank_config(r, 14)
    wl = synth.make_workload(cfg.with_(K=2, M=8, N_d=48, N=64, G=7), S=2)
    t_max = bench.max_over_ranks(0.5 + r, dist, "cpu")
    # each rank's SER counts over its own symbols (the oracle, no noise from other ranks)
    s = synth.qam_symbols(11, 16, (6, 2, 48)).astype(np.complex128)
    d = oracle.make_dims(M=4, K=2, N=64, N_d=48, orders=[1], L=0, G=7, P_T=1.0, S_per_real=3)
    part = s[3 * r:3 * r + 3]
    e, n, _, _ = oracle.ser(d, part, part, np.ones((1, 48)), 16, 0.3, 1000 + r)
    import torch
    tot = torch.tensor([e, n], dtype=torch.int64)
    dist.all_reduce(tot)
    q.put((r, w, local, wl.s[0, 0, :4].tolist(), t_max, bench.job_rate(w, 2000, t_max), tot.tolist(), e, n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_on_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, t0, v0, tot0, e0, n0), (r1, w1, l1, s1, t1, v1, tot1, e1, n1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert s0 != s1                              # every replica draws its own symbols
    assert t0 == t1 == 1.5                       # timing: the slowest rank
    assert v0 == v1 == 2 * 2000 / 1.5            # value: every rank's symbols
    assert tot0 == tot1 == [e0 + e1, n0 + n1]    # counts of the two shards add up
    assert n0 == n1 == 3 * 2 * 48


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None) is None    # returns before reading its arguments
    assert capsys.readouterr().out == ""


def test_single_process_helpers(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (0, 1, 0)
    assert bench.max_over_ranks(0.25, None, "cpu") == 0.25
    assert bench.rank_config(0, 2000).S == 2000 and bench.rank_config(3, 2000).seed == 3
    with pytest.raises(ZeroDivisionError):
        bench.job_rate(1, 10, 0.0)


def _dp_rank_main(rank, world, port, q):
    """One rank of a data-parallel GD step on CPU: the oracle's gradient over this
    rank's shard of symbols (whole realisations), bench.data_parallel_step with a gloo
    all-reduce, the step applied to this rank's copy of theta."""
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    cfg = synth.CONFIGS["m16_k2_n64"].with_(S=4, S_per_real=2)
    w = synth.make_workload(cfg, fc_scale=0.3)
    d = oracle.dims_from_config(cfg, w.P_T)
    W, al = oracle.precode(d, w.H)
    sh = slice(2 * rank, 2 * rank + 2)   # this rank's symbols: realisation `rank`
    theta = torch.from_numpy(w.theta.astype(np.float64))
    lr = 0.5

    def backward():
        g, _ = oracle.backward(d, w.s[sh], w.H[rank:rank + 1], W[rank:rank + 1], al[rank:rank + 1], w.pa, w.theta)
        return torch.from_numpy(g)

    def apply(g, scale):
        theta.sub_(lr * scale * g)

    g = bench.data_parallel_step(backward, dist.all_reduce, apply, world)
    q.put((rank, theta.numpy().copy(), g.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_data_parallel_step_on_gloo():
    """Data-parallel training on two ranks equals one process training on both ranks'
    symbols: the summed per-shard gradients, scaled by 1 / ranks, are the gradient of the
    mean loss over the union (equal shards), and both ranks hold the same theta after
    the step.  The per-rank gradients come from the FP64 oracle."""
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dp_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, th0, g0), (_, th1, g1) = res
    cfg = synth.CONFIGS["m16_k2_n64"].with_(S=4, S_per_real=2)
    w = synth.make_workload(cfg, fc_scale=0.3)
    d = oracle.dims_from_config(cfg, w.P_T)
    W, al = oracle.precode(d, w.H)
    g_all, _ = oracle.backward(d, w.s, w.H, W, al, w.pa, w.theta)
    assert np.array_equal(th0, th1)                       # the same step on every rank
    assert np.array_equal(g0, g1)                         # the all-reduced sum
    assert np.linalg.norm(g_all) > 0
    assert np.allclose(g0 / 2, g_all, rtol=1e-10, atol=1e-12 * np.abs(g_all).max())
    ref = w.theta.astype(np.float64) - 0.5 * g_all
    assert np.allclose(th0, ref, rtol=1e-12, atol=1e-12)


def test_data_parallel_step_single_rank():
    """With one rank the step applies this rank's own gradient unscaled and exchanges nothing."""
    sys.path.insert(0, ROOT)
    import bench
    calls = []
    g = bench.data_parallel_step(lambda: np.array([2.0, -4.0]), lambda x: calls.append("reduce"),
                                 lambda x, sc: calls.append(("apply", sc)), 1)
    assert calls == [("apply", 1.0)] and g.tolist() == [2.0, -4.0]
