"""Batched uneven workload: independent downlink instances of different (M, K, N) recorded
into one CUDA graph (fddpd_graph_*) and replayed as one launch.  The replay must give what
the same calls give one by one (the same kernels on the same inputs), and each instance
stays within the 16-bit tolerances of the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_common import Case, nmse, rel_l2, small_cfg, torch

pytestmark = pytest.mark.gpu

# (M, K, N, orders): K <= M / 4, about 58 % of the bins occupied, odd-order PAs with memory
SHAPES = [(32, 4, 512, {1: [1.0, 0.05 - 0.02j, 0.01, 0.002], 3: [-0.08 + 0.02j, 0.01j, -0.003, 0.001]}),
          (64, 8, 1024, synth.PA_NOMINAL_MP135),
          (32, 8, 512, synth.PA_NOMINAL_MP135),
          (128, 16, 512, {1: [1.0, 0.05 - 0.02j, 0.01, 0.002], 3: [-0.08 + 0.02j, 0.01j, -0.003, 0.001]}),
          (64, 16, 2048, synth.PA_NOMINAL_MP135),
          (128, 32, 1024, synth.PA_NOMINAL_MP135)]


def _instance(i, shape, S=10):
    M, K, N, pa = shape
    N_d = int(round(N * 600 / 1024))
    cfg = small_cfg(name=f"inst{i}", M=M, K=K, N=N, N_d=N_d, Q=64, S=S, S_per_real=5, pa_nominal=pa,
                    G=math.ceil(math.sqrt(N_d)), L_U=1, K_S=1, seed=100 + i)
    c = Case(cfg, S=S, fc_scale=0.2, precision=1)
    c.gpu_zf()
    return c


def test_graph_replays_uneven_instances():
    T = torch()
    cases = [_instance(i, sh) for i, sh in enumerate(SHAPES)]
    # one by one on the default stream
    ref = []
    for c in cases:
        ref.append(c.gpu_distort())
    # recorded on a side stream, replayed as one graph launch (twice)
    stream = T.cuda.Stream()
    ys = [T.empty_like(c.s) for c in cases]
    mets = [T.zeros(5, dtype=T.float64, device="cuda") for c in cases]
    for c in cases:
        c.plan.set_stream(stream)
    import paper_2205_05158_gb300 as fd
    T.cuda.synchronize()
    with fd.Graph.record(stream) as g:
        for c, y, m in zip(cases, ys, mets):
            c.plan.distort(c.s, c.H, c.W, c.alpha, c.pa, c.theta, y, m)
    for _ in range(2):
        g.launch()
    T.cuda.synchronize()
    for c, y, m, (y0, m0) in zip(cases, ys, mets, ref):
        assert np.array_equal(y.cpu().numpy(), y0)
        assert np.allclose(m.cpu().numpy(), m0, rtol=1e-12, atol=0)
    # two instances against the oracle (16-bit tolerances)
    for c, (y0, m0) in list(zip(cases, ref))[:2]:
        Wo, alo = c.oracle_zf()
        yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
        assert nmse(y0, yo) <= 1e-4
        assert abs(oracle.evm_db(m0) - oracle.evm_db(meto)) <= 0.1


def test_graph_replays_training_steps():
    """One GD step of three uneven instances recorded and replayed from the same theta:
    the same step as one by one (up to the order of the split-K sums)."""
    T = torch()
    import paper_2205_05158_gb300 as fd
    cases = [_instance(i, sh) for i, sh in enumerate(SHAPES[:3])]
    th0 = [c.theta.clone() for c in cases]
    for c in cases:
        c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, 1e-3, 1, fd.FDDPD_GD)
    T.cuda.synchronize()
    step_ref = [(c.theta - t).cpu().numpy() for c, t in zip(cases, th0)]
    stream = T.cuda.Stream()
    for c, t in zip(cases, th0):
        c.theta.copy_(t)
        c.plan.set_stream(stream)
    T.cuda.synchronize()
    with fd.Graph.record(stream) as g:
        for c in cases:
            c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, 1e-3, 1, fd.FDDPD_GD)
    g.launch()
    T.cuda.synchronize()
    for c, t, sr in zip(cases, th0, step_ref):
        assert rel_l2((c.theta - t).cpu().numpy(), sr) <= 1e-5


@pytest.mark.parametrize("shape_i", [1, 5], ids=["m64_k8", "m128_k32"])
def test_autotune_picks_an_admitted_implementation(shape_i):
    """fddpd_autotune times the admitted contraction implementations and keeps the faster:
    16-bit plans of up to 256 antennas and 32 users admit both (K = 32: the tensor-core
    form with two user halves); the result stays within the 16-bit tolerances."""
    import paper_2205_05158_gb300 as fd
    c = _instance(shape_i, SHAPES[shape_i])
    t_tc, t_cc = c.plan.autotune(c.s, c.H, c.W, c.alpha, c.pa, c.theta, reps=2)
    assert t_cc > 0 and t_tc > 0
    assert c.plan.get_option(fd.FDDPD_OPT_TENSOR_CONTRACTIONS) == (1 if t_tc <= t_cc else 0)
    y, met = c.gpu_distort()
    Wo, alo = c.oracle_zf()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert nmse(y, yo) <= 1e-4
    assert abs(oracle.evm_db(met) - oracle.evm_db(meto)) <= 0.1


def test_autotune_fp32_plan_has_one_choice():
    cfg = small_cfg()
    c = Case(cfg, S=cfg.S)
    c.gpu_zf()
    t_tc, t_cc = c.plan.autotune(c.s, c.H, c.W, c.alpha, c.pa, c.theta, reps=1)
    assert t_tc == -1.0 and t_cc > 0


def _uneven_case(cfg):
    c = Case(cfg, S=cfg.S, fc_scale=0.2, precision=1)
    c.plan.precode(c.H, None, c.alpha)          # the precoder kept as its factors
    return c


def test_graph_lanes_uneven_instances_with_autotune():
    """Sixteen instances of the uneven batched workload (M 32..256, K 4..32, N 512..4096,
    orders {1,3} or {1,3,5}), each autotuned (choices stored per shape), recorded on four
    concurrent lanes of one graph and replayed twice: the same outputs as one by one; the
    two smallest instances within the 16-bit tolerances of the oracle."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    fd.autotune_forget()
    cfgs = synth.uneven_instances(16, S=6, S_per_real=3)
    cases = [_uneven_case(cfg) for cfg in cfgs]
    for c in cases:
        c.plan.autotune(c.s, c.H, None, c.alpha, c.pa, c.theta, reps=1)
    ref = []
    for c in cases:
        y = T.empty_like(c.s)
        m = T.zeros(5, dtype=T.float64, device="cuda")
        c.plan.distort(c.s, c.H, None, c.alpha, c.pa, c.theta, y, m)
        ref.append((y, m))
    T.cuda.synchronize()
    main = T.cuda.Stream()
    ys = [T.empty_like(c.s) for c in cases]
    ms = [T.zeros(5, dtype=T.float64, device="cuda") for c in cases]
    with fd.Graph.record_lanes(main, 4) as (g, lanes):
        for i, (c, y, m) in enumerate(zip(cases, ys, ms)):
            c.plan.set_stream(lanes[i % 4])
            c.plan.distort(c.s, c.H, None, c.alpha, c.pa, c.theta, y, m)
    for _ in range(2):
        g.launch()
    main.synchronize()
    for c in cases:
        c.plan.set_stream(None)
    for (y0, m0), y, m in zip(ref, ys, ms):
        assert T.equal(y, y0)
        assert np.allclose(m.cpu().numpy(), m0.cpu().numpy(), rtol=1e-12, atol=0)
    small = sorted(range(len(cfgs)), key=lambda i: cfgs[i].M * cfgs[i].N)[:2]
    for i in small:
        c = cases[i]
        Wo, alo = c.oracle_zf()
        yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
        assert nmse(ref[i][0].cpu().numpy(), yo) <= 1e-4
        assert abs(oracle.evm_db(ref[i][1].cpu().numpy()) - oracle.evm_db(meto)) <= 0.1


def test_autotune_choice_stored_per_shape_and_row_ctas_exact():
    import paper_2205_05158_gb300 as fd
    T = torch()
    fd.autotune_forget()
    cfg = synth.uneven_instances(1, S=6, S_per_real=3)[0].with_(M=64, K=8, N=1024, N_d=600)
    a, b = _uneven_case(cfg), _uneven_case(cfg.with_(seed=7))
    ta = a.plan.autotune(a.s, a.H, None, a.alpha, a.pa, a.theta, reps=1)
    tb = b.plan.autotune(b.s, b.H, None, b.alpha, b.pa, b.theta, reps=1)
    assert ta == tb                                   # the stored choice, not a new timing
    for o in (fd.FDDPD_OPT_TENSOR_CONTRACTIONS, fd.FDDPD_OPT_ROW_CTAS, fd.FDDPD_OPT_CONTRACTION_CTAS,
              fd.FDDPD_OPT_CONTRACTION_ITEM):
        assert a.plan.get_option(o) == b.plan.get_option(o)
    a.plan.set_option(fd.FDDPD_OPT_TENSOR_CONTRACTIONS, 1)
    outs = []
    # the grid shapes and the contraction items' size change no arithmetic
    for rc, bc, hi in ((0, 0, 0), (1, 0, 0), (2, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 1, 1)):
        a.plan.set_option(fd.FDDPD_OPT_ROW_CTAS, rc)
        a.plan.set_option(fd.FDDPD_OPT_CONTRACTION_CTAS, bc)
        a.plan.set_option(fd.FDDPD_OPT_CONTRACTION_ITEM, hi)
        assert a.plan.get_option(fd.FDDPD_OPT_CONTRACTION_CTAS) == (1 if bc == 1 else 2)
        assert a.plan.get_option(fd.FDDPD_OPT_CONTRACTION_ITEM) == hi
        y = T.empty_like(a.s)
        a.plan.distort(a.s, a.H, None, a.alpha, a.pa, a.theta, y)
        outs.append(y)
    T.cuda.synchronize()
    assert all(T.equal(outs[0], o) for o in outs[1:])
    with pytest.raises(fd.FddpdError):
        a.plan.set_option(fd.FDDPD_OPT_ROW_CTAS, 9)
    with pytest.raises(fd.FddpdError):
        a.plan.set_option(fd.FDDPD_OPT_CONTRACTION_CTAS, 3)
    with pytest.raises(fd.FddpdError):
        a.plan.set_option(fd.FDDPD_OPT_CONTRACTION_ITEM, 2)
