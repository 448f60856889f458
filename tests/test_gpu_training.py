"""Training runs through the library (Sec. V-A: theta learned by gradient descent through
the PA model): the first GD steps of the 128-antenna, 16-user, N = 2048 system with
per-user FD-CNN parameters against the oracle's own steps, and checkpoint / resume of
theta, the Adam moments and the step counter against an uninterrupted run."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import Case, dev, rel_l2, small_cfg, torch

pytestmark = pytest.mark.gpu


def test_first_gd_steps_match_oracle_per_user():
    """Three GD steps on 4 symbols of the training system (per-user theta_u, FP32 plan,
    the identity predistorter at the start) against oracle.update."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = synth.CONFIGS["m128_k16_n2048_train"].with_(S=4, per_user=1)
    w = synth.make_workload(cfg, fc_scale=0.0)
    d = oracle.dims_from_config(cfg, w.P_T)
    Wo, alo = oracle.precode(d, w.H)
    lr = 30.0   # moves theta far above its FP32 spacing from the identity start
    th_o, met_o = oracle.update(d, w.s, w.H, Wo, alo, w.pa, w.theta, lr, 3)
    plan = fd.Plan.from_config(cfg, w.P_T, max_symbols=cfg.S, precision=fd.FDDPD_FP32)
    s, H, pa, theta = dev(w.s), dev(w.H), dev(w.pa), dev(w.theta)
    W = T.empty((1, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    al = T.empty((1, cfg.N_d), dtype=T.float32, device="cuda")
    plan.precode(H, W, al)
    met = T.zeros(5, dtype=T.float64, device="cuda")
    plan.update(s, H, W, al, pa, theta, lr, 3, fd.FDDPD_GD, met)
    plan.sync()
    th0 = w.theta.astype(np.float64)
    step_gpu = theta.cpu().numpy().astype(np.float64) - th0
    step_o = th_o - th0
    assert np.linalg.norm(step_o) > 0
    assert rel_l2(step_gpu, step_o) <= 1e-4, rel_l2(step_gpu, step_o)
    m = met.cpu().numpy()
    assert abs(m[0] - met_o[0]) <= 1e-6 * met_o[0]     # loss of the third forward pass


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
def test_checkpoint_resume_matches_uninterrupted_run(prec, tmp_path):
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = small_cfg()
    c = Case(cfg, fc_scale=0.3, precision=prec)
    c.gpu_zf()
    lr, n = 1e-3, 3
    th_a = c.theta.clone()
    c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, th_a, lr, 2 * n, fd.FDDPD_ADAM)
    c.plan.sync()
    # first half on a second plan, checkpoint to disk, resume on a third
    p2 = fd.Plan.from_config(cfg, c.w.P_T, max_symbols=c.S, precision=prec)
    th_b = c.theta.clone()
    p2.update(c.s, c.H, c.W, c.alpha, c.pa, th_b, lr, n, fd.FDDPD_ADAM)
    ck = p2.checkpoint(th_b)
    assert ck["adam_t"] == n and np.abs(ck["adam_v"]).max() > 0
    path = str(tmp_path / "ck.npz")
    fd.Plan.save_checkpoint(path, ck)
    p2.close()
    ck2 = fd.Plan.load_checkpoint(path)
    p3 = fd.Plan.from_config(cfg, c.w.P_T, max_symbols=c.S, precision=prec)
    th_c = T.zeros_like(c.theta)
    p3.restore(ck2, th_c)
    back = p3.checkpoint(th_c)                       # the state went in unchanged
    for k in ("theta", "adam_m", "adam_v"):
        assert np.array_equal(back[k], ck[k]), k
    assert back["adam_t"] == n
    p3.update(c.s, c.H, c.W, c.alpha, c.pa, th_c, lr, n, fd.FDDPD_ADAM)
    p3.sync()
    a, b = th_a.cpu().numpy().astype(np.float64), th_c.cpu().numpy().astype(np.float64)
    th0 = c.w.theta.astype(np.float64)
    assert rel_l2(b - th0, a - th0) <= 1e-5, rel_l2(b - th0, a - th0)


def test_restore_rejects_bad_state():
    import paper_2205_05158_gb300 as fd
    T = torch()
    c = Case(synth.CONFIGS["m16_k2_n64"], precision=0)
    ck = c.plan.checkpoint(c.theta)
    with pytest.raises(ValueError):
        c.plan.restore({**ck, "adam_m": ck["adam_m"][:-1]}, c.theta)
    L = fd.load()
    m = T.zeros(c.plan.theta_len, dtype=T.float32, device="cuda")
    assert L.fddpd_set_optimizer_state(c.plan.handle, m.data_ptr(), m.data_ptr(), -1) == fd.FDDPD_ERR_ARG
    assert L.fddpd_set_optimizer_state(c.plan.handle, None, m.data_ptr(), 0) == fd.FDDPD_ERR_ARG
