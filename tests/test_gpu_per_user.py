"""Per-user FD-CNN parameters theta_u (Sec. IV-A; fddpd_dpd_desc.per_user, FP32 plans with
L_U = 1) against the FP64 oracle: the forward chain, the gradient of every user's slice
and a GD step, at the FP32 tolerances of the shared network; and K copies of one theta
against the shared network."""
import numpy as np
import pytest

import oracle
from gpu_common import Case, dev, nmse, rel_l2, small_cfg, torch

pytestmark = pytest.mark.gpu


def _cfg(**kw):
    # 40 antennas, 3 users, 150 bins on a 13 x 13 grid with stride 2, 7 symbols
    return small_cfg(L_U=1, **kw)


def test_per_user_chain_matches_oracle():
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = _cfg(per_user=1)
    c = Case(cfg, fc_scale=0.3)
    one = oracle.theta_len(oracle.dims_from_config(cfg.with_(per_user=0), c.w.P_T))
    assert c.plan.theta_len == cfg.K * one == c.w.theta.size
    c.use_oracle_zf_on_gpu()
    Wo, alo = c.oracle_zf()
    y, met = c.gpu_distort()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert nmse(y, yo) <= 1e-9
    assert abs(met[0] - meto[0]) <= 1e-4 * meto[0]
    g, _ = c.gpu_backward()
    go, _ = oracle.backward(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert rel_l2(g, go) <= 1e-4
    for u in range(cfg.K):
        assert rel_l2(g[u * one:(u + 1) * one], go[u * one:(u + 1) * one]) <= 1e-3, u
    # one GD step moves theta by -lr * grad
    lr = 1.0
    th0 = c.theta.clone()
    c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, lr, 1, fd.FDDPD_GD)
    T.cuda.synchronize()
    step = (c.theta - th0).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(step + lr * go) <= 1e-3 * np.linalg.norm(lr * go)


def test_per_user_copies_of_one_theta_match_the_shared_network():
    """K copies of the shared theta: the same received symbols, and the per-user gradient
    slices add up to the shared gradient."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = _cfg()
    c = Case(cfg, fc_scale=0.3)
    c.gpu_zf()
    y0, _ = c.gpu_distort()
    g0, _ = c.gpu_backward()
    pu = fd.Plan.from_config(cfg.with_(per_user=1), c.w.P_T, max_symbols=c.S)
    thK = dev(np.tile(c.w.theta, cfg.K))
    y = T.empty_like(c.s)
    pu.distort(c.s, c.H, c.W, c.alpha, c.pa, thK, y)
    g = T.empty(pu.theta_len, dtype=T.float32, device="cuda")
    pu.backward(c.s, c.H, c.W, c.alpha, c.pa, thK, g)
    T.cuda.synchronize()
    # the same kernels over per-user column blocks: only FP32 summation orders differ
    assert nmse(y.cpu().numpy(), y0) <= 1e-10
    gsum = g.cpu().numpy().astype(np.float64).reshape(cfg.K, -1).sum(axis=0)
    assert rel_l2(gsum, g0) <= 2e-4
