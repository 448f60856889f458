"""Per-user FD-CNN parameters theta_u (Sec. IV-A; fddpd_dpd_desc.per_user) against the FP64
oracle in every precision and for L_U = 1 and 2: the forward chain, the gradient of every
user's slice and a GD step (FP32 tolerances in FP32 plans; NMSE 1e-4 and gradients 2e-2
in 16-bit plans); and K copies of one theta against the shared network."""
import numpy as np
import pytest

import oracle
from gpu_common import Case, dev, nmse, rel_l2, small_cfg, torch

pytestmark = pytest.mark.gpu

def _cfg(L_U=1, **kw):
    # 40 antennas, 3 users, 150 bins on a 13 x 13 grid with stride 2, 7 symbols
    return small_cfg(L_U=L_U, **kw)


CASES = [(p, l) for p in (0, 1, 2) for l in (1, 2)]
IDS = [f"{('fp32', 'bf16', 'fp16')[p]}-L_U{l}" for p, l in CASES]


@pytest.mark.parametrize("prec,L_U", CASES, ids=IDS)
def test_per_user_chain_matches_oracle(prec, L_U):
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = _cfg(L_U, per_user=1)
    c = Case(cfg, fc_scale=0.3, precision=prec)
    one = oracle.theta_len(oracle.dims_from_config(cfg.with_(per_user=0), c.w.P_T))
    assert c.plan.theta_len == cfg.K * one == c.w.theta.size
    c.use_oracle_zf_on_gpu()
    Wo, alo = c.oracle_zf()
    y, met = c.gpu_distort()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    tol_y, tol_g, tol_u, tol_l = (1e-9, 1e-4, 1e-3, 1e-4) if prec == 0 else (1e-4, 2e-2, 2e-2, 1e-2)
    assert nmse(y, yo) <= tol_y, nmse(y, yo)
    assert abs(met[0] - meto[0]) <= tol_l * meto[0]
    g, _ = c.gpu_backward()
    c.plan.sync()
    go, _ = oracle.backward(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert rel_l2(g, go) <= tol_g, rel_l2(g, go)
    for u in range(cfg.K):
        assert rel_l2(g[u * one:(u + 1) * one], go[u * one:(u + 1) * one]) <= tol_u, u
    # one GD step moves theta by -lr * grad
    lr = 1.0
    th0 = c.theta.clone()
    c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, lr, 1, fd.FDDPD_GD)
    T.cuda.synchronize()
    step = (c.theta - th0).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(step + lr * go) <= (1e-3 if prec == 0 else 2e-2) * np.linalg.norm(lr * go)


@pytest.mark.parametrize("prec,L_U", CASES, ids=IDS)
def test_per_user_copies_of_one_theta_match_the_shared_network(prec, L_U):
    """K copies of the shared theta: the same received symbols, and the per-user gradient
    slices add up to the shared gradient."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = _cfg(L_U)
    c = Case(cfg, fc_scale=0.3, precision=prec)
    c.gpu_zf()
    y0, _ = c.gpu_distort()
    g0, _ = c.gpu_backward()
    pu = fd.Plan.from_config(cfg.with_(per_user=1), c.w.P_T, max_symbols=c.S, precision=prec)
    thK = dev(np.tile(c.w.theta, cfg.K))
    y = T.empty_like(c.s)
    pu.distort(c.s, c.H, c.W, c.alpha, c.pa, thK, y)
    g = T.empty(pu.theta_len, dtype=T.float32, device="cuda")
    pu.backward(c.s, c.H, c.W, c.alpha, c.pa, thK, g)
    T.cuda.synchronize()
    # the same kernels over per-user column blocks: only summation orders differ (and in
    # 16-bit plans the rounding of the per-user weight-gradient partial sums)
    assert nmse(y.cpu().numpy(), y0) <= (1e-10 if prec == 0 else 1e-6)
    gsum = g.cpu().numpy().astype(np.float64).reshape(cfg.K, -1).sum(axis=0)
    assert rel_l2(gsum, g0) <= (2e-4 if prec == 0 else 1e-2)
