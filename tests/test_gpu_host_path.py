"""fddpd_update_host: a training step from host buffers, against the same step through the
device entry points fddpd_precode + fddpd_update.

The host path moves the batch in chunks of whole channel realisations and runs each
chunk's ZF (Eq. 6), forward chain and adjoint while the next chunk is copied, with the
loss normalised by the whole batch and the gradient summed over the chunks.  Every
subcarrier's ZF and every symbol's chain are computed on their own, so only the order
of the FP32 sums over symbols (gradient, metrics) differs: theta's step and the
metrics agree to 1e-5 relative.  A single iteration of a 16-bit plan keeps each chunk's
precoder as its factors (fddpd_precode with W = NULL), so the device path does the same.
"""
import numpy as np
import pytest

import synth
from gpu_common import Case, dev, small_cfg, torch

pytestmark = pytest.mark.gpu

CFGS = [
    ("ragged_14_real", small_cfg(S=40, S_per_real=3)),                 # 14 realisations: chunks of 2, last ragged
    ("full_18_real", small_cfg(M=128, K=16, N=512, N_d=300, S=70, S_per_real=4, G=18)),   # chunks of 3
    ("one_real", small_cfg(S=2, S_per_real=3)),                        # R = 1: a single chunk
]


def _host(a):
    T = torch()
    return T.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("name,cfg", CFGS, ids=[n for n, _ in CFGS])
def test_update_host_matches_device_path(name, cfg, prec):
    import paper_2205_05158_gb300 as fd
    T = torch()
    c = Case(cfg, S=cfg.S, fc_scale=0.3, precision=prec)
    lr = 1e-3
    # device path (16-bit plans: the precoder kept as its factors, as the host path's single
    # iteration keeps it)
    met_d = T.zeros(5, dtype=T.float64, device="cuda")
    W = c.W if prec == 0 else None
    c.plan.precode(c.H, W, c.alpha)
    c.plan.update(c.s, c.H, W, c.alpha, c.pa, c.theta, lr, 1, fd.FDDPD_GD, met_d)
    T.cuda.synchronize()
    th_d, met_d = c.theta.cpu().numpy(), met_d.cpu().numpy()
    # host path, separate plan of the same geometry
    plan_h = fd.Plan.from_config(cfg, c.w.P_T, max_symbols=c.S, precision=prec)
    hs, hH, hpa = _host(c.w.s), _host(c.w.H), _host(c.w.pa)
    th_h = _host(c.w.theta.copy())
    met_h = _host(np.zeros(5))
    plan_h.update_host(hs, hH, hpa, th_h, lr, 1, fd.FDDPD_GD, met_h)
    th0 = c.w.theta.astype(np.float64)
    step_d, step_h = th_d - th0, th_h - th0
    assert np.abs(step_d).max() > 0
    assert np.linalg.norm(step_h - step_d) <= 1e-5 * np.linalg.norm(step_d)
    assert np.allclose(met_h, met_d, rtol=1e-5, atol=0)


@pytest.mark.parametrize("opt", ["gd", "adam"])
def test_update_host_iterations(opt):
    """iters = 3: the first pass is chunk-pipelined, the next two run on the resident batch."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = small_cfg(S=40, S_per_real=3)
    o = fd.FDDPD_GD if opt == "gd" else fd.FDDPD_ADAM
    c = Case(cfg, S=cfg.S, fc_scale=0.3)
    met_d = T.zeros(5, dtype=T.float64, device="cuda")
    c.gpu_zf()
    c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, 1e-3, 3, o, met_d)
    plan_h = fd.Plan.from_config(cfg, c.w.P_T, max_symbols=c.S)
    th_h, met_h = _host(c.w.theta.copy()), _host(np.zeros(5))
    plan_h.update_host(_host(c.w.s), _host(c.w.H), _host(c.w.pa), th_h, 1e-3, 3, o, met_h)
    th0 = c.w.theta.astype(np.float64)
    step_d = c.theta.cpu().numpy() - th0
    diff = (th_h - th0) - step_d
    if o == fd.FDDPD_GD:
        assert np.linalg.norm(diff) <= 1e-4 * np.linalg.norm(step_d)
    else:
        # Adam's early steps are ~lr sign(g): a gradient within rounding of zero may differ
        assert np.mean(np.abs(diff) > 0.1 * 1e-3) < 1e-3
        assert np.linalg.norm(diff) <= 1e-2 * np.linalg.norm(step_d)
    assert np.allclose(met_h, met_d.cpu().numpy(), rtol=1e-4, atol=0)


def test_update_host_zero_iters_keeps_theta():
    import paper_2205_05158_gb300 as fd
    cfg = small_cfg(S=40, S_per_real=3)
    c = Case(cfg, S=cfg.S, fc_scale=0.3)
    th = _host(c.w.theta.copy())
    c.plan.update_host(_host(c.w.s), _host(c.w.H), _host(c.w.pa), th, 1e-3, 0, fd.FDDPD_GD, None)
    assert np.array_equal(th, c.w.theta)


def test_update_host_twice_reuses_staging():
    import paper_2205_05158_gb300 as fd
    cfg = small_cfg(S=40, S_per_real=3)
    c = Case(cfg, S=cfg.S, fc_scale=0.3)
    hs, hH, hpa = _host(c.w.s), _host(c.w.H), _host(c.w.pa)
    th1, th2 = _host(c.w.theta.copy()), _host(c.w.theta.copy())
    m1, m2 = _host(np.zeros(5)), _host(np.zeros(5))
    c.plan.update_host(hs, hH, hpa, th1, 1e-3, 1, fd.FDDPD_GD, m1)
    # a shorter call after a longer one uses only its own realisations
    c.plan.update_host(hs[:7], hH[:3], hpa, th2, 1e-3, 1, fd.FDDPD_GD, m2)
    T = torch()
    ref = fd.Plan.from_config(cfg, c.w.P_T, max_symbols=c.S)
    s7, H3, pa, th = dev(c.w.s[:7]), dev(c.w.H[:3]), dev(c.w.pa), dev(c.w.theta)
    W3 = T.empty((3, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    al3 = T.empty((3, cfg.N_d), dtype=T.float32, device="cuda")
    met = T.zeros(5, dtype=T.float64, device="cuda")
    ref.precode(H3, W3, al3)
    ref.update(s7, H3, W3, al3, pa, th, 1e-3, 1, fd.FDDPD_GD, met)
    th0 = c.w.theta.astype(np.float64)
    sr = th.cpu().numpy() - th0
    assert np.linalg.norm((th2 - th0) - sr) <= 1e-5 * np.linalg.norm(sr)
    assert np.allclose(m2, met.cpu().numpy(), rtol=1e-5, atol=0)


@pytest.mark.parametrize("real", [0, 9, 13])
def test_update_host_singular_leaves_theta(real):
    """A singular Gram matrix in any chunk fails the call before the step: theta unchanged."""
    import paper_2205_05158_gb300 as fd
    cfg = small_cfg(S=40, S_per_real=3)
    c = Case(cfg, S=cfg.S, fc_scale=0.3)
    H = c.w.H.copy()
    H[real, 7, 1] = H[real, 7, 0]        # two identical users on one subcarrier
    hs, hH, hpa = _host(c.w.s), _host(H), _host(c.w.pa)
    th = _host(c.w.theta.copy())
    with pytest.raises(fd.FddpdError) as e:
        c.plan.update_host(hs, hH, hpa, th, 1e-3, 1, fd.FDDPD_GD, None)
    assert e.value.code == fd.FDDPD_ERR_SINGULAR
    assert np.array_equal(th, c.w.theta)
    # the plan stays usable
    c.plan.update_host(hs, _host(c.w.H), hpa, th, 1e-3, 1, fd.FDDPD_GD, None)
    assert not np.array_equal(th, c.w.theta)


@pytest.mark.parametrize("chunks", [1, 3, 16])
def test_update_host_chunk_counts(chunks):
    """FDDPD_OPT_HOST_CHUNKS changes only how the batch is pipelined."""
    import paper_2205_05158_gb300 as fd
    cfg = small_cfg(S=40, S_per_real=3)
    c = Case(cfg, S=cfg.S, fc_scale=0.3, precision=1)
    args = (_host(c.w.s), _host(c.w.H), _host(c.w.pa))
    th_ref, m_ref = _host(c.w.theta.copy()), _host(np.zeros(5))
    c.plan.update_host(*args, th_ref, 1e-3, 1, fd.FDDPD_GD, m_ref)
    plan = fd.Plan.from_config(cfg, c.w.P_T, max_symbols=c.S, precision=1)
    plan.set_option(fd.FDDPD_OPT_HOST_CHUNKS, chunks)
    th, m = _host(c.w.theta.copy()), _host(np.zeros(5))
    plan.update_host(*args, th, 1e-3, 1, fd.FDDPD_GD, m)
    th0 = c.w.theta.astype(np.float64)
    assert np.linalg.norm((th - th0) - (th_ref - th0)) <= 1e-5 * np.linalg.norm(th_ref - th0)
    assert np.allclose(m, m_ref, rtol=1e-5, atol=0)
    for bad in (0, 17):
        with pytest.raises(fd.FddpdError):
            plan.set_option(fd.FDDPD_OPT_HOST_CHUNKS, bad)
