"""Failure detection and fault injection without a GPU fault.

- A bounded device wait made to run out (fddpd_selftest_wait: an mbarrier nothing arrives
  at, no copy or MMA in flight) is reported by the next fddpd_sync as FDDPD_ERR_TIMEOUT,
  the report is cleared, and the plan keeps computing correctly.
- Failed device allocations (fddpd_debug_fail_allocs) turn into FDDPD_ERR_NOMEM at plan
  creation, at the host-buffer staging, at the first Adam step and at the kept-PA-input
  option, and the library works again afterwards.
- NaN inputs: a NaN in H makes the Gram check fail (FDDPD_ERR_SINGULAR, nothing used);
  a NaN symbol propagates to the metrics without any sticky state in the plan.
"""
import numpy as np
import pytest

import synth
from gpu_common import Case, dev, nmse, small_cfg, torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_is_reported():
    import paper_2205_05158_gb300 as fd
    c = Case(small_cfg(), fc_scale=0.3, precision=1)
    c.gpu_zf()
    y0, _ = c.gpu_distort()
    c.plan.sync()
    c.plan.selftest_wait(20000)          # 20 ms
    with pytest.raises(fd.FddpdError) as e:
        c.plan.sync()
    assert e.value.code == fd.FDDPD_ERR_TIMEOUT
    c.plan.sync()                        # the report was cleared
    y1, _ = c.gpu_distort()
    assert np.array_equal(y0, y1)
    with pytest.raises(fd.FddpdError):
        c.plan.selftest_wait(0)


def test_failed_allocations_become_nomem():
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = small_cfg()
    w = synth.make_workload(cfg, fc_scale=0.3)
    fd.debug_fail_allocs(1)
    with pytest.raises(fd.FddpdError) as e:
        fd.Plan.from_config(cfg, w.P_T, max_symbols=cfg.S, precision=1)
    assert e.value.code == fd.FDDPD_ERR_NOMEM
    c = Case(cfg, fc_scale=0.3, precision=1)       # allocations work again
    c.gpu_zf()
    fd.debug_fail_allocs(1)
    with pytest.raises(fd.FddpdError) as e:        # the first Adam step allocates the moments
        c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, 1e-3, 1, fd.FDDPD_ADAM)
    assert e.value.code == fd.FDDPD_ERR_NOMEM
    th = c.theta.clone()
    c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, 1e-3, 1, fd.FDDPD_ADAM)
    T.cuda.synchronize()
    assert not T.equal(th, c.theta)
    fd.debug_fail_allocs(1)
    with pytest.raises(fd.FddpdError) as e:
        c.plan.set_option(fd.FDDPD_OPT_KEEP_PA_INPUT, 1)
    assert e.value.code == fd.FDDPD_ERR_NOMEM
    assert c.plan.get_option(fd.FDDPD_OPT_KEEP_PA_INPUT) == 0
    hs = T.from_numpy(w.s).pin_memory().numpy()
    hH = T.from_numpy(w.H).pin_memory().numpy()
    hpa = T.from_numpy(w.pa).pin_memory().numpy()
    hth = T.from_numpy(w.theta.copy()).pin_memory().numpy()
    fd.debug_fail_allocs(1)
    with pytest.raises(fd.FddpdError) as e:        # the host path's staging buffers
        c.plan.update_host(hs, hH, hpa, hth, 1e-3, 1, fd.FDDPD_GD)
    assert e.value.code == fd.FDDPD_ERR_NOMEM
    assert np.array_equal(hth, w.theta)            # theta untouched
    c.plan.update_host(hs, hH, hpa, hth, 1e-3, 1, fd.FDDPD_GD)
    assert not np.array_equal(hth, w.theta)
    fd.debug_fail_allocs(0)


def test_nan_inputs():
    import paper_2205_05158_gb300 as fd
    T = torch()
    c = Case(small_cfg(), fc_scale=0.3, precision=1)
    c.gpu_zf()
    y_ok, m_ok = c.gpu_distort()
    Hn = c.H.clone()
    Hn[0, 3, 1, 5] = float("nan")
    with pytest.raises(fd.FddpdError) as e:
        c.plan.precode(Hn, c.W, c.alpha)
    assert e.value.code == fd.FDDPD_ERR_SINGULAR
    c.gpu_zf()                                     # the clean channel again
    s_clean = c.s.clone()
    c.s[2, 1, 7] = complex(float("nan"), 0.0)
    _, m_nan = c.gpu_distort()
    assert np.isnan(m_nan[0])
    c.s.copy_(s_clean)
    y2, m2 = c.gpu_distort()
    assert nmse(y2, y_ok) == 0.0 and np.array_equal(m2, m_ok)
