"""The benchmark's own training step against the FP64 oracle.

System: M = 128 antennas, K = 16 users, N = 2048 with N_d = 1200 data subcarriers, the
memory-polynomial PAs (orders 1, 3, 5, taps 0..3), FD-CNN G = 35, on 28 symbols (two
channel realisations of 14).  Each plan runs the GPU's own zero-forcing build
(fddpd_precode), then fddpd_backward and one GD step of fddpd_update, in the arithmetic
the benchmark times: BF16 with tensor-core contractions and x(t) recomputed in the
adjoint (the default), BF16 with x(t) kept in BF16 and an FP32 Gram factor (the faster
variant), FP16, and FP32.  The oracle's gradient (Sec. V-A, the training criterion) is
the reference.  Tolerances: 16-bit plans relative L2 <= 2e-2 overall and per parameter
block (BF16 keeps 8 significant bits), EVM within 0.1 dB; FP32 <= 1e-4 overall and 1e-3
per block (FP32 sums of O(10^5) terms), loss within 1e-6.
"""
import functools

import numpy as np
import pytest

import oracle
import synth
from gpu_common import dev, rel_l2, torch

pytestmark = pytest.mark.gpu

S = 28
LR = 1.0   # a step far above theta's FP32 spacing


@functools.lru_cache(maxsize=1)
def _reference():
    cfg = synth.CONFIGS["m128_k16_n2048"].with_(S=S)
    w = synth.make_workload(cfg, fc_scale=0.05)
    d = oracle.dims_from_config(cfg, w.P_T)
    Wo, alo = oracle.precode(d, w.H)
    go, meto = oracle.backward(d, w.s, w.H, Wo, alo, w.pa, w.theta)
    return cfg, w, go, meto


def _blocks(cfg):
    sz = synth.theta_sizes(cfg)
    out, o = {}, 0
    for k, n in sz.items():
        out[k] = slice(o, o + n)
        o += n
    return out


VARIANTS = [
    # name, precision, options
    ("bf16", 1, {}),
    ("bf16_kept_fp32factor", 1, {"FDDPD_OPT_KEEP_PA_INPUT": 1, "FDDPD_OPT_FACTOR_FP64": 0}),
    ("fp16", 2, {}),
    ("fp32", 0, {}),
]


@pytest.mark.parametrize("name,prec,opts", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_bench_step_gradient_and_update(name, prec, opts):
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg, w, go, meto = _reference()
    plan = fd.Plan.from_config(cfg, w.P_T, max_symbols=S, precision=prec)
    for k, v in opts.items():
        plan.set_option(getattr(fd, k), v)
    s, H, pa, theta = dev(w.s), dev(w.H), dev(w.pa), dev(w.theta)
    R = w.H.shape[0]
    W = T.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    al = T.empty((R, cfg.N_d), dtype=T.float32, device="cuda")
    plan.precode(H, W, al)
    g = T.empty(plan.theta_len, dtype=T.float32, device="cuda")
    met = T.zeros(5, dtype=T.float64, device="cuda")
    plan.backward(s, H, W, al, pa, theta, g, met)
    plan.sync()
    g, met = g.cpu().numpy().astype(np.float64), met.cpu().numpy()
    tol, tol_blk = (1e-4, 1e-3) if prec == 0 else (2e-2, 2e-2)
    assert np.isfinite(g).all()
    assert rel_l2(g, go) <= tol, (name, rel_l2(g, go))
    for blk, sl in _blocks(cfg).items():
        assert rel_l2(g[sl], go[sl]) <= tol_blk, (name, blk, rel_l2(g[sl], go[sl]))
    if prec == 0:
        assert abs(met[0] - meto[0]) <= 1e-6 * meto[0]
    else:
        assert abs(met[0] - meto[0]) <= 1e-2 * meto[0]
        assert abs(oracle.evm_db(met) - oracle.evm_db(meto)) <= 0.1
        assert abs(oracle.acpr_db(met) - oracle.acpr_db(meto)) <= 0.2
    # one GD step: theta - lr * grad
    th0 = theta.clone()
    plan.update(s, H, W, al, pa, theta, LR, 1, fd.FDDPD_GD)
    plan.sync()
    step = (theta - th0).cpu().numpy().astype(np.float64)
    assert rel_l2(step, -LR * go) <= tol, (name, rel_l2(step, -LR * go))


def test_keep_option_matches_recompute_bf16():
    """The kept BF16 x(t) and the recomputed FP32 x(t) give the same gradient up to the
    BF16 rounding of the PA input."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg, w, go, _ = _reference()
    plan = fd.Plan.from_config(cfg, w.P_T, max_symbols=S, precision=fd.FDDPD_BF16)
    s, H, pa, theta = dev(w.s), dev(w.H), dev(w.pa), dev(w.theta)
    R = w.H.shape[0]
    W = T.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    al = T.empty((R, cfg.N_d), dtype=T.float32, device="cuda")
    plan.precode(H, W, al)
    out = []
    for keep in (0, 1, 0):
        plan.set_option(fd.FDDPD_OPT_KEEP_PA_INPUT, keep)
        g = T.empty(plan.theta_len, dtype=T.float32, device="cuda")
        plan.backward(s, H, W, al, pa, theta, g)
        plan.sync()
        out.append(g.cpu().numpy().astype(np.float64))
    assert rel_l2(out[2], out[0]) <= 1e-6          # switching back: the same arithmetic
    assert rel_l2(out[1], out[0]) <= 2e-2
    assert rel_l2(out[1], go) <= 2e-2


def test_zf_residual_fp64_check():
    """fddpd_zf_residual against the same FP64 definition in numpy on a sample of
    subcarriers, and on a precoder with one planted error."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg, w, _, _ = _reference()
    plan = fd.Plan.from_config(cfg, w.P_T, max_symbols=S, precision=fd.FDDPD_BF16)
    H = dev(w.H)
    R = w.H.shape[0]
    W = T.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    al = T.empty((R, cfg.N_d), dtype=T.float32, device="cuda")
    plan.precode(H, W, al)
    every = 7
    r_gpu = plan.zf_residual(H, W, every)
    Hn = w.H.reshape(-1, cfg.K, cfg.M).astype(np.complex128)
    Wn = W.cpu().numpy().reshape(-1, cfg.M, cfg.K).astype(np.complex128)
    idx = np.arange(0, Hn.shape[0], every)
    E = np.einsum("bkm,bmj->bkj", Hn[idx], Wn[idx]) - np.eye(cfg.K)[None]
    r_np = float(np.abs(E).max())
    assert 0 < r_gpu <= 1e-3                    # the W of a 16-bit plan (FP32 array)
    assert abs(r_gpu - r_np) <= 1e-9 * max(r_np, 1e-12) + 1e-15
    # a planted error on a checked subcarrier shows up as its size times |h|
    Wp = W.clone()
    b = idx[5]
    Wp.view(-1, cfg.M, cfg.K)[b, 3, 2] += 0.01
    r_planted = plan.zf_residual(H, Wp, every)
    Wpn = Wp.cpu().numpy().reshape(-1, cfg.M, cfg.K).astype(np.complex128)
    Ep = Hn[b] @ Wpn[b] - np.eye(cfg.K)
    assert abs(r_planted - max(r_np, float(np.abs(Ep).max()))) <= 1e-9


def test_alu_peaks_measured():
    import paper_2205_05158_gb300 as fd
    p32, p32x2, p64 = fd.alu_peak("fp32"), fd.alu_peak("fp32x2"), fd.alu_peak("fp64")
    for v in (p32, p32x2, p64):
        assert np.isfinite(v) and v > 0
    assert p64 < p32 < 400 and p32x2 < 400   # below any plausible FP32 rate of one GPU


def test_options_validated():
    import paper_2205_05158_gb300 as fd
    cfg = synth.CONFIGS["m16_k2_n64"]
    plan = fd.Plan.from_config(cfg, 1.0, precision=fd.FDDPD_FP32)
    plan.set_option(fd.FDDPD_OPT_KEEP_PA_INPUT, 1)     # accepted, ignored by FP32 plans
    plan.set_option(fd.FDDPD_OPT_FACTOR_FP64, 0)       # FP32 plans still factor in FP64
    for opt in (fd.FDDPD_OPT_KEEP_PA_INPUT, fd.FDDPD_OPT_FACTOR_FP64):
        with pytest.raises(fd.FddpdError) as e:
            plan.set_option(opt, 2)
        assert e.value.code == fd.FDDPD_ERR_ARG


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
def test_precoder_kept_as_factors(prec):
    """fddpd_precode(H, NULL, alpha): no W is formed; the chain applies alpha H^H (Z s) with
    Z = Y^H Y from the FP64 factor (Eq. 6 by associativity).  Forward, gradient and one
    GD step against the oracle at the 16-bit tolerances, and against the W path."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg, w, go, meto = _reference()
    plan = fd.Plan.from_config(cfg, w.P_T, max_symbols=S, precision=prec)
    s, H, pa, theta = dev(w.s), dev(w.H), dev(w.pa), dev(w.theta)
    R = w.H.shape[0]
    W = T.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    al = T.empty((R, cfg.N_d), dtype=T.float32, device="cuda")
    al2 = T.empty_like(al)
    plan.precode(H, W, al)
    y_w = T.empty_like(s)
    plan.distort(s, H, W, al, pa, theta, y_w)
    plan.precode(H, None, al2)
    assert T.equal(al, al2)
    y = T.empty_like(s)
    met = T.zeros(5, dtype=T.float64, device="cuda")
    plan.distort(s, H, None, al2, pa, theta, y, met)
    g = T.empty(plan.theta_len, dtype=T.float32, device="cuda")
    plan.backward(s, H, None, al2, pa, theta, g)
    plan.sync()
    yn, yw = y.cpu().numpy(), y_w.cpu().numpy()
    assert np.sum(np.abs(yn - yw) ** 2) / np.sum(np.abs(yw) ** 2) <= 1e-4
    m = met.cpu().numpy()
    assert abs(oracle.evm_db(m) - oracle.evm_db(meto)) <= 0.1
    assert abs(oracle.acpr_db(m) - oracle.acpr_db(meto)) <= 0.2
    g = g.cpu().numpy().astype(np.float64)
    assert rel_l2(g, go) <= 2e-2, rel_l2(g, go)
    for blk, sl in _blocks(cfg).items():
        assert rel_l2(g[sl], go[sl]) <= 2e-2, (blk, rel_l2(g[sl], go[sl]))
    th0 = theta.clone()
    plan.update(s, H, None, al2, pa, theta, LR, 1, fd.FDDPD_GD)
    plan.sync()
    step = (theta - th0).cpu().numpy().astype(np.float64)
    assert rel_l2(step, -LR * go) <= 2e-2


def test_precoder_kept_as_factors_errors():
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = synth.CONFIGS["m16_k2_n64"]
    w = synth.make_workload(cfg)
    H, s, pa, th = dev(w.H), dev(w.s), dev(w.pa), dev(w.theta)
    al = T.empty((1, cfg.N_d), dtype=T.float32, device="cuda")
    W = T.empty((1, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    p32 = fd.Plan.from_config(cfg, w.P_T, precision=fd.FDDPD_FP32)
    with pytest.raises(fd.FddpdError) as e:
        p32.precode(H, None, al)
    assert e.value.code == fd.FDDPD_ERR_UNSUPPORTED
    p16 = fd.Plan.from_config(cfg, w.P_T, precision=fd.FDDPD_BF16)
    with pytest.raises(fd.FddpdError) as e:        # no factor kept yet
        p16.distort(s, H, None, al, pa, th)
    assert e.value.code == fd.FDDPD_ERR_ARG
    p16.precode(H, W, al)                           # the W path keeps no factor
    with pytest.raises(fd.FddpdError) as e:
        p16.distort(s, H, None, al, pa, th)
    assert e.value.code == fd.FDDPD_ERR_ARG
    p16.precode(H, None, al)
    p16.distort(s, H, None, al, pa, th)             # accepted
    with pytest.raises(fd.FddpdError) as e:        # another H
        p16.distort(s, H.clone(), None, al, pa, th)
    assert e.value.code == fd.FDDPD_ERR_ARG
    p16.invalidate_operands()
    with pytest.raises(fd.FddpdError) as e:
        p16.distort(s, H, None, al, pa, th)
    assert e.value.code == fd.FDDPD_ERR_ARG
