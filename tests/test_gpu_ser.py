"""Symbol errors at the users (fddpd_ser, Sec. V-B with the noise of Eq. 4-5) against the
FP64 oracle, which draws the same Philox-4x32-10 noise with its own generator.

The noise and the decision are computed in FP32 on the GPU and in FP64 in the oracle, so
a decision may differ only where the noisy symbol lies within rounding of a decision
boundary: the tests count the oracle's symbols within 1e-4 of a level step of a boundary
and allow that many differences.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_common import Case, dev, small_cfg, torch

pytestmark = pytest.mark.gpu


def _near_boundary(z, Q, tol=1e-4):
    """Oracle symbols whose real or imaginary part is within `tol` level steps of a
    decision boundary (midpoints between levels, in the constellation's range)."""
    side = int(round(math.sqrt(Q)))
    inv_step = math.sqrt(2.0 * (Q - 1) / 3.0) / 2.0
    near = np.zeros(z.shape, dtype=bool)
    for comp in (z.real, z.imag):
        x = comp * inv_step + 0.5 * (side - 1)
        frac = x - np.floor(x)
        inside = (x > 0) & (x < side - 1)
        near |= inside & (np.abs(frac - 0.5) < tol)
    return int(near.sum())


def _gpu_ser(plan, y, s, alpha, Q, N0, seed):
    T = torch()
    counts = T.zeros(2, dtype=T.int64, device="cuda")
    plan.ser(y, s, alpha, Q, N0, seed, counts)
    T.cuda.synchronize()
    c = counts.cpu().numpy()
    return int(c[0]), int(c[1])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("snr_db", [10.0, 16.0, None], ids=["snr10", "snr16", "noiseless"])
def test_ser_matches_oracle(prec, snr_db):
    """Distorted symbols of a 16-QAM system (m16_k2_n64 with 60 symbols) through the noise and
    the decisions on both sides: equal counts up to the near-boundary symbols."""
    T = torch()
    cfg = synth.CONFIGS["m16_k2_n64"]
    c = Case(cfg, S=60, fc_scale=0.3, precision=prec)
    c.gpu_zf()
    y = T.empty_like(c.s)
    c.plan.distort(c.s, c.H, c.W, c.alpha, c.pa, c.theta, y)
    al = c.alpha.cpu().numpy()
    N0 = 0.0 if snr_db is None else float(np.mean(al ** 2)) * 10 ** (-snr_db / 10)
    e_g, n_g = _gpu_ser(c.plan, y, c.s, c.alpha, cfg.Q, N0, 2024)
    e_o, n_o, z, _ = oracle.ser(c.d, y.cpu().numpy(), c.w.s, al, cfg.Q, N0, 2024)
    assert n_g == n_o == c.w.s.size
    slack = _near_boundary(z, cfg.Q)
    assert abs(e_g - e_o) <= slack, (e_g, e_o, slack)
    if snr_db is not None:
        assert e_o > 0


@pytest.mark.parametrize("Q,snr_db", [(4, 7.0), (16, 14.0), (64, 20.0), (256, 26.0)])
def test_ser_awgn_closed_form(Q, snr_db):
    """y = s, alpha = 1: square Q-QAM in AWGN, P_s = 1 - (1 - p)^2 with
    p = 2 (1 - Q^-1/2) Q(sqrt(3 SNR / (Q - 1))), from 1.6 M symbols."""
    T = torch()
    cfg = small_cfg(K=16, N=1024, N_d=1000, S=100, S_per_real=10, Q=Q, G=32)
    c = Case(cfg, S=cfg.S)
    al = T.ones((c.R, cfg.N_d), dtype=T.float32, device="cuda")
    N0 = 10 ** (-snr_db / 10)
    e, n = _gpu_ser(c.plan, c.s, c.s, al, Q, N0, 77)
    assert n == c.w.s.size
    side = math.sqrt(Q)
    p = 2 * (1 - 1 / side) * 0.5 * math.erfc(math.sqrt(3 * 10 ** (snr_db / 10) / (Q - 1)) / math.sqrt(2))
    ps = 1 - (1 - p) ** 2
    assert abs(e / n - ps) < 4 * math.sqrt(ps * (1 - ps) / n), (e / n, ps)


def test_ser_counts_accumulate_and_errors():
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = synth.CONFIGS["m16_k2_n64"]
    c = Case(cfg, S=20)
    c.gpu_zf()
    counts = T.zeros(2, dtype=T.int64, device="cuda")
    for _ in range(2):
        c.plan.ser(c.s, c.s, c.alpha, cfg.Q, 0.5, 5, counts)
    T.cuda.synchronize()
    e1, n1 = _gpu_ser(c.plan, c.s, c.s, c.alpha, cfg.Q, 0.5, 5)
    assert counts.cpu().tolist() == [2 * e1, 2 * n1]
    with pytest.raises(fd.FddpdError) as ei:
        c.plan.ser(c.s, c.s, c.alpha, 8, 0.5, 5, counts)
    assert ei.value.code == fd.FDDPD_ERR_ARG
    with pytest.raises(fd.FddpdError) as ei:
        c.plan.ser(c.s, c.s, c.alpha, cfg.Q, -1.0, 5, counts)
    assert ei.value.code == fd.FDDPD_ERR_ARG
    raw = T.zeros(5, dtype=T.int64, device="cuda")
    with pytest.raises(fd.FddpdError) as ei:
        c.plan.ser(c.s, c.s, c.alpha, cfg.Q, 0.5, 5, raw.data_ptr() + 4)
    assert ei.value.code == fd.FDDPD_ERR_LAYOUT


def test_ser_singular_subcarriers_skipped():
    T = torch()
    cfg = synth.CONFIGS["m16_k2_n64"]
    c = Case(cfg, S=20)
    al = T.ones((c.R, cfg.N_d), dtype=T.float32, device="cuda")
    al[1, 3] = 0.0
    e, n = _gpu_ser(c.plan, c.s, c.s, al, cfg.Q, 0.0, 1)
    assert (e, n) == (0, c.w.s.size - cfg.S_per_real * cfg.K)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
def test_imperfect_csi_chain(prec):
    """Imperfect CSI (Sec. II-A): the precoder from H_est, the channel H; the GPU chain
    against the oracle given the same two channels."""
    from gpu_common import nmse
    T = torch()
    cfg = synth.CONFIGS["m16_k2_n64"]
    c = Case(cfg, S=30, fc_scale=0.3, precision=prec)
    He = synth.channel_estimate(cfg, 0.1, S=30)
    W = T.empty_like(c.W)
    al = T.empty_like(c.alpha)
    c.plan.precode(dev(He), W, al)
    y = T.empty_like(c.s)
    met = T.zeros(5, dtype=T.float64, device="cuda")
    c.plan.distort(c.s, c.H, W, al, c.pa, c.theta, y, met)
    Wo, alo = oracle.precode(c.d, He)
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert nmse(y.cpu().numpy(), yo) <= (1e-9 if prec == 0 else 1e-4)
    assert abs(oracle.evm_db(met.cpu().numpy()) - oracle.evm_db(meto)) <= (1e-3 if prec == 0 else 0.1)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
def test_clipping_pa_ser_pipeline(prec):
    """The Fig. 3 reference PA (linear clipping) through forward, noise and decisions:
    GPU counts against the oracle's on the oracle's own forward output."""
    T = torch()
    cfg = small_cfg(N=512, N_d=300, G=18, pa_nominal=synth.PA_LINEAR_CLIP, ibo_db=3.0, S=20, S_per_real=4)
    c = Case(cfg, S=cfg.S, fc_scale=0.0, precision=prec)
    c.use_oracle_zf_on_gpu()
    y, met = c.gpu_distort()
    Wo, alo = c.oracle_zf()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    from gpu_common import nmse
    assert nmse(y, yo) <= (1e-9 if prec == 0 else 1e-4)
    assert meto[3] > 0                                    # clipping spreads power into the guard bins
    N0 = float(np.mean(alo ** 2)) * 10 ** (-12 / 10)
    e_g, n_g = _gpu_ser(c.plan, dev(y.astype(np.complex64)), c.s, c.alpha, cfg.Q, N0, 9)
    e_o, n_o, z, _ = oracle.ser(c.d, y, c.w.s, c.alpha.cpu().numpy(), cfg.Q, N0, 9)
    assert n_g == n_o and abs(e_g - e_o) <= _near_boundary(z, cfg.Q)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
def test_ser_sweep_over_drive(prec):
    """SER versus PA drive (the structure of Fig. 3) with the linear-clipping PA and fixed
    N0: at each P_T the GPU's PA output power and error count against the oracle's own
    precoder, forward chain and noise; the curve falls while noise dominates and rises
    again once clipping dominates.  The slack counts the oracle's symbols within the
    forward chain's error of a decision boundary (2e-3 level steps in FP32, 0.05 in BF16)."""
    import paper_2205_05158_gb300 as fd
    cfg = small_cfg(N=512, N_d=300, G=18, pa_nominal=synth.PA_LINEAR_CLIP, S=20, S_per_real=4, Q=16, ibo_db=0.0)
    c = Case(cfg, S=cfg.S, fc_scale=0.0, precision=prec)
    P0 = synth.transmit_power(cfg)
    P_Ts = [P0 * 10 ** (-ibo / 10) for ibo in (18, 12, 6, 0)]
    N0 = 1.0
    res = c.plan.ser_sweep(c.s, c.H, c.pa, c.theta, P_Ts, cfg.Q, N0, 5)
    assert c.plan.P_T == c.w.P_T
    tol = 2e-3 if prec == 0 else 0.05
    ser_o = []
    for r, P_T in zip(res, P_Ts):
        d = oracle.dims_from_config(cfg, P_T, 1)
        Wo, alo = oracle.precode(d, c.w.H)
        yo, meto = oracle.distort(d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
        e_o, n_o, z, _ = oracle.ser(d, yo, c.w.s, alo, cfg.Q, N0, 5)
        P_PA_o = (meto[3] + meto[4]) / (cfg.M * cfg.S * cfg.N)
        assert r["symbols"] == n_o == c.w.s.size
        assert abs(r["P_PA"] - P_PA_o) <= (1e-4 if prec == 0 else 1e-2) * P_PA_o
        assert abs(r["errors"] - e_o) <= _near_boundary(z, cfg.Q, tol), (P_T, r["errors"], e_o)
        ser_o.append(e_o / n_o)
    ser = [r["SER"] for r in res]
    assert ser_o[0] > ser_o[1] > ser_o[2] and ser_o[3] > ser_o[2]
    assert ser[0] > ser[1] > ser[2] and ser[3] > ser[2]
    # the plan's own precoder is back at its P_T
    W = torch().empty_like(c.W)
    al = torch().empty_like(c.alpha)
    c.plan.precode(c.H, W, al)
    Wo, alo = c.oracle_zf()
    assert np.allclose(al.cpu().numpy(), alo, rtol=1e-4)
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(fd.FddpdError) as ei:
            c.plan.set_power(bad)
        assert ei.value.code == fd.FDDPD_ERR_ARG


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
def test_ser_decisions_symbol_by_symbol(prec):
    """fddpd_ser_decisions against the oracle's per-symbol wrong[]: equal at every symbol
    whose noisy value is not within 1e-4 level steps of a decision boundary, and the
    per-symbol flags add up to the counts."""
    T = torch()
    cfg = synth.CONFIGS["m16_k2_n64"]
    c = Case(cfg, S=60, fc_scale=0.3, precision=prec)
    c.gpu_zf()
    y = T.empty_like(c.s)
    c.plan.distort(c.s, c.H, c.W, c.alpha, c.pa, c.theta, y)
    al = c.alpha.cpu().numpy()
    N0 = float(np.mean(al ** 2)) * 10 ** (-12.0 / 10)
    counts = T.zeros(2, dtype=T.int64, device="cuda")
    wrong = T.full(tuple(c.s.shape), 255, dtype=T.uint8, device="cuda")
    c.plan.ser_decisions(y, c.s, c.alpha, cfg.Q, N0, 77, counts, wrong)
    T.cuda.synchronize()
    wg = wrong.cpu().numpy()
    e_o, n_o, z, wo = oracle.ser(c.d, y.cpu().numpy(), c.w.s, al, cfg.Q, N0, 77)
    side = int(round(math.sqrt(cfg.Q)))
    inv_step = math.sqrt(2.0 * (cfg.Q - 1) / 3.0) / 2.0
    near = np.zeros(z.shape, dtype=bool)
    for comp in (z.real, z.imag):
        x = comp * inv_step + 0.5 * (side - 1)
        near |= (x > 0) & (x < side - 1) & (np.abs(x - np.floor(x) - 0.5) < 1e-4)
    assert set(np.unique(wg)) <= {0, 1}
    assert np.array_equal(wg[~near], wo[~near].astype(np.uint8))
    assert int(wg.sum()) == int(counts.cpu().numpy()[0]) and e_o > 0
