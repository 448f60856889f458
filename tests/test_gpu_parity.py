"""Parity of the CUDA library (through its C-ABI) with the FP64 oracle.

Tolerances (FP32 plans): the equalised outputs y satisfy NMSE <= 1e-9 against the
oracle; gradients, which sum O(S K N_d) FP32 terms, agree to a relative L2 error
of 1e-4 overall and 1e-3 per parameter block; ZF precoders to 1e-5 relative.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import Case, dev, nmse, rel_l2, small_cfg, torch

pytestmark = pytest.mark.gpu

NMSE_FP32 = 1e-9
# PA shapes beyond the compiled fast paths: odd orders with memory, even orders, order 7
PA_13_MEM = {1: [1.0, 0.05 - 0.02j, 0.01, -0.004], 3: [-0.08 + 0.02j, 0.01j, -0.003, 0.001]}
PA_EVEN = {1: [1.0, 0.03j], 2: [0.02 - 0.01j, 0.004], 3: [-0.06 + 0.02j, -0.002]}
PA_1357 = {1: [1.0], 3: [-0.08 + 0.02j], 5: [-0.002 + 0.0005j], 7: [1e-4 - 2e-5j]}


def _blocks(d, g):
    ncw = d.N_conv * 2 * d.L_U * d.K_C * d.K_C
    Go = -(-d.G // d.K_S)
    nfw = 2 * d.N_d * d.N_conv * Go * Go
    return {"conv_w": g[:ncw], "conv_b": g[ncw:ncw + d.N_conv], "fc_w": g[ncw + d.N_conv:ncw + d.N_conv + nfw],
            "fc_b": g[ncw + d.N_conv + nfw:]}


# --- ZF (Eq. 6) ---------------------------------------------------------------
@pytest.mark.parametrize("cfg", [synth.CONFIGS["m16_k2_n64"], small_cfg(),
                                 synth.CONFIGS["m128_k16_n2048"].with_(S=28),
                                 small_cfg(M=96, K=16, S=6, S_per_real=2),      # K = 16 Gram, 3 chunks of 32
                                 small_cfg(M=100, K=16, S=6, S_per_real=2),     # K = 16, ragged chunk
                                 small_cfg(M=256, K=32, N=512, N_d=300, S=2, S_per_real=1, G=18)])
def test_zf_matches_oracle(cfg):
    c = Case(cfg, S=cfg.S)
    W, al = c.gpu_zf()
    Wo, alo = c.oracle_zf()
    Wg, alg = W.cpu().numpy().astype(np.complex128), al.cpu().numpy().astype(np.float64)
    assert np.abs(Wg - Wo).max() <= 1e-5 * np.abs(Wo).max()
    assert np.abs(alg - alo).max() <= 1e-5 * alo.max()
    HW = np.einsum("rbkm,rbmu->rbku", c.w.H.astype(np.complex128), Wg)
    assert np.abs(HW - np.eye(cfg.K)).max() <= 1e-4


def test_zf_singular_flagged():
    import paper_2205_05158_gb300 as fd
    cfg = synth.CONFIGS["m16_k2_n64"]
    c = Case(cfg)
    H = c.w.H.copy()
    H[0, 5, 1] = H[0, 5, 0]          # two identical users on one subcarrier
    with pytest.raises(fd.FddpdError) as e:
        c.plan.precode(dev(H), c.W, c.alpha)
    assert e.value.code == fd.FDDPD_ERR_SINGULAR


# --- forward chain ----------------------------------------------------------------
# the paper's PA model (Sec. V-A): the GMP of Eq. 9 with orders 1..7, memory 3, G = 1
PA_GMP_1TO7 = {1: [1.0, 0.05 - 0.02j, 0.01, 0.002], 2: [0.02j, 0.004, 0.0, 0.0],
               3: [-0.08 + 0.02j, 0.01j, -0.003, 0.001], 4: [0.005, 0.0, 0.0, 0.0],
               5: [-0.002 + 0.0005j, 3e-4, -1e-4, 0.0], 6: [1e-4, 0.0, 0.0, 0.0], 7: [1e-5j, 0.0, 0.0, 0.0]}


def _gmp_case(**kw):
    """A ragged system with the GMP PA: the memory polynomial of PA_GMP_1TO7 per antenna
    plus seeded lagging / leading cross terms, flattened per antenna."""
    cfg = small_cfg(N=256, pa_nominal=PA_GMP_1TO7, pa_G=1, ibo_db=10.0)
    a = synth.pa_coefficients(cfg.seed, cfg.M, cfg.pa_nominal, cfg.pa_spread)
    rng = np.random.default_rng(11)
    bc = 0.01 * (rng.standard_normal((2,) + a.shape + (1,)) + 1j * rng.standard_normal((2,) + a.shape + (1,)))
    pa = np.concatenate([a.reshape(cfg.M, -1), bc[0].reshape(cfg.M, -1), bc[1].reshape(cfg.M, -1)], axis=1)
    return Case(cfg, pa=pa, **kw)


FWD_CASES = [
    ("m16_k2_n64", lambda: Case(synth.CONFIGS["m16_k2_n64"], fc_scale=0.3)),
    ("ragged", lambda: Case(small_cfg(), fc_scale=0.3)),
    ("ragged_literal", lambda: Case(small_cfg(L_U=1, K_S=1), fc_scale=0.5, residual=0)),
    ("m64_k8_n1024_28", lambda: Case(synth.CONFIGS["m64_k8_n1024"], S=28, fc_scale=0.2)),
    ("n4096_nd_full", lambda: Case(small_cfg(M=8, K=2, N=4096, N_d=4096, S=3, S_per_real=2, G=64, L_U=1, K_S=1),
                                   fc_scale=0.05)),
    ("n64_siso", lambda: Case(small_cfg(M=1, K=1, N=64, N_d=40, S=5, S_per_real=5, G=7, L_U=1, K_S=1), fc_scale=0.3)),
    ("pa13_mem3", lambda: Case(small_cfg(N=512, pa_nominal=PA_13_MEM), fc_scale=0.3)),
    ("pa_general_even", lambda: Case(small_cfg(N=128, N_d=100, G=10, pa_nominal=PA_EVEN), fc_scale=0.3)),
    ("pa_general_1357", lambda: Case(small_cfg(N=2048, N_d=1200, M=12, G=35, pa_nominal=PA_1357), fc_scale=0.1)),
    # the ideal linear-clipping PA of Sec. V-B driven into clipping (IBO 0 dB)
    ("pa_clip", lambda: Case(small_cfg(N=512, N_d=300, G=18, pa_nominal=synth.PA_LINEAR_CLIP, ibo_db=0.0),
                             fc_scale=0.3)),
    ("pa_gmp_G1", lambda: _gmp_case(fc_scale=0.3)),
]


@pytest.mark.parametrize("name,mk", FWD_CASES, ids=[c[0] for c in FWD_CASES])
def test_distort_matches_oracle(name, mk):
    c = mk()
    c.use_oracle_zf_on_gpu()
    y, met = c.gpu_distort()
    Wo, alo = c.oracle_zf()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert nmse(y, yo) <= NMSE_FP32, nmse(y, yo)
    assert abs(oracle.evm_db(met) - oracle.evm_db(meto)) < 1e-3
    if meto[3] > 0:
        assert abs(oracle.acpr_db(met) - oracle.acpr_db(meto)) < 1e-3
    else:
        assert met[3] <= 1e-12 * met[4]
    assert abs(met[0] - meto[0]) <= 1e-4 * meto[0]
    assert abs(met[2] - meto[2]) <= 1e-6 * meto[2]


def test_end_to_end_with_gpu_zf():
    c = Case(small_cfg(), fc_scale=0.3)
    c.gpu_zf()
    y, _ = c.gpu_distort()
    Wo, alo = c.oracle_zf()
    yo, _ = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert nmse(y, yo) <= NMSE_FP32


def test_linear_pa_is_identity():
    cfg = small_cfg()
    c = Case(cfg, fc_scale=0.0, pa=synth.linear_pa(cfg))
    c.gpu_zf()
    y, met = c.gpu_distort()
    assert nmse(y, c.w.s) <= 1e-11
    assert met[3] <= 1e-10 * met[4]
    g, _ = c.gpu_backward()
    assert np.abs(g).max() <= 1e-6


# --- adjoint -----------------------------------------------------------------------
BWD_CASES = [
    ("m16_k2_n64", lambda: Case(synth.CONFIGS["m16_k2_n64"], fc_scale=0.3)),
    ("pa13_mem3", lambda: Case(small_cfg(N=512, pa_nominal=PA_13_MEM), fc_scale=0.3)),
    ("pa_general_even", lambda: Case(small_cfg(N=128, N_d=100, G=10, pa_nominal=PA_EVEN), fc_scale=0.3)),
    ("n4096", lambda: Case(small_cfg(M=8, K=2, N=4096, N_d=2400, S=3, S_per_real=2, G=49, L_U=1, K_S=1),
                           fc_scale=0.05)),
    ("ragged", lambda: Case(small_cfg(), fc_scale=0.3)),
    ("ragged_literal", lambda: Case(small_cfg(L_U=1, K_S=1), fc_scale=0.5, residual=0)),
    ("m64_k8_n1024_14", lambda: Case(synth.CONFIGS["m64_k8_n1024"], S=14, fc_scale=0.2)),
    ("pa_clip", lambda: Case(small_cfg(N=512, N_d=300, G=18, pa_nominal=synth.PA_LINEAR_CLIP, ibo_db=0.0),
                             fc_scale=0.3)),
    ("pa_gmp_G1", lambda: _gmp_case(fc_scale=0.3)),
]


@pytest.mark.parametrize("name,mk", BWD_CASES, ids=[c[0] for c in BWD_CASES])
def test_backward_matches_oracle(name, mk):
    c = mk()
    c.use_oracle_zf_on_gpu()
    g, met = c.gpu_backward()
    Wo, alo = c.oracle_zf()
    go, meto = oracle.backward(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert rel_l2(g, go) <= 1e-4, rel_l2(g, go)
    for k, (a, b) in zip(_blocks(c.d, g), zip(_blocks(c.d, g).values(), _blocks(c.d, go).values())):
        assert rel_l2(a, b) <= 1e-3, (k, rel_l2(a, b))
    assert abs(met[0] - meto[0]) <= 1e-4 * meto[0]


def test_gd_update_matches_oracle():
    import paper_2205_05158_gb300 as fd
    T = torch()
    c = Case(synth.CONFIGS["m16_k2_n64"], fc_scale=0.3)
    c.use_oracle_zf_on_gpu()
    Wo, alo = c.oracle_zf()
    th0 = c.w.theta.astype(np.float64)
    th_o, meto = oracle.update(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, th0, 1e-2, 3)
    met = T.zeros(5, dtype=T.float64, device="cuda")
    c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, 1e-2, 3, fd.FDDPD_GD, met)
    th_g = c.theta.cpu().numpy().astype(np.float64)
    assert rel_l2(th_g - th0, th_o - th0) <= 1e-4
    assert abs(met.cpu().numpy()[0] - meto[0]) <= 1e-4 * meto[0]


def test_adam_update_matches_oracle():
    import paper_2205_05158_gb300 as fd
    c = Case(synth.CONFIGS["m16_k2_n64"], fc_scale=0.3)
    c.use_oracle_zf_on_gpu()
    Wo, alo = c.oracle_zf()
    th0 = c.w.theta.astype(np.float64)
    g0, _ = oracle.backward(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, th0)
    st = oracle.AdamState(len(th0))
    th_o, _ = oracle.update(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, th0, 1e-3, 2, adam=st)
    c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, c.theta, 1e-3, 2, fd.FDDPD_ADAM)
    th_g = c.theta.cpu().numpy().astype(np.float64)
    # Adam's first steps are ~lr sign(g): compare where the gradient is not negligible
    mask = np.abs(g0) > 1e-2 * np.abs(g0).max()
    assert mask.sum() > 100
    assert rel_l2((th_g - th0)[mask], (th_o - th0)[mask]) <= 1e-3


@pytest.mark.parametrize("opt", ["gd", "adam"])
def test_apply_gradient_equals_update(opt):
    """fddpd_apply_gradient (the step of a data-parallel loop: backward, an all-reduce,
    then this) on the plan's own gradient gives fddpd_update's step bit for bit, for GD
    and over two Adam steps; a gradient passed doubled with scale 1/2 gives the same
    step (the scaling is exact)."""
    import paper_2205_05158_gb300 as fd
    T = torch()
    o = fd.FDDPD_GD if opt == "gd" else fd.FDDPD_ADAM
    lr = 1e-2 if opt == "gd" else 1e-3
    a = Case(synth.CONFIGS["m16_k2_n64"], fc_scale=0.3)
    b = Case(synth.CONFIGS["m16_k2_n64"], fc_scale=0.3)
    for c in (a, b):
        c.use_oracle_zf_on_gpu()
    g = T.empty(b.plan.theta_len, dtype=T.float32, device="cuda")
    for it in range(2):
        a.plan.update(a.s, a.H, a.W, a.alpha, a.pa, a.theta, lr, 1, o)
        b.plan.backward(b.s, b.H, b.W, b.alpha, b.pa, b.theta, g)
        g2 = g * 2.0
        b.plan.apply_gradient(b.theta, g2, lr, o, scale=0.5)
    T.cuda.synchronize()
    assert T.equal(a.theta, b.theta)
    assert not T.equal(a.theta, a.theta.new_tensor(a.w.theta))   # the steps moved theta
    with pytest.raises(fd.FddpdError):
        b.plan.apply_gradient(b.theta, g, float("nan"), o)


# --- argument errors reported by the device-facing entry points ------------------------
def test_call_argument_errors():
    import paper_2205_05158_gb300 as fd
    T = torch()
    c = Case(synth.CONFIGS["m16_k2_n64"])
    c.gpu_zf()
    with pytest.raises(fd.FddpdError) as e:
        c.plan.distort(c.s, c.H, c.W, c.alpha, c.pa, c.theta, S=c.S + 1)
    assert e.value.code == fd.FDDPD_ERR_ARG
    raw = T.empty(c.s.numel() * 2 + 1, dtype=T.float32, device="cuda")
    with pytest.raises(fd.FddpdError) as e:
        c.plan.distort(raw.data_ptr() + 4, c.H, c.W, c.alpha, c.pa, c.theta, S=c.S)
    assert e.value.code == fd.FDDPD_ERR_LAYOUT


# --- full-size 128 x 16 x 2048 workload (the benchmark's launch shape) ----------------------
@pytest.mark.slow
def test_m128_k16_n2048_full_size_sampled_symbols():
    cfg = synth.CONFIGS["m128_k16_n2048"]
    c = Case(cfg, fc_scale=0.05)
    c.gpu_zf()
    y, met = c.gpu_distort()
    Wg = c.W.cpu().numpy()
    alg = c.alpha.cpu().numpy()
    rng = np.random.default_rng(2000)
    picks = sorted(set([0, 13, 1999] + list(rng.choice(2000, 2, replace=False))))
    for t in picks:
        r = t // cfg.S_per_real
        Wo, alo = oracle.precode(c.d, c.w.H[r:r + 1])
        assert np.abs(Wg[r] - Wo[0]).max() <= 1e-5 * np.abs(Wo).max()
        assert np.abs(alg[r] - alo[0]).max() <= 1e-5 * alo.max()
        yo, _ = oracle.distort(c.d, c.w.s[t:t + 1], c.w.H[r:r + 1], Wo, alo, c.w.pa, c.w.theta)
        assert nmse(y[t:t + 1], yo) <= NMSE_FP32, (t, nmse(y[t:t + 1], yo))
    # the loss is a mean over symbols: whole = weighted halves (a property at any size)
    T = torch()
    m1 = T.zeros(5, dtype=T.float64, device="cuda")
    m2 = T.zeros(5, dtype=T.float64, device="cuda")
    half = 1008
    c.plan.distort(c.s[:half], c.H, c.W, c.alpha, c.pa, c.theta, None, m1)
    c.plan.distort(c.s[half:], c.H[half // 14:], c.W[half // 14:], c.alpha[half // 14:], c.pa, c.theta, None, m2)
    T.cuda.synchronize()
    m1, m2 = m1.cpu().numpy(), m2.cpu().numpy()
    # per-thread FP32 partial sums before the FP64 reduction: ~1e-7 relative per sum
    assert abs((m1[1] + m2[1]) - met[1]) <= 1e-6 * met[1]
    assert abs((m1[3] + m2[3]) - met[3]) <= 1e-6 * met[3]
