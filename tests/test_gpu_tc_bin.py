"""tcgen05 per-subcarrier contractions (precode, combine and their adjoints) of 16-bit
plans against the FP64 oracle and against the CUDA-core kernels with FP32 activations.

The tensor-core path also rounds the activations (s~, x, g_y, g_x) to the plan's 16-bit
type, which adds about 2^-9 relative error per BF16 operand: NMSE of y within 1e-4 of
the oracle, EVM within 0.1 dB, gradients within 2e-2 relative L2, as for the other
16-bit results.  ZF comes from the oracle so that only the contractions differ.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import Case, nmse, rel_l2, small_cfg

pytestmark = pytest.mark.gpu

CFGS = [
    ("ragged", small_cfg()),                                           # M 40, K 3, realisations of 3
    ("pad", small_cfg(M=100, K=13, S=45, S_per_real=20)),               # M % 8 = 4, K % 4 = 1, 2 symbol chunks
    ("full", small_cfg(M=128, K=16, S=33, S_per_real=14)),             # full tiles, ragged subcarrier groups
    ("m128_k16_n2048_140", synth.CONFIGS["m128_k16_n2048"].with_(S=140)),                   # several items per CTA
]
# beyond 128 antennas and 16 users: antenna parts of 128 (expand items; reduce MMAs
# accumulating in TMEM) and user halves of 16 (4 subcarriers a expand item, 32 user slots
# a tile row; reduce TMEM column blocks)
WIDE = [
    ("m256_k32", small_cfg(M=256, K=32, N=512, N_d=300, S=10, S_per_real=5, G=18)),   # whole parts and halves
    ("m200_k20", small_cfg(M=200, K=20, S=7, S_per_real=3)),                           # ragged part (72) and half (4)
    ("m250_k21", small_cfg(M=250, K=21, S=5, S_per_real=5)),                           # M % 4 = 2, K % 4 = 1
    ("m256_k8", small_cfg(M=256, K=8, S=6, S_per_real=3)),                             # two parts, one user half
    ("m136_k4", small_cfg(M=136, K=4, S=4, S_per_real=2)),                             # a second part of 8 antennas
]
CFGS = CFGS + WIDE


def _opt(c, on):
    import paper_2205_05158_gb300 as fd
    c.plan.set_option(fd.FDDPD_OPT_TENSOR_CONTRACTIONS, 1 if on else 0)


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("name,cfg", CFGS, ids=[n for n, _ in CFGS])
def test_tc_forward(name, cfg, prec):
    c = Case(cfg, S=cfg.S, fc_scale=0.3, precision=prec)
    c.use_oracle_zf_on_gpu()
    _opt(c, True)
    y_tc, met_tc = c.gpu_distort()
    _opt(c, False)
    y_cc, met_cc = c.gpu_distort()
    Wo, alo = c.oracle_zf()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert np.isfinite(y_tc).all()
    assert nmse(y_tc, yo) <= 1e-4, nmse(y_tc, yo)
    assert nmse(y_tc, y_cc) <= 1e-4, nmse(y_tc, y_cc)
    assert abs(oracle.evm_db(met_tc) - oracle.evm_db(meto)) <= 0.1
    assert abs(met_tc[0] - meto[0]) <= 1e-2 * meto[0]


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("name,cfg", CFGS[:3] + WIDE, ids=[n for n, _ in CFGS[:3] + WIDE])
def test_tc_backward(name, cfg, prec):
    c = Case(cfg, S=cfg.S, fc_scale=0.3, precision=prec)
    c.use_oracle_zf_on_gpu()
    _opt(c, True)
    g_tc, _ = c.gpu_backward()
    _opt(c, False)
    g_cc, _ = c.gpu_backward()
    Wo, alo = c.oracle_zf()
    go, _ = oracle.backward(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert np.isfinite(g_tc).all()
    assert rel_l2(g_tc, go) <= 2e-2, rel_l2(g_tc, go)
    assert rel_l2(g_tc, g_cc) <= 2e-2, rel_l2(g_tc, g_cc)


HALF_CFGS = [CFGS[0], CFGS[2], ("m128_k16_n2048_28", synth.CONFIGS["m128_k16_n2048"].with_(S=28)), WIDE[0], WIDE[2]]


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("name,cfg", HALF_CFGS, ids=[n for n, _ in HALF_CFGS])
def test_tc_half_items(name, cfg, prec):
    """Contraction items of half the subcarriers (FDDPD_OPT_CONTRACTION_ITEM = 1; for the
    128 x 16 BF16 shape the generic kernels replace the pipelined ones): forward and
    gradient against the oracle, and against whole items.  In the generic kernels every
    subcarrier's MMAs are the same either way, so their results are identical; the
    pipelined kernels of the 128 x 16 BF16 shape may round differently."""
    import paper_2205_05158_gb300 as fd
    c = Case(cfg, S=cfg.S, fc_scale=0.3, precision=prec)
    c.use_oracle_zf_on_gpu()
    _opt(c, True)
    y1, met1 = c.gpu_distort()
    g1, _ = c.gpu_backward()
    c.plan.set_option(fd.FDDPD_OPT_CONTRACTION_ITEM, 1)
    yh, meth = c.gpu_distort()
    gh, _ = c.gpu_backward()
    Wo, alo = c.oracle_zf()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    go, _ = oracle.backward(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert nmse(yh, yo) <= 1e-4 and rel_l2(gh, go) <= 2e-2
    assert abs(oracle.evm_db(meth) - oracle.evm_db(meto)) <= 0.1
    pipelined = cfg.M == 128 and cfg.K == 16 and prec == 1 and cfg.S_per_real <= 16
    if pipelined:
        assert nmse(yh, y1) <= 1e-6 and rel_l2(gh, g1) <= 1e-3
    else:
        assert np.array_equal(yh, y1) and np.array_equal(gh, g1)


def test_option_ignored_by_fp32_plans():
    c = Case(small_cfg(), fc_scale=0.3, precision=0)
    c.use_oracle_zf_on_gpu()
    _opt(c, True)
    y1, _ = c.gpu_distort()
    _opt(c, False)
    y0, _ = c.gpu_distort()
    assert np.array_equal(y1, y0)


def test_option_rejects_unknown():
    import paper_2205_05158_gb300 as fd
    c = Case(synth.CONFIGS["m16_k2_n64"], precision=1)
    with pytest.raises(fd.FddpdError) as e:
        c.plan.set_option(99, 1)
    assert e.value.code == fd.FDDPD_ERR_ARG
    with pytest.raises(fd.FddpdError):
        c.plan.set_option(fd.FDDPD_OPT_TENSOR_CONTRACTIONS, 2)


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("name,cfg", [CFGS[0], CFGS[1], ("m128_k16_n2048_28", synth.CONFIGS["m128_k16_n2048"].with_(S=28)),
                                      WIDE[0]],
                         ids=["ragged", "pad", "m128_k16_n2048_28", "m256_k32"])
def test_tc_zf_apply(name, cfg, prec):
    """W = H^H (H H^H)^{-1} (Eq. 6) from the tensor-core apply (BF16 hi / lo splits)
    against the oracle and against the CUDA-core apply; alpha comes from the same factor.
    Beyond 128 antennas or 16 users the apply stays on CUDA cores with the option on."""
    c = Case(cfg, S=cfg.S, precision=prec)
    _opt(c, True)
    W1, a1 = (x.clone() for x in c.gpu_zf())
    _opt(c, False)
    W0, a0 = (x.clone() for x in c.gpu_zf())
    Wo, alo = c.oracle_zf()
    W1n, W0n = W1.cpu().numpy().astype(np.complex128), W0.cpu().numpy().astype(np.complex128)
    assert np.array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    assert np.abs(W1n - Wo).max() <= 1e-4 * np.abs(Wo).max()
    assert np.abs(W1n - W0n).max() <= 1e-4 * np.abs(Wo).max()
    HW = np.einsum("rbkm,rbmu->rbku", c.w.H.astype(np.complex128), W1n)
    assert np.abs(HW - np.eye(cfg.K)).max() <= 1e-3


# K = 24 (the K > 16 forms of Z x and of the tensor-core contractions) with 17 symbols per realisation
# (two staged passes of symbols); 150 data bins put realisation boundaries inside 32-bin blocks
FACTOR_CFGS = CFGS[:3] + [("k24", small_cfg(M=64, K=24, S=40, S_per_real=17)), WIDE[0], WIDE[2]]


@pytest.mark.parametrize("tc", [True, False], ids=["tcgen05", "cuda_cores"])
@pytest.mark.parametrize("name,cfg", FACTOR_CFGS, ids=[n for n, _ in FACTOR_CFGS])
def test_precoder_kept_as_factors_ragged(name, cfg, tc):
    """fddpd_precode(H, NULL, alpha) on ragged shapes (K = 3, 13, 16, 24; the generic and
    the K = 16 Gram kernels write H^H; Z x with 3, 20 and 17 symbols per realisation):
    forward and gradient against the oracle."""
    c = Case(cfg, S=cfg.S, fc_scale=0.3, precision=1)
    _opt(c, tc)
    c.plan.precode(c.H, None, c.alpha)
    T = __import__("torch")
    y = T.empty_like(c.s)
    met = T.zeros(5, dtype=T.float64, device="cuda")
    c.plan.distort(c.s, c.H, None, c.alpha, c.pa, c.theta, y, met)
    g = T.empty(c.plan.theta_len, dtype=T.float32, device="cuda")
    c.plan.backward(c.s, c.H, None, c.alpha, c.pa, c.theta, g)
    c.plan.sync()
    Wo, alo = c.oracle_zf()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    go, _ = oracle.backward(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert nmse(y.cpu().numpy(), yo) <= 1e-4
    assert abs(oracle.evm_db(met.cpu().numpy()) - oracle.evm_db(meto)) <= 0.1
    assert rel_l2(g.cpu().numpy(), go) <= 2e-2
