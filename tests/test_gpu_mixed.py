"""16-bit plans (BF16 / FP16 operands on the tensor cores, FP32 accumulation, FFT and
PA in FP32) against the FP64 oracle: EVM within 0.1 dB and ACPR within 0.2 dB;
gradients within 2e-2 relative L2 (BF16 keeps 8 significant bits)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import Case, nmse, rel_l2, small_cfg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("name,mk", [
    ("ragged", lambda p: Case(small_cfg(), fc_scale=0.3, precision=p)),
    ("m64_k8_n1024_28", lambda p: Case(synth.CONFIGS["m64_k8_n1024"], S=28, fc_scale=0.2, precision=p)),
    ("m128_k16_n2048_28", lambda p: Case(synth.CONFIGS["m128_k16_n2048"].with_(S=28), fc_scale=0.05, precision=p)),
])
def test_mixed_forward_quality(name, mk, prec):
    c = mk(prec)
    c.gpu_zf()
    y, met = c.gpu_distort()
    Wo, alo = c.oracle_zf()
    yo, meto = oracle.distort(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert abs(oracle.evm_db(met) - oracle.evm_db(meto)) <= 0.1
    assert abs(oracle.acpr_db(met) - oracle.acpr_db(meto)) <= 0.2
    assert nmse(y, yo) <= 1e-4


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
def test_mixed_backward(prec):
    c = Case(small_cfg(), fc_scale=0.3, precision=prec)
    c.use_oracle_zf_on_gpu()
    g, met = c.gpu_backward()
    c.plan.sync()
    Wo, alo = c.oracle_zf()
    go, meto = oracle.backward(c.d, c.w.s, c.w.H, Wo, alo, c.w.pa, c.w.theta)
    assert rel_l2(g, go) <= 2e-2, rel_l2(g, go)
    assert abs(met[0] - meto[0]) <= 1e-2 * meto[0]


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("cfg", [small_cfg(), synth.CONFIGS["m128_k16_n2048"].with_(S=28)], ids=["ragged", "m128_k16_n2048_28"])
def test_mixed_zf_fp32_factor(cfg, prec):
    """16-bit plans set to factor the Gram matrix in FP32 (FDDPD_OPT_FACTOR_FP64 = 0): W
    and alpha (Eq. 6) still agree with the FP64 oracle far inside the 16-bit rounding
    that W undergoes afterwards."""
    import paper_2205_05158_gb300 as fd
    c = Case(cfg, S=cfg.S, precision=prec)
    c.plan.set_option(fd.FDDPD_OPT_FACTOR_FP64, 0)
    W, al = c.gpu_zf()
    Wo, alo = c.oracle_zf()
    Wg, alg = W.cpu().numpy().astype(np.complex128), al.cpu().numpy().astype(np.float64)
    assert np.abs(Wg - Wo).max() <= 1e-4 * np.abs(Wo).max()
    assert np.abs(alg - alo).max() <= 1e-4 * alo.max()


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("cfg", [small_cfg(), synth.CONFIGS["m128_k16_n2048"].with_(S=28)], ids=["ragged", "m128_k16_n2048_28"])
def test_mixed_zf_fp64_factor(cfg, prec):
    """16-bit plans factor in FP64 by default: alpha (from tr(G^-1) of the FP64 inverse
    and the FP32 Gram) within 1e-5 of the oracle's, W (split-BF16 tensor-core apply or
    FP32 CUDA-core apply of Z) within 1e-4, and the 16-bit copy only rounded after."""
    c = Case(cfg, S=cfg.S, precision=prec)
    W, al = c.gpu_zf()
    Wo, alo = c.oracle_zf()
    Wg, alg = W.cpu().numpy().astype(np.complex128), al.cpu().numpy().astype(np.float64)
    assert np.abs(Wg - Wo).max() <= 1e-4 * np.abs(Wo).max()
    assert np.abs(alg - alo).max() <= 1e-5 * alo.max()


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
def test_mixed_zf_singular_flagged(prec):
    import paper_2205_05158_gb300 as fd
    from gpu_common import dev
    c = Case(synth.CONFIGS["m16_k2_n64"], precision=prec)
    H = c.w.H.copy()
    H[0, 5, 1] = H[0, 5, 0]          # two identical users on one subcarrier
    with pytest.raises(fd.FddpdError) as e:
        c.plan.precode(dev(H), c.W, c.alpha)
    assert e.value.code == fd.FDDPD_ERR_SINGULAR

