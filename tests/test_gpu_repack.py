"""Re-packing a 16-bit plan's operands after H and W were rewritten in place under the
same pointers (fddpd_invalidate_operands), with the new W from the plan-free ZF entry
point: the chain then uses the new channel (16-bit tolerances against the oracle)."""
import pytest

import oracle
import synth
from gpu_common import Case, dev, nmse, small_cfg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
def test_operands_rewritten_in_place_by_noalloc(prec):
    """H and W rewritten in place under the same pointers (another channel, precoded by
    the plan-free ZF entry point): after fddpd_invalidate_operands the chain packs and
    uses the new ones (16-bit tolerances against the oracle on the new channel)."""
    import paper_2205_05158_gb300 as fd
    cfg = small_cfg()
    c = Case(cfg, fc_scale=0.3, precision=prec)
    c.gpu_zf()
    c.gpu_distort()                                   # 16-bit copies of the first channel
    H2 = synth.channel_estimate(cfg, 0.1)
    c.H.copy_(dev(H2))
    fd.precode_noalloc(c.H, c.W, c.alpha, c.w.P_T)
    c.plan.invalidate_operands()
    y, met = c.gpu_distort()
    Wo, alo = oracle.precode(c.d, H2)
    yo, meto = oracle.distort(c.d, c.w.s, H2, Wo, alo, c.w.pa, c.w.theta)
    assert nmse(y, yo) <= 1e-4
    assert abs(oracle.evm_db(met) - oracle.evm_db(meto)) <= 0.1
