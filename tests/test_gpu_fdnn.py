"""The FD-NN comparison workload of Sec. III-C on the GPU (FP32 plan) against the FP64
oracle: the ZF precoder of every bin, and the chain -- per-user IDFT, the time-domain
network, per-user DFT, precoding of every bin, IDFT / PA / DFT, combining -- at the FP32
tolerances (NMSE of y <= 1e-9, loss within 1e-6, ACPR within 1e-3 dB); the identity
network against the FD-CNN plan with the identity predistorter."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import dev, nmse, small_cfg, torch

pytestmark = pytest.mark.gpu


def _case(cfg, out_scale=0.5, residual=1):
    import paper_2205_05158_gb300 as fd
    T = torch()
    w = synth.make_workload(cfg)
    H_all = synth.channel_all_bins(cfg)
    d = oracle.dims_from_config(cfg, w.P_T, residual=residual)
    th = synth.fdnn_theta_init(cfg, 11, out_scale=out_scale)
    plan = fd.Plan.fdnn_from_config(cfg, w.P_T, max_symbols=cfg.S, residual=residual)
    assert plan.theta_len == th.size == oracle.fdnn_theta_len(d)
    R = H_all.shape[0]
    Wa = T.empty((R, cfg.N, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    ala = T.empty((R, cfg.N), dtype=T.float32, device="cuda")
    Hd, Ha = dev(w.H), dev(H_all)
    plan.precode(Ha, Wa, ala)
    return plan, w, H_all, d, th, Hd, Ha, Wa, ala


def _run(plan, w, Hd, Wa, ala, th):
    T = torch()
    s = dev(w.s)
    y = T.empty_like(s)
    met = T.zeros(5, dtype=T.float64, device="cuda")
    plan.distort(s, Hd, Wa, ala, dev(w.pa), dev(th), y, met)
    T.cuda.synchronize()
    return y.cpu().numpy(), met.cpu().numpy()


CFGS = [
    ("ragged", small_cfg(L_U=1, K_S=1, nn_D=15, nn_layers=1)),                 # 40 x 3, N 256, 150 bins
    ("two_layers", small_cfg(L_U=1, K_S=1, nn_D=9, nn_layers=2, nn_L4=2)),
    ("m128_k16_n2048_14", synth.CONFIGS["m128_k16_n2048"].with_(S=14)),       # the benchmark system, one realisation
]


@pytest.mark.parametrize("name,cfg", CFGS, ids=[n for n, _ in CFGS])
def test_fdnn_chain_matches_oracle(name, cfg):
    plan, w, H_all, d, th, Hd, Ha, Wa, ala = _case(cfg)
    Wo, alo = oracle.precode(oracle.all_bins_dims(d), H_all)
    Wg, alg = Wa.cpu().numpy().astype(np.complex128), ala.cpu().numpy().astype(np.float64)
    assert np.abs(Wg - Wo).max() <= 1e-5 * np.abs(Wo).max()
    assert np.abs(alg - alo).max() <= 1e-5 * alo.max()
    y, met = _run(plan, w, Hd, Wa, ala, th)
    yo, meto = oracle.fdnn_distort(d, w.s, w.H, Wo, alo, w.pa, th)
    assert nmse(y, yo) <= 1e-9, nmse(y, yo)
    assert abs(met[0] - meto[0]) <= 1e-6 * meto[0]
    assert abs(oracle.acpr_db(met) - oracle.acpr_db(meto)) <= 1e-3


def test_fdnn_identity_equals_fdcnn_identity():
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = small_cfg(L_U=1, K_S=1)
    plan, w, H_all, d, th0, Hd, Ha, Wa, ala = _case(cfg, out_scale=0.0)
    y, met = _run(plan, w, Hd, Wa, ala, th0)
    p2 = fd.Plan.from_config(cfg, w.P_T, max_symbols=cfg.S)
    R = w.H.shape[0]
    W = T.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
    al = T.empty((R, cfg.N_d), dtype=T.float32, device="cuda")
    p2.precode(Hd, W, al)
    s = dev(w.s)
    y2 = T.empty_like(s)
    met2 = T.zeros(5, dtype=T.float64, device="cuda")
    p2.distort(s, Hd, W, al, dev(w.pa), dev(w.theta), y2, met2)      # theta: FC zero, the identity
    T.cuda.synchronize()
    assert nmse(y, y2.cpu().numpy()) <= 1e-10
    assert np.allclose(met, met2.cpu().numpy(), rtol=1e-5, atol=0)


def test_fdnn_plan_limits():
    import paper_2205_05158_gb300 as fd
    T = torch()
    cfg = small_cfg(L_U=1, K_S=1)
    plan, w, H_all, d, th, Hd, Ha, Wa, ala = _case(cfg)
    g = T.empty(plan.theta_len, dtype=T.float32, device="cuda")
    with pytest.raises(fd.FddpdError) as e:
        plan.backward(dev(w.s), Hd, Wa, ala, dev(w.pa), dev(th), g)
    assert e.value.code == fd.FDDPD_ERR_UNSUPPORTED
    with pytest.raises(fd.FddpdError) as e:
        plan.update(dev(w.s), Hd, Wa, ala, dev(w.pa), dev(th), 1e-3)
    assert e.value.code == fd.FDDPD_ERR_UNSUPPORTED
    with pytest.raises(fd.FddpdError) as e:
        fd.Plan(cfg.M, cfg.K, cfg.N, cfg.N_d, cfg.S_per_real, cfg.S, w.P_T, cfg.orders, cfg.L, cfg.grid,
                precision=fd.FDDPD_BF16, fdnn=(3, 15, 1))
    assert e.value.code == fd.FDDPD_ERR_UNSUPPORTED
    with pytest.raises(fd.FddpdError) as e:
        fd.Plan(cfg.M, cfg.K, cfg.N, cfg.N_d, cfg.S_per_real, cfg.S, w.P_T, cfg.orders, cfg.L, cfg.grid,
                fdnn=(3, 33, 1))
    assert e.value.code == fd.FDDPD_ERR_ARG
