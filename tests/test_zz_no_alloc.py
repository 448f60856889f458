"""The plan-free, allocation-free ZF entry point (fddpd_precode_noalloc).

It exists for callers that may not allocate device memory (a real-time pipeline that
reserves all device memory up front); its scratch is a static device array.  This file
is collected last so that a run stopping at the first failure has run everything else.
Two calls in a row, on different channels, must each reproduce fddpd_precode.
"""
import numpy as np
import pytest

import synth
from gpu_common import dev, torch

pytestmark = pytest.mark.gpu


def test_noalloc_precode_matches_plan_precode_twice():
    import paper_2205_05158_gb300 as fd
    from paper_2205_05158_gb300 import binding
    T = torch()
    cfg = synth.CONFIGS["m128_k16_n2048"].with_(S=28)            # 2 realisations x 1200 subcarriers
    outs = []
    for seed in (0, 5):
        w = synth.make_workload(cfg.with_(seed=seed))
        R = w.H.shape[0]
        H = dev(w.H)
        plan = fd.Plan.from_config(cfg, w.P_T, max_symbols=cfg.S)
        W_ref = T.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
        a_ref = T.empty((R, cfg.N_d), dtype=T.float32, device="cuda")
        plan.precode(H, W_ref, a_ref)
        outs.append((H, W_ref, a_ref, w.P_T))
    for H, W_ref, a_ref, P_T in outs:                  # two no-alloc calls in a row
        W = T.full_like(W_ref, float("nan"))
        a = T.full_like(a_ref, float("nan"))
        binding.precode_noalloc(H, W, a, P_T)
        T.cuda.synchronize()
        Wr, ar = W_ref.cpu().numpy(), a_ref.cpu().numpy()
        assert np.abs(W.cpu().numpy() - Wr).max() <= 1e-5 * np.abs(Wr).max()
        assert np.abs(a.cpu().numpy() - ar).max() <= 1e-5 * ar.max()


def test_noalloc_rejects_oversized_request():
    from paper_2205_05158_gb300 import binding
    T = torch()
    L = binding.load()
    buf = T.zeros(16, dtype=T.complex64, device="cuda")
    al = T.zeros(16, dtype=T.float32, device="cuda")
    rc = L.fddpd_precode_noalloc(128, 16, 1200, 100, 1.0, buf.data_ptr(), buf.data_ptr(), al.data_ptr(), None)
    assert rc == binding.FDDPD_ERR_UNSUPPORTED
    assert b"static" in L.fddpd_last_error(None)
