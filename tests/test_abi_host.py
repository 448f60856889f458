"""C-ABI library: it loads, exports every declared entry point, and rejects bad
arguments on the host before any device work (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2205_05158_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fddpd_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_library_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert decl, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fddpd_[a-z_0-9]+)", out))
    assert decl <= exported, decl - exported
    assert set(binding.EXPORTED) == decl
    for name in decl:
        assert getattr(lib, name) is not None


def _create(lib, **over):
    d = dict(M=16, K=2, N=64, N_d=48, first_bin=-1, S_per_real=10, max_symbols=10, precision=0, P_T=10.0)
    pa = dict(orders=[1, 3], L=0, G_pa=0)
    dpd = dict(G=7, L_U=1, K_C=3, K_S=1, N_conv=2, residual=1, per_user=0)
    for k, v in over.items():
        (d if k in d else pa if k in pa else dpd)[k] = v
    dims = binding.Dims(d["M"], d["K"], d["N"], d["N_d"], d["first_bin"], d["S_per_real"], d["max_symbols"],
                        d["precision"], d["P_T"])
    pad = binding.PaDesc()
    pad.n_orders = len(pa["orders"])
    for i, p in enumerate(pa["orders"]):
        pad.orders[i] = p
    pad.L = pa["L"]
    pad.G = pa["G_pa"]
    dd = binding.DpdDesc(dpd["G"], dpd["L_U"], dpd["K_C"], dpd["K_S"], dpd["N_conv"], dpd["residual"],
                         dpd["per_user"])
    h = C.c_void_p()
    rc = lib.fddpd_plan_create(C.byref(h), C.byref(dims), C.byref(pad), C.byref(dd), None)
    return rc, h


@pytest.mark.parametrize("over,code", [
    (dict(M=0), binding.FDDPD_ERR_ARG), (dict(K=40), binding.FDDPD_ERR_ARG), (dict(K=20, M=16), binding.FDDPD_ERR_ARG),
    (dict(N=100), binding.FDDPD_ERR_UNSUPPORTED), (dict(N=8192), binding.FDDPD_ERR_UNSUPPORTED),
    (dict(N_d=65), binding.FDDPD_ERR_ARG), (dict(N_d=0), binding.FDDPD_ERR_ARG),
    (dict(first_bin=64), binding.FDDPD_ERR_ARG), (dict(S_per_real=0), binding.FDDPD_ERR_ARG),
    (dict(max_symbols=0), binding.FDDPD_ERR_ARG), (dict(max_symbols=2 ** 31 // 16 + 1), binding.FDDPD_ERR_ARG),
    (dict(P_T=0.0), binding.FDDPD_ERR_ARG),
    (dict(precision=7), binding.FDDPD_ERR_ARG), (dict(G=6), binding.FDDPD_ERR_ARG),
    (dict(L_U=3), binding.FDDPD_ERR_ARG), (dict(K_C=2), binding.FDDPD_ERR_ARG),
    (dict(N_conv=0), binding.FDDPD_ERR_ARG), (dict(residual=2), binding.FDDPD_ERR_ARG),
    (dict(orders=[-1]), binding.FDDPD_ERR_ARG), (dict(L=9), binding.FDDPD_ERR_ARG),
    # order 0 is the linear-clipping PA: alone and memoryless only
    (dict(orders=[0, 3]), binding.FDDPD_ERR_ARG), (dict(orders=[0], L=1), binding.FDDPD_ERR_ARG),
    # cross terms of Eq. 9: G in 0..2, none for the clipping PA
    (dict(G_pa=3), binding.FDDPD_ERR_ARG), (dict(G_pa=-1), binding.FDDPD_ERR_ARG),
    (dict(orders=[0], G_pa=1), binding.FDDPD_ERR_ARG),
    # per-user FD-CNN parameters: 0 or 1, FP32 plans with one input user each
    (dict(per_user=2), binding.FDDPD_ERR_ARG),
])
def test_plan_rejects_bad_descriptors(lib, over, code):
    rc, h = _create(lib, **over)
    assert rc == code
    assert not h.value
    assert lib.fddpd_last_error(None)


def test_null_plan_calls(lib):
    assert lib.fddpd_plan_destroy(None) == 0
    assert lib.fddpd_precode(None, 1, None, None, None) == binding.FDDPD_ERR_ARG
    assert lib.fddpd_distort(None, 1, *([None] * 8)) == binding.FDDPD_ERR_ARG
    assert lib.fddpd_theta_len(None) == 0


PLAN_CALLS = ["fddpd_set_stream", "fddpd_precode", "fddpd_distort", "fddpd_backward", "fddpd_update",
              "fddpd_reset_optimizer", "fddpd_update_host", "fddpd_profile_enable", "fddpd_profile_read",
              "fddpd_sync", "fddpd_set_option", "fddpd_set_power", "fddpd_invalidate_operands", "fddpd_ser",
              "fddpd_autotune", "fddpd_apply_gradient"]


@pytest.mark.parametrize("name", PLAN_CALLS)
def test_every_plan_call_rejects_a_null_plan(lib, name):
    """Every entry point that takes a plan returns FDDPD_ERR_ARG for NULL before any
    device work (the remaining arguments are placeholders of their declared types)."""
    f = getattr(lib, name)
    args = [None]
    for t in f.argtypes[1:]:
        if t in (C.c_float, C.c_double):
            args.append(1.0)
        elif t in (C.c_int, C.c_ulonglong):
            args.append(1)
        else:
            args.append(None)
    assert f(*args) == binding.FDDPD_ERR_ARG


def test_plan_free_calls_reject_bad_arguments(lib):
    out = C.c_void_p()
    assert lib.fddpd_graph_begin(None) == binding.FDDPD_ERR_ARG      # the default stream cannot record
    assert lib.fddpd_graph_end(None, C.byref(out)) == binding.FDDPD_ERR_ARG
    assert lib.fddpd_graph_launch(None, None) == binding.FDDPD_ERR_ARG
    assert lib.fddpd_graph_destroy(None) == 0
    assert lib.fddpd_precode_noalloc(0, 1, 1, 1, 1.0, None, None, None, None) == binding.FDDPD_ERR_ARG
    assert lib.fddpd_precode_noalloc(8, 2, 4, 1, 0.0, None, None, None, None) == binding.FDDPD_ERR_ARG
    assert lib.fddpd_tc_gemm(-1, 1, 1, None, 1, None, 1, None, 1, 0, 1, None) == binding.FDDPD_ERR_ARG
    assert lib.fddpd_stage_name(-1) is None and lib.fddpd_stage_name(10 ** 6) is None
    assert lib.fddpd_launch_count(None) == 0 and lib.fddpd_workspace_bytes(None) == 0
