"""Thin ctypes binding of the fddpd C-ABI (include/fddpd.h).

Argument marshalling only: every step of the chain runs in the CUDA library.
Tensors must be contiguous CUDA tensors of the documented dtypes (complex64 for
fddpd_c32 arrays, float32, float64 for metrics); raw integer device pointers are
accepted too.  If the library is missing this module raises instead of falling
back to any other implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

from . import build as _build

FDDPD_OK = 0
FDDPD_ERR_ARG, FDDPD_ERR_LAYOUT, FDDPD_ERR_SINGULAR = -1, -2, -3
FDDPD_ERR_CUDA, FDDPD_ERR_TIMEOUT, FDDPD_ERR_UNSUPPORTED, FDDPD_ERR_NOMEM = -4, -5, -6, -7
FDDPD_FP32, FDDPD_BF16, FDDPD_FP16 = 0, 1, 2
FDDPD_GD, FDDPD_ADAM = 0, 1
FDDPD_OPT_TENSOR_CONTRACTIONS = 1
FDDPD_OPT_HOST_CHUNKS = 2
FDDPD_OPT_KEEP_PA_INPUT = 3
FDDPD_OPT_FACTOR_FP64 = 4
FDDPD_OPT_ROW_CTAS = 5
FDDPD_OPT_CONTRACTION_CTAS = 6
FDDPD_OPT_CONTRACTION_ITEM = 7

EXPORTED = ["fddpd_plan_create", "fddpd_plan_destroy", "fddpd_last_error", "fddpd_theta_len",
            "fddpd_workspace_bytes", "fddpd_set_stream", "fddpd_precode", "fddpd_distort",
            "fddpd_backward", "fddpd_update", "fddpd_reset_optimizer", "fddpd_update_host",
            "fddpd_profile_enable", "fddpd_profile_read", "fddpd_stage_name", "fddpd_launch_count",
            "fddpd_sync", "fddpd_tc_gemm", "fddpd_precode_noalloc", "fddpd_set_option", "fddpd_ser",
            "fddpd_graph_begin", "fddpd_graph_end", "fddpd_graph_launch", "fddpd_graph_destroy", "fddpd_autotune",
            "fddpd_set_power", "fddpd_invalidate_operands", "fddpd_zf_residual", "fddpd_alu_peak",
            "fddpd_get_optimizer_state", "fddpd_set_optimizer_state", "fddpd_fdnn_plan_create", "fddpd_get_option",
            "fddpd_autotune_forget", "fddpd_graph_begin_lanes", "fddpd_ser_decisions", "fddpd_selftest_wait",
            "fddpd_debug_fail_allocs", "fddpd_apply_gradient"]

STAGES = ["zf_gram", "zf_factor", "zf_apply", "conv_fwd", "fc_fwd", "precode", "fftpa_fwd", "combine", "adj_combine", "fftpa_adj",
          "adj_precode", "fc_bwd_w", "fc_bwd_b", "fc_bwd_d", "conv_bwd", "step", "pack", "zmul", "fdnn_rows",
          "fdnn_mlp"]


class Dims(C.Structure):
    _fields_ = [("M", C.c_int), ("K", C.c_int), ("N", C.c_int), ("N_d", C.c_int), ("first_bin", C.c_int),
                ("S_per_real", C.c_int), ("max_symbols", C.c_int), ("precision", C.c_int), ("P_T", C.c_double)]


class PaDesc(C.Structure):
    _fields_ = [("n_orders", C.c_int), ("orders", C.c_int * 8), ("L", C.c_int), ("G", C.c_int)]


class DpdDesc(C.Structure):
    _fields_ = [("G", C.c_int), ("L_U", C.c_int), ("K_C", C.c_int), ("K_S", C.c_int), ("N_conv", C.c_int),
                ("residual", C.c_int), ("per_user", C.c_int)]


class FdnnDesc(C.Structure):
    _fields_ = [("L4", C.c_int), ("D", C.c_int), ("layers", C.c_int), ("residual", C.c_int)]


class FddpdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fddpd error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfddpd.so (building it with nvcc when absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} is missing; run paper_2205_05158_gb300.build.build()")
        _build.build()
    L = C.CDLL(path)
    P, I = C.c_void_p, C.c_int
    L.fddpd_plan_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Dims), C.POINTER(PaDesc), C.POINTER(DpdDesc), P]
    L.fddpd_fdnn_plan_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Dims), C.POINTER(PaDesc),
                                         C.POINTER(FdnnDesc), P]
    L.fddpd_plan_destroy.argtypes = [P]
    L.fddpd_last_error.argtypes = [P]
    L.fddpd_last_error.restype = C.c_char_p
    L.fddpd_theta_len.argtypes = [P]
    L.fddpd_theta_len.restype = C.c_size_t
    L.fddpd_workspace_bytes.argtypes = [P]
    L.fddpd_workspace_bytes.restype = C.c_size_t
    L.fddpd_set_stream.argtypes = [P, P]
    L.fddpd_precode.argtypes = [P, I, P, P, P]
    L.fddpd_distort.argtypes = [P, I, P, P, P, P, P, P, P, P]
    L.fddpd_backward.argtypes = [P, I, P, P, P, P, P, P, P, P]
    L.fddpd_update.argtypes = [P, I, P, P, P, P, P, P, C.c_float, I, I, P]
    L.fddpd_reset_optimizer.argtypes = [P]
    L.fddpd_apply_gradient.argtypes = [P, P, P, C.c_float, C.c_float, I]
    L.fddpd_update_host.argtypes = [P, I, P, P, P, P, C.c_float, I, I, P]
    L.fddpd_profile_enable.argtypes = [P, I]
    L.fddpd_profile_read.argtypes = [P, P, P]
    L.fddpd_stage_name.argtypes = [I]
    L.fddpd_stage_name.restype = C.c_char_p
    L.fddpd_launch_count.argtypes = [P]
    L.fddpd_launch_count.restype = C.c_longlong
    L.fddpd_sync.argtypes = [P]
    L.fddpd_tc_gemm.argtypes = [I, I, I, P, I, P, I, P, I, I, I, P]
    L.fddpd_precode_noalloc.argtypes = [I, I, I, I, C.c_double, P, P, P, P]
    L.fddpd_set_option.argtypes = [P, I, I]
    L.fddpd_set_power.argtypes = [P, C.c_double]
    L.fddpd_invalidate_operands.argtypes = [P]
    L.fddpd_ser.argtypes = [P, I, P, P, P, I, C.c_float, C.c_ulonglong, P]
    L.fddpd_autotune.argtypes = [P, I, P, P, P, P, P, P, I, P]
    L.fddpd_graph_begin.argtypes = [P]
    L.fddpd_graph_begin_lanes.argtypes = [P, I, C.POINTER(C.c_void_p)]
    L.fddpd_get_option.argtypes = [P, I, C.POINTER(C.c_int)]
    L.fddpd_autotune_forget.argtypes = []
    L.fddpd_ser_decisions.argtypes = [P, I, P, P, P, I, C.c_float, C.c_ulonglong, P, P]
    L.fddpd_selftest_wait.argtypes = [P, I]
    L.fddpd_debug_fail_allocs.argtypes = [I]
    L.fddpd_graph_end.argtypes = [P, C.POINTER(C.c_void_p)]
    L.fddpd_graph_launch.argtypes = [P, P]
    L.fddpd_graph_destroy.argtypes = [P]
    L.fddpd_zf_residual.argtypes = [P, I, P, P, I, P]
    L.fddpd_alu_peak.argtypes = [I, C.POINTER(C.c_double), P]
    L.fddpd_get_optimizer_state.argtypes = [P, P, P, C.POINTER(C.c_longlong)]
    L.fddpd_set_optimizer_state.argtypes = [P, P, P, C.c_longlong]
    for f in ("fddpd_plan_create", "fddpd_fdnn_plan_create", "fddpd_plan_destroy", "fddpd_set_stream", "fddpd_precode", "fddpd_distort",
              "fddpd_backward", "fddpd_update", "fddpd_reset_optimizer", "fddpd_update_host",
              "fddpd_profile_enable", "fddpd_profile_read", "fddpd_sync", "fddpd_tc_gemm",
              "fddpd_precode_noalloc", "fddpd_set_option", "fddpd_set_power",
              "fddpd_invalidate_operands", "fddpd_zf_residual", "fddpd_alu_peak", "fddpd_get_optimizer_state",
              "fddpd_set_optimizer_state", "fddpd_get_option", "fddpd_autotune_forget", "fddpd_graph_begin_lanes",
              "fddpd_ser_decisions", "fddpd_selftest_wait", "fddpd_debug_fail_allocs", "fddpd_apply_gradient"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _ptr(x, dtype=None) -> Optional[int]:
    """Device address of a contiguous CUDA tensor (or pass an int through)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {x.dtype}")
    return x.data_ptr()


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Plan:
    """Owns one fddpd_plan.  Methods mirror the C entry points one to one."""

    def __init__(self, M: int, K: int, N: int, N_d: int, S_per_real: int, max_symbols: int, P_T: float,
                 orders: Sequence[int], L: int, G: int, L_U: int = 1, K_C: int = 3, K_S: int = 1, N_conv: int = 2,
                 residual: int = 1, precision: int = FDDPD_FP32, first_bin: int = -1, stream=None,
                 pa_G: int = 0, per_user: int = 0, fdnn: Optional[Sequence[int]] = None):
        self._lib = load()
        d = Dims(M, K, N, N_d, first_bin, S_per_real, max_symbols, precision, float(P_T))
        pa = PaDesc()
        pa.n_orders = len(orders)
        for i, p in enumerate(orders):
            pa.orders[i] = int(p)
        pa.L = L
        pa.G = pa_G
        h = C.c_void_p()
        if fdnn is not None:   # the FD-NN comparison plan: fdnn = (L4, D, layers)
            nn = FdnnDesc(int(fdnn[0]), int(fdnn[1]), int(fdnn[2]), residual)
            rc = self._lib.fddpd_fdnn_plan_create(C.byref(h), C.byref(d), C.byref(pa), C.byref(nn),
                                                  _stream_ptr(stream))
        else:
            dpd = DpdDesc(G, L_U, K_C, K_S, N_conv, residual, per_user)
            rc = self._lib.fddpd_plan_create(C.byref(h), C.byref(d), C.byref(pa), C.byref(dpd), _stream_ptr(stream))
        if rc:
            raise FddpdError(rc, self._lib.fddpd_last_error(None).decode())
        self._h = h
        self.M, self.K, self.N, self.N_d, self.S_per_real = M, K, N, N_d, S_per_real
        self.precision = precision
        self.P_T = float(P_T)

    @classmethod
    def from_config(cls, cfg, P_T: float, max_symbols: Optional[int] = None, precision: int = FDDPD_FP32,
                    residual: int = 1, stream=None) -> "Plan":
        return cls(cfg.M, cfg.K, cfg.N, cfg.N_d, cfg.S_per_real, max_symbols or cfg.S, P_T, cfg.orders, cfg.L,
                   cfg.grid, cfg.L_U, cfg.K_C, cfg.K_S, cfg.N_conv, residual, precision, cfg.first_bin, stream,
                   getattr(cfg, "pa_G", 0), getattr(cfg, "per_user", 0))

    @classmethod
    def fdnn_from_config(cls, cfg, P_T: float, max_symbols: Optional[int] = None, residual: int = 1,
                         stream=None) -> "Plan":
        """The FD-NN comparison plan (Sec. III-C, fddpd_fdnn_plan_create; FP32): precode takes
        the channel of all N bins, distort the data-bin H for combining and W / alpha of
        every bin."""
        return cls(cfg.M, cfg.K, cfg.N, cfg.N_d, cfg.S_per_real, max_symbols or cfg.S, P_T, cfg.orders, cfg.L,
                   cfg.grid, residual=residual, precision=FDDPD_FP32, first_bin=cfg.first_bin, stream=stream,
                   pa_G=getattr(cfg, "pa_G", 0), fdnn=(cfg.nn_L4, cfg.nn_D, cfg.nn_layers))

    def _check(self, rc: int):
        if rc:
            raise FddpdError(rc, self._lib.fddpd_last_error(self._h).decode())

    @property
    def handle(self) -> int:
        return self._h.value

    @property
    def theta_len(self) -> int:
        return self._lib.fddpd_theta_len(self._h)

    @property
    def workspace_bytes(self) -> int:
        return self._lib.fddpd_workspace_bytes(self._h)

    def set_stream(self, stream):
        self._check(self._lib.fddpd_set_stream(self._h, _stream_ptr(stream)))

    def precode(self, H, W, alpha, R: Optional[int] = None):
        import torch
        R = H.shape[0] if R is None else R
        self._check(self._lib.fddpd_precode(self._h, R, _ptr(H, torch.complex64), _ptr(W, torch.complex64),
                                            _ptr(alpha, torch.float32)))

    def distort(self, s, H, W, alpha, pa, theta, y=None, metrics=None, S: Optional[int] = None):
        import torch
        S = s.shape[0] if S is None else S
        self._check(self._lib.fddpd_distort(self._h, S, _ptr(s, torch.complex64), _ptr(H, torch.complex64),
                                            _ptr(W, torch.complex64), _ptr(alpha, torch.float32),
                                            _ptr(pa, torch.complex64), _ptr(theta, torch.float32),
                                            _ptr(y, torch.complex64), _ptr(metrics, torch.float64)))

    def backward(self, s, H, W, alpha, pa, theta, grad, metrics=None, S: Optional[int] = None):
        import torch
        S = s.shape[0] if S is None else S
        self._check(self._lib.fddpd_backward(self._h, S, _ptr(s, torch.complex64), _ptr(H, torch.complex64),
                                             _ptr(W, torch.complex64), _ptr(alpha, torch.float32),
                                             _ptr(pa, torch.complex64), _ptr(theta, torch.float32),
                                             _ptr(grad, torch.float32), _ptr(metrics, torch.float64)))

    def update(self, s, H, W, alpha, pa, theta, lr: float, iters: int = 1, optimizer: int = FDDPD_GD, metrics=None,
               S: Optional[int] = None):
        import torch
        S = s.shape[0] if S is None else S
        self._check(self._lib.fddpd_update(self._h, S, _ptr(s, torch.complex64), _ptr(H, torch.complex64),
                                           _ptr(W, torch.complex64), _ptr(alpha, torch.float32),
                                           _ptr(pa, torch.complex64), _ptr(theta, torch.float32), float(lr),
                                           int(iters), int(optimizer), _ptr(metrics, torch.float64)))

    def apply_gradient(self, theta, grad, lr: float, optimizer: int = FDDPD_GD, scale: float = 1.0):
        """fddpd_apply_gradient: one GD / Adam step of theta from `grad` (scaled by `scale`),
        e.g. a gradient summed over data-parallel ranks with scale = 1 / ranks."""
        import torch
        self._check(self._lib.fddpd_apply_gradient(self._h, _ptr(theta, torch.float32), _ptr(grad, torch.float32),
                                                   float(scale), float(lr), int(optimizer)))

    def reset_optimizer(self):
        self._check(self._lib.fddpd_reset_optimizer(self._h))

    def checkpoint(self, theta) -> dict:
        """Training state for a later resume: theta (copied from the caller's tensor) and
        the plan's Adam moments and step counter (fddpd_get_optimizer_state), as numpy."""
        import numpy as np
        n = self.theta_len
        m = np.empty(n, dtype=np.float32)
        v = np.empty(n, dtype=np.float32)
        t = C.c_longlong(0)
        self._check(self._lib.fddpd_get_optimizer_state(self._h, m.ctypes.data, v.ctypes.data, C.byref(t)))
        return {"theta": theta.detach().cpu().numpy().copy(), "adam_m": m, "adam_v": v, "adam_t": int(t.value)}

    def restore(self, ckpt: dict, theta):
        """Resume from `checkpoint`: theta is overwritten in place, the moments and the
        step counter go back into the plan (fddpd_set_optimizer_state)."""
        import numpy as np
        import torch
        m = np.ascontiguousarray(ckpt["adam_m"], dtype=np.float32)
        v = np.ascontiguousarray(ckpt["adam_v"], dtype=np.float32)
        if m.size != self.theta_len or v.size != self.theta_len or ckpt["theta"].size != self.theta_len:
            raise ValueError("checkpoint of a plan with another theta length")
        self._check(self._lib.fddpd_set_optimizer_state(self._h, m.ctypes.data, v.ctypes.data, int(ckpt["adam_t"])))
        theta.copy_(torch.from_numpy(np.ascontiguousarray(ckpt["theta"], dtype=np.float32)))

    @staticmethod
    def save_checkpoint(path: str, ckpt: dict):
        import numpy as np
        np.savez(path, theta=ckpt["theta"], adam_m=ckpt["adam_m"], adam_v=ckpt["adam_v"],
                 adam_t=np.int64(ckpt["adam_t"]))

    @staticmethod
    def load_checkpoint(path: str) -> dict:
        import numpy as np
        with np.load(path) as z:
            return {"theta": z["theta"], "adam_m": z["adam_m"], "adam_v": z["adam_v"], "adam_t": int(z["adam_t"])}

    def set_option(self, option: int, value: int):
        """fddpd_set_option, e.g. FDDPD_OPT_TENSOR_CONTRACTIONS = 0 to run the per-subcarrier
        contractions of a 16-bit plan on CUDA cores instead of the tensor cores."""
        self._check(self._lib.fddpd_set_option(self._h, int(option), int(value)))

    def get_option(self, option: int) -> int:
        v = C.c_int(0)
        self._check(self._lib.fddpd_get_option(self._h, int(option), C.byref(v)))
        return v.value

    def invalidate_operands(self):
        """fddpd_invalidate_operands: the next call re-packs H and W (16-bit plans) --
        needed after H or W was rewritten in place other than by ``precode``."""
        self._check(self._lib.fddpd_invalidate_operands(self._h))

    def set_power(self, P_T: float):
        """fddpd_set_power: the transmit power P_T of the next precode / update_host calls."""
        self._check(self._lib.fddpd_set_power(self._h, float(P_T)))
        self.P_T = float(P_T)

    def ser_sweep(self, s, H, pa, theta, P_T_values, Q: int, N0: float, seed: int, S: Optional[int] = None):
        """SER versus drive level (Sec. V-B, the structure of Fig. 3).  For each P_T the plan
        runs the ZF precoder (fddpd_precode), the forward chain (fddpd_distort) and the
        symbol errors under receiver noise N0 (fddpd_ser); the plan's P_T is restored
        afterwards.  Returns one dict per P_T: P_T, P_PA (mean PA output power per antenna
        sample: the data- plus guard-bin power of the unitary DFT of x^PA over M S N
        samples), errors, symbols and SER."""
        import torch
        S = s.shape[0] if S is None else S
        R = (S + self.S_per_real - 1) // self.S_per_real
        dev = s.device
        W = torch.empty((R, self.N_d, self.M, self.K), dtype=torch.complex64, device=dev)
        alpha = torch.empty((R, self.N_d), dtype=torch.float32, device=dev)
        y = torch.empty_like(s)
        n = len(P_T_values)
        metrics = torch.zeros((n, 5), dtype=torch.float64, device=dev)
        counts = torch.zeros((n, 2), dtype=torch.int64, device=dev)
        P_T0 = self.P_T
        try:
            for i, P_T in enumerate(P_T_values):
                self.set_power(P_T)
                self.precode(H[:R], W, alpha, R)
                self.distort(s, H, W, alpha, pa, theta, y, metrics[i], S)
                self.ser(y, s, alpha, Q, N0, seed, counts[i], S)
        finally:
            self.set_power(P_T0)
        self._check(self._lib.fddpd_sync(self._h))
        m, c = metrics.cpu().numpy(), counts.cpu().numpy()
        out = []
        for i, P_T in enumerate(P_T_values):
            e, k = int(c[i, 0]), int(c[i, 1])
            out.append(dict(P_T=float(P_T), P_PA=float(m[i, 3] + m[i, 4]) / (self.M * S * self.N), errors=e,
                            symbols=k, SER=e / k if k else float("nan")))
        return out

    def autotune(self, s, H, W, alpha, pa, theta, reps: int = 3, S: Optional[int] = None):
        """fddpd_autotune: keeps the faster contraction implementation for this shape;
        returns the mean forward times (tensor-core, CUDA-core) in ms (-1: not admitted)."""
        import torch
        S = s.shape[0] if S is None else S
        ms = (C.c_float * 2)()
        self._check(self._lib.fddpd_autotune(self._h, S, _ptr(s, torch.complex64), _ptr(H, torch.complex64),
                                             _ptr(W, torch.complex64), _ptr(alpha, torch.float32),
                                             _ptr(pa, torch.complex64), _ptr(theta, torch.float32), int(reps), ms))
        return float(ms[0]), float(ms[1])

    def zf_residual(self, H, W, every: int = 1, out=None, R: Optional[int] = None):
        """fddpd_zf_residual: max over every `every`-th subcarrier of max |H_k W_k - I| in
        FP64; returns the host float (or writes the device float64[1] `out`, async)."""
        import torch
        R = H.shape[0] if R is None else R
        o = torch.zeros(1, dtype=torch.float64, device=H.device) if out is None else out
        self._check(self._lib.fddpd_zf_residual(self._h, R, _ptr(H, torch.complex64), _ptr(W, torch.complex64),
                                                int(every), _ptr(o, torch.float64)))
        return float(o.item()) if out is None else None

    def ser(self, y, s, alpha, Q: int, N0: float, seed: int, counts, S: Optional[int] = None):
        """fddpd_ser: adds (errors, symbols compared) of the noisy, equalised symbols
        y + w / alpha against s to `counts` (a device int64[2] tensor; asynchronous)."""
        import torch
        S = y.shape[0] if S is None else S
        self._check(self._lib.fddpd_ser(self._h, S, _ptr(y, torch.complex64), _ptr(s, torch.complex64),
                                        _ptr(alpha, torch.float32), int(Q), float(N0),
                                        int(seed) & (2 ** 64 - 1), _ptr(counts, torch.int64)))

    def ser_decisions(self, y, s, alpha, Q: int, N0: float, seed: int, counts, wrong, S: Optional[int] = None):
        """fddpd_ser_decisions: as ``ser``, and wrong (a device uint8 tensor shaped like y)
        receives 1 / 0 per symbol (2 on singular subcarriers)."""
        import torch
        S = y.shape[0] if S is None else S
        self._check(self._lib.fddpd_ser_decisions(self._h, S, _ptr(y, torch.complex64), _ptr(s, torch.complex64),
                                                  _ptr(alpha, torch.float32), int(Q), float(N0),
                                                  int(seed) & (2 ** 64 - 1), _ptr(counts, torch.int64),
                                                  _ptr(wrong, torch.uint8)))

    def selftest_wait(self, limit_us: int):
        """fddpd_selftest_wait: a bounded wait that must run out (the next sync raises
        FDDPD_ERR_TIMEOUT)."""
        self._check(self._lib.fddpd_selftest_wait(self._h, int(limit_us)))

    def update_host(self, s, H, pa, theta, lr: float, iters: int = 1, optimizer: int = FDDPD_GD, metrics=None,
                    S: Optional[int] = None):
        """Training step from host numpy arrays (complex64 / float32, C-contiguous);
        theta (and metrics, float64[5]) are updated in place."""
        import numpy as np

        def hp(a, dt):
            if a is None:
                return None
            if not (isinstance(a, np.ndarray) and a.dtype == dt and a.flags.c_contiguous):
                raise TypeError(f"expected a C-contiguous {dt} numpy array")
            return a.ctypes.data

        S = s.shape[0] if S is None else S
        self._check(self._lib.fddpd_update_host(self._h, S, hp(s, np.complex64), hp(H, np.complex64),
                                                hp(pa, np.complex64), hp(theta, np.float32), float(lr), int(iters),
                                                int(optimizer), hp(metrics, np.float64)))

    def profile(self, enable: bool = True):
        self._check(self._lib.fddpd_profile_enable(self._h, int(enable)))

    def profile_read(self):
        """{stage: (milliseconds, brackets)} since the last read (synchronises the stream)."""
        ms = (C.c_double * len(STAGES))()
        cnt = (C.c_longlong * len(STAGES))()
        self._check(self._lib.fddpd_profile_read(self._h, ms, cnt))
        return {STAGES[i]: (ms[i], cnt[i]) for i in range(len(STAGES))}

    @property
    def launch_count(self) -> int:
        return self._lib.fddpd_launch_count(self._h)

    def sync(self):
        """Synchronise the plan's stream; raises on a recorded device-side timeout."""
        self._check(self._lib.fddpd_sync(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fddpd_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_gemm(A, B, C, splits: int = 1, stream=None):
    """C (+)= A @ B.T on the tensor cores; A [M][lda], B [N][ldb] bf16/fp16 CUDA tensors
    (row strides multiples of 8), C [M][ldc] float32."""
    import torch
    L = load()
    if A.dtype != B.dtype or A.dtype not in (torch.bfloat16, torch.float16):
        raise TypeError("A and B must both be bfloat16 or both float16")
    if C.dtype != torch.float32:
        raise TypeError("C must be float32")
    M, K = A.shape
    N = B.shape[0]
    rc = L.fddpd_tc_gemm(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), C.data_ptr(), C.stride(0),
                         1 if A.dtype == torch.bfloat16 else 0, splits, _stream_ptr(stream))
    if rc:
        raise FddpdError(rc, L.fddpd_last_error(None).decode())


ALU_PEAK_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def alu_peak(kind: str, stream=None) -> float:
    """fddpd_alu_peak: measured FMA-loop peak in TFLOP/s of the FP32 pipe (kind "fp32",
    scalar fma; "fp32x2", packed pair fma) or of the FP64 pipe ("fp64")."""
    L = load()
    out = C.c_double(0.0)
    rc = L.fddpd_alu_peak(ALU_PEAK_KINDS[kind], C.byref(out), _stream_ptr(stream))
    if rc:
        raise FddpdError(rc, L.fddpd_last_error(None).decode())
    return out.value


def precode_noalloc(H, W, alpha, P_T: float, stream=None):
    """Zero-forcing precoder without a plan and without any device allocation (for
    callers that may not allocate device memory); H [R][N_d][K][M] complex64 CUDA
    tensor in, W [R][N_d][M][K] complex64 and alpha [R][N_d] float32 out."""
    import torch
    L = load()
    R, N_d, K, M = H.shape
    rc = L.fddpd_precode_noalloc(M, K, N_d, R, float(P_T), _ptr(H, torch.complex64), _ptr(W, torch.complex64),
                                 _ptr(alpha, torch.float32), _stream_ptr(stream))
    if rc:
        raise FddpdError(rc, L.fddpd_last_error(None).decode())


class Graph:
    """A CUDA graph of recorded library calls (fddpd_graph_*): calls of plans on `stream`
    made inside ``with Graph.record(stream) as g:`` are recorded, then ``g.launch()``
    replays them as one launch."""

    def __init__(self, stream):
        self._lib = load()
        self._stream = _stream_ptr(stream)
        self._h = C.c_void_p()

    @classmethod
    def record(cls, stream):
        return _Recording(cls(stream))

    @classmethod
    def record_lanes(cls, stream, lanes: int):
        """Record on `stream` and `lanes` side streams forked from it
        (fddpd_graph_begin_lanes): ``with Graph.record_lanes(s, 8) as (g, lane_streams):``
        bind plans to the lane streams (Plan.set_stream) and call them; the lanes run
        concurrently inside the one launch."""
        return _LaneRecording(cls(stream), lanes)

    def launch(self):
        rc = self._lib.fddpd_graph_launch(self._h, self._stream)
        if rc:
            raise FddpdError(rc, self._lib.fddpd_last_error(None).decode())

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.fddpd_graph_destroy(self._h)
            self._h = C.c_void_p()


class _LaneRecording:
    def __init__(self, g: Graph, lanes: int):
        self.g = g
        self.lanes = lanes

    def __enter__(self):
        arr = (C.c_void_p * self.lanes)()
        rc = self.g._lib.fddpd_graph_begin_lanes(self.g._stream, self.lanes, arr)
        if rc:
            raise FddpdError(rc, self.g._lib.fddpd_last_error(None).decode())
        return self.g, [int(arr[i]) for i in range(self.lanes)]

    def __exit__(self, exc_type, exc, tb):
        rc = self.g._lib.fddpd_graph_end(self.g._stream, C.byref(self.g._h))
        if rc and exc_type is None:
            raise FddpdError(rc, self.g._lib.fddpd_last_error(None).decode())
        return False


def debug_fail_allocs(n: int):
    """fddpd_debug_fail_allocs: the library's next n device allocations fail (NOMEM)."""
    load().fddpd_debug_fail_allocs(int(n))


def autotune_forget():
    """fddpd_autotune_forget: clear the per-shape choices of fddpd_autotune."""
    load().fddpd_autotune_forget()


class _Recording:
    def __init__(self, g: Graph):
        self.g = g

    def __enter__(self) -> Graph:
        rc = self.g._lib.fddpd_graph_begin(self.g._stream)
        if rc:
            raise FddpdError(rc, self.g._lib.fddpd_last_error(None).decode())
        return self.g

    def __exit__(self, exc_type, exc, tb):
        rc = self.g._lib.fddpd_graph_end(self.g._stream, C.byref(self.g._h))
        if rc and exc_type is None:
            raise FddpdError(rc, self.g._lib.fddpd_last_error(None).decode())
        return False
