"""FP64 CPU oracle for the FD-DPD chain: TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package; the library never does.  The arithmetic lives in plain C
(``oracle.c``); this module compiles it with gcc (``build()``) and marshals
numpy arrays through ctypes.  Inputs are up-cast to complex128/float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-D_GNU_SOURCE", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Dims(C.Structure):
    _fields_ = [("M", C.c_int), ("K", C.c_int), ("N", C.c_int), ("N_d", C.c_int),
                ("first_bin", C.c_int), ("S_per_real", C.c_int),
                ("n_orders", C.c_int), ("orders", C.c_int * 8), ("L", C.c_int),
                ("G", C.c_int), ("L_U", C.c_int), ("K_C", C.c_int), ("K_S", C.c_int),
                ("N_conv", C.c_int), ("residual", C.c_int), ("P_T", C.c_double), ("Gx", C.c_int),
                ("per_user", C.c_int), ("nn_L4", C.c_int), ("nn_D", C.c_int), ("nn_layers", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        P = C.c_void_p
        L.orc_num_threads.restype = C.c_int
        L.orc_dft.argtypes = [C.c_int, P, P, C.c_int]
        L.orc_zf.argtypes = [C.c_int, C.c_int, P, C.c_double, P, P]
        L.orc_precode_all.argtypes = [C.POINTER(Dims), C.c_int, P, P, P]
        L.orc_pa.argtypes = [C.c_int, P, C.c_int, P, C.c_int, P, P]
        L.orc_pa_gmp.argtypes = [C.c_int, P, C.c_int, P, C.c_int, C.c_int, P, P]
        L.orc_fdcnn.argtypes = [C.POINTER(Dims), P, P, P, P, P]
        L.orc_distort.argtypes = [C.POINTER(Dims), C.c_int, P, P, P, P, P, P, P, P]
        L.orc_backward.argtypes = [C.POINTER(Dims), C.c_int, P, P, P, P, P, P, P, P]
        L.orc_update.argtypes = [C.POINTER(Dims), C.c_int, P, P, P, P, P, P, C.c_double, C.c_int,
                                 C.c_int, P, P, C.POINTER(C.c_int), P]
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_ser.argtypes = [C.POINTER(Dims), C.c_int, P, P, P, C.c_int, C.c_double, C.c_ulonglong, P, P, P]
        L.orc_fdnn.argtypes = [C.POINTER(Dims), P, P, P]
        L.orc_fdnn_distort.argtypes = [C.POINTER(Dims), C.c_int, P, P, P, P, P, P, P, P]
        for f in ("orc_zf", "orc_precode_all", "orc_distort", "orc_backward", "orc_update", "orc_ser",
                  "orc_fdnn_distort"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().orc_num_threads()


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_dims(M, K, N, N_d, orders: Sequence[int], L, G, P_T, S_per_real=1, first_bin=None,
              L_U=1, K_C=3, K_S=1, N_conv=2, residual=1, Gx=0, per_user=0, nn_L4=3, nn_D=15,
              nn_layers=1) -> Dims:
    d = Dims()
    d.M, d.K, d.N, d.N_d = M, K, N, N_d
    d.first_bin = N - N_d // 2 if first_bin is None else first_bin
    d.S_per_real = S_per_real
    d.n_orders = len(orders)
    for i, p in enumerate(orders):
        d.orders[i] = p
    d.L, d.G, d.L_U, d.K_C, d.K_S, d.N_conv, d.residual = L, G, L_U, K_C, K_S, N_conv, residual
    d.P_T = P_T
    d.Gx = Gx
    d.per_user = per_user
    d.nn_L4, d.nn_D, d.nn_layers = nn_L4, nn_D, nn_layers
    return d


def dims_from_config(cfg, P_T: float, residual: int = 1) -> Dims:
    return make_dims(cfg.M, cfg.K, cfg.N, cfg.N_d, cfg.orders, cfg.L, cfg.grid, P_T,
                     S_per_real=cfg.S_per_real, first_bin=cfg.first_bin, L_U=cfg.L_U,
                     K_C=cfg.K_C, K_S=cfg.K_S, N_conv=cfg.N_conv, residual=residual, Gx=cfg.pa_G,
                     per_user=getattr(cfg, "per_user", 0), nn_L4=cfg.nn_L4, nn_D=cfg.nn_D,
                     nn_layers=cfg.nn_layers)


# -- single stages -----------------------------------------------------------
def dft(x, inverse: bool = False) -> np.ndarray:
    """Unitary DFT along the last axis (Eq. 2 for inverse=True), direct O(N^2)."""
    x = _c128(x)
    out = np.empty_like(x)
    N = x.shape[-1]
    for xi, oi in zip(x.reshape(-1, N), out.reshape(-1, N)):
        lib().orc_dft(N, _p(xi), _p(oi), int(inverse))
    return out


def zf(Hk, P_T: float):
    """Eq. (6) for one subcarrier: Hk [K][M] -> (W [M][K], alpha)."""
    Hk = _c128(Hk)
    K, M = Hk.shape
    W = np.empty((M, K), dtype=np.complex128)
    a = np.zeros(1)
    rc = lib().orc_zf(K, M, _p(Hk), float(P_T), _p(W), _p(a))
    if rc:
        raise np.linalg.LinAlgError("singular Gram matrix")
    return W, float(a[0])


def precode(d: Dims, H):
    """ZF for every realisation and data bin: H [R][N_d][K][M] -> W [R][N_d][M][K], alpha [R][N_d]."""
    H = _c128(H)
    R = H.shape[0]
    W = np.empty((R, d.N_d, d.M, d.K), dtype=np.complex128)
    al = np.empty((R, d.N_d))
    rc = lib().orc_precode_all(C.byref(d), R, _p(H), _p(W), _p(al))
    if rc:
        raise np.linalg.LinAlgError("singular Gram matrix")
    return W, al


def pa(x, orders: Sequence[int], coef) -> np.ndarray:
    """Memory-polynomial PA (Eq. 9, no cross terms) on one N-sample row; coef [P][L+1]."""
    x = _c128(x)
    coef = _c128(coef)
    o = np.ascontiguousarray(orders, dtype=np.int32)
    y = np.empty_like(x)
    lib().orc_pa(x.shape[-1], _p(x), len(o), _p(o), coef.shape[1] - 1, _p(coef), _p(y))
    return y


def pa_gmp(x, orders: Sequence[int], coef, Gx: int) -> np.ndarray:
    """Eq. (9) with cross terms on one N-sample row; coef [P][(L+1)(1 + 2 Gx)] laid out as
    a [P][L+1], then b [P][L+1][Gx], then c [P][L+1][Gx] (flattened per antenna)."""
    x = _c128(x)
    coef = _c128(coef).reshape(-1)
    o = np.ascontiguousarray(orders, dtype=np.int32)
    L1 = coef.size // (len(o) * (1 + 2 * Gx))
    y = np.empty_like(x)
    lib().orc_pa_gmp(x.shape[-1], _p(x), len(o), _p(o), L1 - 1, int(Gx), _p(coef), _p(y))
    return y


def theta_len(d: Dims) -> int:
    Go = -(-d.G // d.K_S)
    F = d.N_conv * Go * Go
    one = d.N_conv * 2 * d.L_U * d.K_C * d.K_C + d.N_conv + 2 * d.N_d * F + 2 * d.N_d
    return one * (d.K if d.per_user else 1)


def fdcnn(d: Dims, s_sym, theta):
    """FD-CNN of one symbol: s_sym [K][N_d] -> (s_tilde [K][N_d], pre [K][F], act [K][F])."""
    s_sym = _c128(s_sym)
    th = _f64(theta)
    if th.size != theta_len(d):
        raise ValueError(f"theta has {th.size} entries, expected {theta_len(d)}")
    Go = -(-d.G // d.K_S)
    F = d.N_conv * Go * Go
    st = np.empty_like(s_sym)
    pre = np.empty((d.K, F))
    act = np.empty((d.K, F))
    lib().orc_fdcnn(C.byref(d), _p(s_sym), _p(th), _p(st), _p(pre), _p(act))
    return st, pre, act


# -- whole chain ---------------------------------------------------------------
def _check_chain(d: Dims, s, H, W, alpha, pa_coef, theta):
    """Shapes the C routines index without bounds checks: s [S][K][N_d], H [R][N_d][K][M],
    W [R][N_d][M][K], alpha [R][N_d] with R covering the S symbols' realisations, the PA
    coefficients [M][n_orders][L + 1] and theta."""
    S = s.shape[0]
    R = -(-S // d.S_per_real)
    pa_shape = (d.M, d.n_orders, d.L + 1) if d.Gx == 0 else (d.M, d.n_orders * (d.L + 1) * (1 + 2 * d.Gx))
    want = {"s": (s.shape, (S, d.K, d.N_d)), "pa": (pa_coef.shape, pa_shape)}
    for name, (got, exp) in want.items():
        if tuple(got) != exp:
            raise ValueError(f"{name} has shape {tuple(got)}, expected {exp}")
    for name, a, tail in (("H", H, (d.N_d, d.K, d.M)), ("W", W, (d.N_d, d.M, d.K)), ("alpha", alpha, (d.N_d,))):
        if tuple(a.shape[1:]) != tail or a.shape[0] < R:
            raise ValueError(f"{name} has shape {tuple(a.shape)}, expected ({R}+, {', '.join(map(str, tail))})")
    if theta.size != theta_len(d):
        raise ValueError(f"theta has {theta.size} entries, expected {theta_len(d)}")


def distort(d: Dims, s, H, W, alpha, pa_coef, theta):
    """Forward chain over S symbols -> (y_eq [S][K][N_d], metrics[5])."""
    s, H, W, pa_coef = _c128(s), _c128(H), _c128(W), _c128(pa_coef)
    alpha, th = _f64(alpha), _f64(theta)
    _check_chain(d, s, H, W, alpha, pa_coef, th)
    y = np.empty_like(s)
    met = np.zeros(5)
    rc = lib().orc_distort(C.byref(d), s.shape[0], _p(s), _p(H), _p(W), _p(alpha), _p(pa_coef),
                           _p(th), _p(y), _p(met))
    if rc:
        raise ValueError("bad dims")
    return y, met


def backward(d: Dims, s, H, W, alpha, pa_coef, theta):
    """Gradient of the mean-squared symbol error w.r.t. theta -> (grad, metrics[5])."""
    s, H, W, pa_coef = _c128(s), _c128(H), _c128(W), _c128(pa_coef)
    alpha, th = _f64(alpha), _f64(theta)
    _check_chain(d, s, H, W, alpha, pa_coef, th)
    g = np.zeros(theta_len(d))
    met = np.zeros(5)
    rc = lib().orc_backward(C.byref(d), s.shape[0], _p(s), _p(H), _p(W), _p(alpha), _p(pa_coef),
                            _p(th), _p(g), _p(met))
    if rc:
        raise ValueError("bad dims")
    return g, met


class AdamState:
    def __init__(self, n: int):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = C.c_int(0)


def update(d: Dims, s, H, W, alpha, pa_coef, theta, lr: float, iters: int, adam: Optional[AdamState] = None):
    """`iters` x (forward, adjoint, step); returns (theta_new, metrics of the last forward)."""
    s, H, W, pa_coef = _c128(s), _c128(H), _c128(W), _c128(pa_coef)
    alpha = _f64(alpha)
    th = _f64(theta).copy()
    _check_chain(d, s, H, W, alpha, pa_coef, th)
    met = np.zeros(5)
    st = adam if adam is not None else AdamState(1)
    rc = lib().orc_update(C.byref(d), s.shape[0], _p(s), _p(H), _p(W), _p(alpha), _p(pa_coef),
                          _p(th), float(lr), int(iters), int(adam is not None), _p(st.m), _p(st.v),
                          C.byref(st.t), _p(met))
    if rc:
        raise ValueError("bad dims")
    return th, met


# -- the FD-NN comparison workload (Sec. III-C) -----------------------------------
def fdnn_theta_len(d: Dims) -> int:
    """W_0 [D][2U(L_4+1)], b_0 [D], (W_k [D][D], b_k [D]) x (K^NN - 1), W_o [2U][D], b_o [2U]."""
    U, L1, D = d.K, d.nn_L4 + 1, d.nn_D
    return D * 2 * U * L1 + D + (d.nn_layers - 1) * (D * D + D) + 2 * U * D + 2 * U


def all_bins_dims(d: Dims) -> Dims:
    """The same system with every one of the N subcarriers taken as a data bin (in FFT bin
    order): the geometry of the ZF precoder of all bins that the FD-NN chain needs."""
    e = Dims.from_buffer_copy(d)
    e.N_d, e.first_bin = d.N, 0
    return e


def fdnn(d: Dims, s_sym, theta) -> np.ndarray:
    """FD-NN of one symbol (Sec. III-C): s_sym [K][N_d] -> predistorted [K][N] on every bin."""
    s_sym = _c128(s_sym)
    th = _f64(theta)
    if s_sym.shape != (d.K, d.N_d):
        raise ValueError(f"s_sym has shape {s_sym.shape}, expected ({d.K}, {d.N_d})")
    if th.size != fdnn_theta_len(d):
        raise ValueError(f"theta has {th.size} entries, expected {fdnn_theta_len(d)}")
    out = np.empty((d.K, d.N), dtype=np.complex128)
    lib().orc_fdnn(C.byref(d), _p(s_sym), _p(th), _p(out))
    return out


def fdnn_distort(d: Dims, s, H, W_all, alpha_all, pa_coef, theta):
    """FD-NN chain over S symbols: FD-NN, ZF precoding of every subcarrier (W_all
    [R][N][M][K], alpha_all [R][N] by FFT bin), IDFT, PA, DFT, combining at the data bins
    (H [R][N_d][K][M]) -> (y [S][K][N_d], metrics[5])."""
    s, H, W_all, pa_coef = _c128(s), _c128(H), _c128(W_all), _c128(pa_coef)
    alpha_all, th = _f64(alpha_all), _f64(theta)
    S = s.shape[0]
    R = -(-S // d.S_per_real)
    if s.shape[1:] != (d.K, d.N_d) or H.shape[1:] != (d.N_d, d.K, d.M) or H.shape[0] < R:
        raise ValueError("s / H shapes")
    if W_all.shape[1:] != (d.N, d.M, d.K) or W_all.shape[0] < R or alpha_all.shape[1:] != (d.N,) \
            or alpha_all.shape[0] < R:
        raise ValueError("W_all / alpha_all must cover every bin of the symbols' realisations")
    if th.size != fdnn_theta_len(d):
        raise ValueError(f"theta has {th.size} entries, expected {fdnn_theta_len(d)}")
    y = np.empty_like(s)
    met = np.zeros(5)
    rc = lib().orc_fdnn_distort(C.byref(d), S, _p(s), _p(H), _p(W_all), _p(alpha_all), _p(pa_coef), _p(th),
                                _p(y), _p(met))
    if rc:
        raise ValueError("bad dims")
    return y, met


# -- symbol errors at the users (Sec. V-B) -------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """The oracle's own Philox-4x32-10 (C): ctr uint32[4], key uint32[2] -> uint32[4]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def ser(d: Dims, y, s, alpha, Q: int, N0: float, seed: int):
    """Noisy equalised symbols z = y + w / alpha (w ~ CN(0, N0) from Philox-4x32-10),
    nearest-point Q-QAM decisions against s -> (errors, compared, z, wrong[S][K][N_d])."""
    y, s = _c128(y), _c128(s)
    alpha = _f64(alpha)
    if y.shape != s.shape or y.ndim != 3 or y.shape[1:] != (d.K, d.N_d):
        raise ValueError(f"y / s shapes {y.shape} / {s.shape}, expected (S, {d.K}, {d.N_d})")
    R = -(-y.shape[0] // d.S_per_real)
    if alpha.shape[0] < R or alpha.shape[1:] != (d.N_d,):
        raise ValueError(f"alpha has shape {alpha.shape}, expected ({R}+, {d.N_d})")
    z = np.empty_like(y)
    wrong = np.zeros(y.shape, dtype=np.int32)
    counts = np.zeros(2, dtype=np.int64)
    rc = lib().orc_ser(C.byref(d), y.shape[0], _p(y), _p(s), _p(alpha), int(Q), float(N0), int(seed) & (2**64 - 1),
                       _p(z), _p(wrong), _p(counts))
    if rc:
        raise ValueError("Q must be a square")
    return int(counts[0]), int(counts[1]), z, wrong


def evm_db(met) -> float:
    return 10.0 * np.log10(met[1] / met[2])


def acpr_db(met) -> float:
    return 10.0 * np.log10(met[3] / met[4])
