"""Seeded synthetic inputs for the FD-DPD downlink (shared by the oracle and the GPU path).

This module draws the *inputs* of the method and nothing else: QAM symbols,
channel taps and their per-subcarrier response, per-antenna PA coefficients,
the drive level and an initial parameter vector.  It holds none of the
predistortion, precoding, OFDM, PA or loss arithmetic; the oracle and the CUDA
path each implement those on their own.  Values are produced in FP64 and then
rounded to the storage type the library consumes (complex64 / float32), so
that the oracle (which up-casts exactly) and the GPU read identical numbers.

System model (Sec. II-A): K single-antenna users, M base-station antennas,
N-point OFDM with N_d data subcarriers, a T-tap block-constant Rayleigh channel
(Eq. 3, taps of variance 1/T), and per-antenna memory-polynomial PAs (Eq. 9
with no cross terms) whose coefficients are spread around a nominal set
(Sec. V-A).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

from .philox import Stream, philox4x32_10, splitmix64  # noqa: F401

# Nominal memory-polynomial sets (rows: odd orders, columns: taps 0..L).  The
# paper's measured coefficient set is not public, so these stand in for it.
PA_NOMINAL_TOY = {1: [1.0 + 0j], 3: [-0.08 + 0.02j]}
PA_NOMINAL_MP135 = {
    1: [1.0, 0.08 - 0.04j, -0.02 + 0.01j, 0.005],
    3: [-0.08 + 0.02j, 0.012 - 0.006j, -0.004 + 0.002j, 0.001],
    5: [-0.002 + 0.0005j, 3e-4, -1e-4, 5e-5],
}


@dataclasses.dataclass
class Config:
    name: str
    M: int                      # BS antennas
    K: int                      # users
    N: int                      # OFDM size
    N_d: int                    # data subcarriers
    Q: int                      # QAM order
    S: int                      # OFDM symbols in the workload
    S_per_real: int             # symbols per channel realisation
    pa_nominal: Dict[int, List[complex]]
    pa_spread: float = 0.10     # real multiplicative spread, uniform in [-spread, spread]
    pa_spread_orders: Optional[Sequence[int]] = None   # None: every coefficient
    pa_G: int = 0               # PA cross-term length of Eq. 9 (0: memory polynomial)
    per_user: int = 0           # 1: each user its own FD-CNN parameters theta_u (Sec. IV-A)
    ibo_db: float = 6.0
    T: int = 10                 # channel taps
    rho: float = 0.0            # exponential antenna correlation
    G: int = 0                  # FD-CNN grid side (0: ceil(sqrt(N_d)))
    L_U: int = 1
    K_C: int = 3
    K_S: int = 1
    N_conv: int = 2
    nn_L4: int = 3              # FD-NN (Sec. III-C): memory length, neurons, hidden layers
    nn_D: int = 15
    nn_layers: int = 1
    iters: int = 1
    seed: int = 0

    @property
    def grid(self) -> int:
        return self.G if self.G else int(math.ceil(math.sqrt(self.N_d)))

    @property
    def first_bin(self) -> int:
        return self.N - self.N_d // 2

    @property
    def R(self) -> int:
        return (self.S + self.S_per_real - 1) // self.S_per_real

    @property
    def orders(self) -> List[int]:
        return sorted(self.pa_nominal)

    @property
    def L(self) -> int:
        return max(len(v) for v in self.pa_nominal.values()) - 1

    def with_(self, **kw) -> "Config":
        return dataclasses.replace(self, **kw)


# The workloads, named by their sizes: a 16x2 toy system, a 64x8 N=1024 system, the
# 128x16 N=2048 system of the benchmark, and the same system with 256 symbols for long
# training runs (500 iterations).
CONFIGS = {
    "m16_k2_n64": Config("m16_k2_n64", M=16, K=2, N=64, N_d=48, Q=16, S=10, S_per_real=10,
                   pa_nominal=PA_NOMINAL_TOY, pa_spread_orders=(3,), iters=3, G=7),
    "m64_k8_n1024": Config("m64_k8_n1024", M=64, K=8, N=1024, N_d=600, Q=64, S=1000, S_per_real=14,
                   pa_nominal=PA_NOMINAL_MP135, iters=4, G=25),
    "m128_k16_n2048": Config("m128_k16_n2048", M=128, K=16, N=2048, N_d=1200, Q=256, S=2000, S_per_real=14,
                   pa_nominal=PA_NOMINAL_MP135, rho=0.5, iters=1, G=35),
    "m128_k16_n2048_train": Config("m128_k16_n2048_train", M=128, K=16, N=2048, N_d=1200, Q=256, S=256, S_per_real=14,
                   pa_nominal=PA_NOMINAL_MP135, rho=0.5, iters=500, G=35),
}


def data_bins(N: int, N_d: int, first_bin: Optional[int] = None) -> np.ndarray:
    """FFT bin of data subcarrier i: a contiguous block centred on DC, in
    increasing frequency, (first_bin + i) mod N with first_bin = N - N_d/2."""
    fb = N - N_d // 2 if first_bin is None else first_bin
    return (fb + np.arange(N_d)) % N


# ----------------------------------------------------------------------------
# QAM source (Sec. II-A: i.i.d. symbols from a square Q-QAM, unit mean power)
# ----------------------------------------------------------------------------
def qam_levels(Q: int) -> np.ndarray:
    side = int(round(math.sqrt(Q)))
    if side * side != Q or side & (side - 1):
        raise ValueError("square QAM with a power-of-two side expected")
    lv = 2.0 * np.arange(side) - (side - 1)
    return lv / math.sqrt(2.0 * (Q - 1) / 3.0)


def qam_symbols(seed: int, Q: int, shape: Sequence[int], tag: str = "qam",
                offset: int = 0) -> np.ndarray:
    """Unit-power Q-QAM symbols; one 32-bit word per symbol (I in the low bits,
    Q in the next ones).  `offset` skips that many symbols of the stream."""
    side = int(round(math.sqrt(Q)))
    bits = side.bit_length() - 1
    n = int(np.prod(shape))
    st = Stream(seed, tag)
    if offset:
        st.block = offset // 4
        w = st.u32(n + offset % 4)[offset % 4:]
    else:
        w = st.u32(n)
    lv = qam_levels(Q)
    i = w & np.uint32(side - 1)
    q = (w >> np.uint32(bits)) & np.uint32(side - 1)
    return (lv[i] + 1j * lv[q]).reshape(shape)


# ----------------------------------------------------------------------------
# Channel (Eq. 3 taps; Eq. 4 per-subcarrier response of the data bins)
# ----------------------------------------------------------------------------
def _corr_sqrt(M: int, rho: float) -> np.ndarray:
    if rho == 0.0:
        return np.eye(M)
    idx = np.arange(M)
    Rm = rho ** np.abs(idx[:, None] - idx[None, :])
    return np.linalg.cholesky(Rm)


def channel_taps(seed: int, R: int, T: int, K: int, M: int, rho: float = 0.0,
                 first_real: int = 0) -> np.ndarray:
    """[R][T][K][M] complex taps, entries CN(0, 1/T); with rho > 0 each user's
    row is coloured across antennas by R_ij = rho^|i-j| (H_t = G_t R^{1/2})."""
    Lc = _corr_sqrt(M, rho)
    out = np.empty((R, T, K, M), dtype=np.complex128)
    for r in range(R):
        st = Stream(seed, f"taps/{first_real + r}")
        g = st.normal(2 * T * K * M).reshape(T, K, M, 2)
        g = (g[..., 0] + 1j * g[..., 1]) * math.sqrt(0.5 / T)
        out[r] = g @ Lc.T if rho else g
    return out


def channel_estimate(cfg: "Config", eta: float, S: Optional[int] = None, symbol_offset: int = 0) -> np.ndarray:
    """Imperfect CSI at the base station (Sec. II-A): taps H_t^est = sqrt(1 - eta) H_t +
    sqrt(eta) H_t^err with H_t^err entries CN(0, 1), as the per-subcarrier response of the
    data bins [R][N_d][K][M] (complex64) of the same realisations make_workload draws."""
    if not 0.0 <= eta <= 1.0:
        raise ValueError("eta outside [0, 1]")
    S = cfg.S if S is None else S
    r0 = symbol_offset // cfg.S_per_real
    R = (S + cfg.S_per_real - 1) // cfg.S_per_real
    bins = data_bins(cfg.N, cfg.N_d)
    out = np.empty((R, cfg.N_d, cfg.K, cfg.M), dtype=np.complex64)
    for r in range(R):
        taps = channel_taps(cfg.seed, 1, cfg.T, cfg.K, cfg.M, cfg.rho, first_real=r0 + r)
        st = Stream(cfg.seed, f"taps_err/{r0 + r}")
        g = st.normal(2 * cfg.T * cfg.K * cfg.M).reshape(1, cfg.T, cfg.K, cfg.M, 2)
        err = (g[..., 0] + 1j * g[..., 1]) * math.sqrt(0.5)
        out[r] = channel_fd(math.sqrt(1.0 - eta) * taps + math.sqrt(eta) * err, cfg.N, bins)[0]
    return out


def channel_all_bins(cfg: "Config", S: Optional[int] = None, symbol_offset: int = 0) -> np.ndarray:
    """The per-subcarrier channel of EVERY one of the N bins (natural bin order), [R][N][K][M]
    complex64, of the same realisations make_workload draws (its H is this array at the
    data bins): the precoder of the FD-NN workload covers the guard bins too."""
    S = cfg.S if S is None else S
    if symbol_offset % cfg.S_per_real:
        raise ValueError("symbol_offset must start a realisation")
    r0 = symbol_offset // cfg.S_per_real
    R = (S + cfg.S_per_real - 1) // cfg.S_per_real
    out = np.empty((R, cfg.N, cfg.K, cfg.M), dtype=np.complex64)
    bins = np.arange(cfg.N)
    for r in range(0, R, 8):
        n = min(8, R - r)
        taps = channel_taps(cfg.seed, n, cfg.T, cfg.K, cfg.M, cfg.rho, first_real=r0 + r)
        out[r:r + n] = channel_fd(taps, cfg.N, bins)
    return out


def channel_fd(taps: np.ndarray, N: int, bins: np.ndarray) -> np.ndarray:
    """Per-subcarrier channel of the data bins: H_k = sum_t H_t exp(-j 2 pi k t / N).
    taps [R][T][K][M] -> [R][N_d][K][M]."""
    R, T, K, M = taps.shape
    ph = np.exp(-2j * np.pi * np.outer(bins, np.arange(T)) / N)        # [N_d][T]
    return np.einsum("bt,rtkm->rbkm", ph, taps, optimize=True)


# ----------------------------------------------------------------------------
# PA coefficients (Sec. V-A: per-antenna coefficients spread around a nominal set)
# ----------------------------------------------------------------------------
def pa_coefficients(seed: int, M: int, nominal: Dict[int, List[complex]], spread: float,
                    spread_orders: Optional[Sequence[int]] = None) -> np.ndarray:
    """[M][P][L+1] complex: c^b_{p,l} = c_{p,l} (1 + delta), delta ~ U[-spread, spread]
    real and i.i.d. per antenna and coefficient (orders outside spread_orders fixed)."""
    orders = sorted(nominal)
    L1 = max(len(v) for v in nominal.values())
    base = np.zeros((len(orders), L1), dtype=np.complex128)
    for pi, p in enumerate(orders):
        base[pi, :len(nominal[p])] = nominal[p]
    u = Stream(seed, "pa").uniform(M * len(orders) * L1).reshape(M, len(orders), L1)
    delta = spread * (2.0 * u - 1.0)
    if spread_orders is not None:
        mask = np.array([p in spread_orders for p in orders])[None, :, None]
        delta = np.where(mask, delta, 0.0)
    return base[None] * (1.0 + delta)


PA_NOMINAL_MP13 = {p: PA_NOMINAL_MP135[p] for p in (1, 3)}


def uneven_instances(n: int, S: int = 50, seed: int = 0, S_per_real: int = 14) -> List[Config]:
    """Independent downlink instances of uneven size (the batched workload): instance i
    draws M from {32, 64, 128, 256}, K from {4, 8, 16, 32} (redrawn until K <= M / 4), N
    from {512, 1024, 2048, 4096} with N_d = round(600 N / 1024) data bins (about 58 %),
    64-QAM, an i.i.d. Rayleigh channel, and a memory-polynomial PA of orders {1, 3} or
    {1, 3, 5} (taps 0..3), each with its own seed; S symbols each."""
    st = Stream(seed, "uneven")
    out = []
    for i in range(n):
        u = st.u32(8)
        M = (32, 64, 128, 256)[int(u[0]) % 4]
        K = (4, 8, 16, 32)[int(u[1]) % 4]
        j = 2
        while K > M // 4:
            K = (4, 8, 16, 32)[int(u[j % 8]) % 4] if j < 8 else 4
            j += 1
        N = (512, 1024, 2048, 4096)[int(u[7]) % 4]
        N_d = int(round(N * 600 / 1024))
        pa = PA_NOMINAL_MP13 if int(u[6]) % 2 == 0 else PA_NOMINAL_MP135
        out.append(Config(f"uneven{i}", M=M, K=K, N=N, N_d=N_d, Q=64, S=S, S_per_real=S_per_real, pa_nominal=pa,
                          seed=1000 + i))
    return out


# The ideal linear-clipping PA of Sec. V-B (Fig. 3): order 0 with one coefficient, the
# clipping amplitude A (y = x for |x| <= A, A x / |x| above).
PA_LINEAR_CLIP = {0: [1.0]}


def saturation_amplitude(nominal: Dict[int, List[complex]]) -> float:
    """Drive-level reference: the first local maximum over A > 0 of the nominal
    static AM/AM curve |sum_p (sum_l c_{p,l}) A^p| (found on a fine grid, then
    refined by golden-section search)."""
    orders = sorted(nominal)
    if orders == [0]:   # the linear-clipping PA saturates at its clipping amplitude
        return float(abs(nominal[0][0]))
    cs = [sum(nominal[p]) for p in orders]

    def f(a):
        return abs(sum(c * a ** p for c, p in zip(cs, orders)))

    grid = np.linspace(1e-3, 20.0, 200001)
    vals = np.array([abs(sum(c * grid ** p for c, p in zip(cs, orders)))])[0]
    d = np.diff(vals)
    peaks = np.nonzero((d[:-1] > 0) & (d[1:] <= 0))[0]
    if len(peaks) == 0:
        raise ValueError("AM/AM curve has no maximum below A=20")
    lo, hi = grid[peaks[0]], grid[peaks[0] + 2]
    g = (math.sqrt(5) - 1) / 2
    for _ in range(200):
        a, b = hi - g * (hi - lo), lo + g * (hi - lo)
        if f(a) > f(b):
            hi = b
        else:
            lo = a
    return 0.5 * (lo + hi)


def transmit_power(cfg: Config) -> float:
    """P_T such that the mean time-domain power per antenna sample sits ibo_db
    below A_sat^2 (unit-power symbols, N_d loaded bins of a unitary IDFT):
    P_T = M (N / N_d) A_sat^2 10^(-IBO/10)."""
    a = saturation_amplitude(cfg.pa_nominal)
    return cfg.M * (cfg.N / cfg.N_d) * a * a * 10.0 ** (-cfg.ibo_db / 10.0)


# ----------------------------------------------------------------------------
# FD-CNN parameter vector (flat FP32; conv_w, conv_b, W_fc, b_fc)
# ----------------------------------------------------------------------------
def theta_sizes(cfg: Config) -> Dict[str, int]:
    G, Go = cfg.grid, -(-cfg.grid // cfg.K_S)
    return {
        "conv_w": cfg.N_conv * 2 * cfg.L_U * cfg.K_C * cfg.K_C,
        "conv_b": cfg.N_conv,
        "fc_w": 2 * cfg.N_d * Go * Go * cfg.N_conv,
        "fc_b": 2 * cfg.N_d,
    }


def theta_init(cfg: Config, seed: int, fc_scale: float = 0.0) -> np.ndarray:
    """conv ~ U(+-1/sqrt(fan_in)), conv bias ~ U(+-1/sqrt(fan_in)); the FC weight is
    fc_scale * U(+-1/sqrt(fan_in_fc)) (0 gives the identity predistorter with
    the residual form) and the FC bias is fc_scale * 0.01 * U(+-1).  With per-user
    parameters the K sets are stacked by user, user u's drawn from its own stream."""
    if cfg.per_user:
        return np.concatenate([_theta_one(cfg, Stream(seed, f"theta/user{u}"), fc_scale) for u in range(cfg.K)])
    return _theta_one(cfg, Stream(seed, "theta"), fc_scale)


def _theta_one(cfg: Config, st: "Stream", fc_scale: float) -> np.ndarray:
    sz = theta_sizes(cfg)
    fan = 2 * cfg.L_U * cfg.K_C * cfg.K_C
    b = 1.0 / math.sqrt(fan)
    cw = b * (2 * st.uniform(sz["conv_w"]) - 1)
    cb = b * (2 * st.uniform(sz["conv_b"]) - 1)
    fan_fc = sz["fc_w"] // (2 * cfg.N_d)
    if fc_scale == 0.0:   # the identity predistorter: the dense layer is zero (no draws needed)
        fw, fb = np.zeros(sz["fc_w"]), np.zeros(sz["fc_b"])
    else:
        fw = fc_scale * (2 * st.uniform(sz["fc_w"]) - 1) / math.sqrt(fan_fc)
        fb = fc_scale * 0.01 * (2 * st.uniform(sz["fc_b"]) - 1)
    return np.concatenate([cw, cb, fw, fb]).astype(np.float32)


def fdnn_theta_len(cfg: Config) -> int:
    U, L1, D = cfg.K, cfg.nn_L4 + 1, cfg.nn_D
    return D * 2 * U * L1 + D + (cfg.nn_layers - 1) * (D * D + D) + 2 * U * D + 2 * U


def fdnn_theta_init(cfg: Config, seed: int, out_scale: float = 0.0) -> np.ndarray:
    """FD-NN parameters (Sec. III-C), flat FP32: W_0 [D][2U(L_4+1)], b_0 [D], the further
    hidden layers (W_k [D][D], b_k [D]), W_o [2U][D], b_o [2U].  Hidden layers ~
    U(+-1/sqrt(fan_in)); the output layer times out_scale (0 with the residual form gives
    the identity predistorter)."""
    st = Stream(seed, "fdnn")
    U, L1, D = cfg.K, cfg.nn_L4 + 1, cfg.nn_D
    parts = []
    fan = 2 * U * L1
    for k in range(cfg.nn_layers):
        n_in = fan if k == 0 else D
        b = 1.0 / math.sqrt(n_in)
        parts.append(b * (2 * st.uniform(D * n_in) - 1))
        parts.append(b * (2 * st.uniform(D) - 1))
    b = 1.0 / math.sqrt(D)
    parts.append(out_scale * b * (2 * st.uniform(2 * U * D) - 1))
    parts.append(out_scale * b * (2 * st.uniform(2 * U) - 1))
    return np.concatenate(parts).astype(np.float32)


# ----------------------------------------------------------------------------
# Whole workload
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    cfg: Config
    s: np.ndarray          # complex64 [S][K][N_d]
    H: np.ndarray          # complex64 [R][N_d][K][M]
    pa: np.ndarray         # complex64 [M][P][L+1]
    theta: np.ndarray      # float32 flat
    P_T: float


def batch(cfg: Config, S: int, symbol_offset: int):
    """Symbols [S][K][N_d] and data-bin channel [R][N_d][K][M] (complex64) of the S symbols
    from `symbol_offset` on (a realisation boundary): the mini-batches of a training run,
    each with its own symbols and channel realisations."""
    if symbol_offset % cfg.S_per_real:
        raise ValueError("symbol_offset must start a realisation")
    r0 = symbol_offset // cfg.S_per_real
    R = (S + cfg.S_per_real - 1) // cfg.S_per_real
    s = qam_symbols(cfg.seed, cfg.Q, (S, cfg.K, cfg.N_d), offset=symbol_offset * cfg.K * cfg.N_d).astype(np.complex64)
    taps = channel_taps(cfg.seed, R, cfg.T, cfg.K, cfg.M, cfg.rho, first_real=r0)
    return s, channel_fd(taps, cfg.N, data_bins(cfg.N, cfg.N_d)).astype(np.complex64)


def make_workload(cfg: Config, S: Optional[int] = None, fc_scale: float = 0.0,
                  symbol_offset: int = 0, pa_override: Optional[np.ndarray] = None) -> Workload:
    """Draw a workload of S symbols (default cfg.S) starting at symbol
    `symbol_offset` of the config's streams; realisations follow the symbols."""
    S = cfg.S if S is None else S
    if symbol_offset % cfg.S_per_real:
        raise ValueError("symbol_offset must start a realisation")
    r0 = symbol_offset // cfg.S_per_real
    R = (S + cfg.S_per_real - 1) // cfg.S_per_real
    s = qam_symbols(cfg.seed, cfg.Q, (S, cfg.K, cfg.N_d),
                    offset=symbol_offset * cfg.K * cfg.N_d).astype(np.complex64)
    bins = data_bins(cfg.N, cfg.N_d)
    H = np.empty((R, cfg.N_d, cfg.K, cfg.M), dtype=np.complex64)
    chunk = 8
    for r in range(0, R, chunk):
        n = min(chunk, R - r)
        taps = channel_taps(cfg.seed, n, cfg.T, cfg.K, cfg.M, cfg.rho, first_real=r0 + r)
        H[r:r + n] = channel_fd(taps, cfg.N, bins)
    if pa_override is not None:
        pa = pa_override.astype(np.complex64)
    else:
        pa = pa_coefficients(cfg.seed, cfg.M, cfg.pa_nominal, cfg.pa_spread,
                             cfg.pa_spread_orders).astype(np.complex64)
    theta = theta_init(cfg, cfg.seed, fc_scale)
    return Workload(cfg, s, H, pa, theta, transmit_power(cfg))


def linear_pa(cfg: Config) -> np.ndarray:
    """Coefficients of an ideal linear PA (c_{1,0} = 1, every other c = 0)."""
    P, L1 = len(cfg.orders), cfg.L + 1
    pa = np.zeros((cfg.M, P, L1), dtype=np.complex64)
    pa[:, cfg.orders.index(1), 0] = 1.0
    return pa
