"""Input generator: Philox known answers, QAM power, channel statistics, PA spread, drive level."""
import math
import os

import numpy as np

import synth
from synth.philox import Stream, philox4x32_10, splitmix64

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        out = philox4x32_10(np.array(w[:4], dtype=np.uint32), np.array(w[4:6], dtype=np.uint32))
        assert [int(v) for v in out] == w[6:10]


def test_splitmix_known_answer():
    # first outputs of SplitMix64 seeded with 0 (state advanced before mixing)
    assert splitmix64(0) == 0xE220A8397B1DCDAF


def test_stream_split_invariance():
    a = Stream(3, "x").u32(10)
    st = Stream(3, "x")
    b = np.concatenate([st.u32(4), st.u32(6)])
    assert np.array_equal(a, b)
    assert not np.array_equal(Stream(3, "x").u32(8), Stream(3, "y").u32(8))


def test_uniform_normal_moments():
    st = Stream(1, "m")
    u = st.uniform(200000)
    assert 0 < u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.005
    z = Stream(1, "n").normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01


def test_qam_unit_power_and_alphabet():
    for Q in (16, 64, 256):
        s = synth.qam_symbols(0, Q, (4000,))
        lv = synth.qam_levels(Q)
        assert abs(np.mean(lv ** 2) * 2 - 1) < 1e-12          # exact unit power of the alphabet
        assert abs(np.mean(np.abs(s) ** 2) - 1) < 0.05
        assert set(np.round(s.real * 1e9)).issubset(set(np.round(lv * 1e9)))


def test_channel_statistics():
    taps = synth.channel_taps(0, 64, 10, 4, 32)
    assert abs(np.mean(np.abs(taps) ** 2) - 0.1) < 0.005        # variance 1/T per tap
    H = synth.channel_fd(taps, 64, synth.data_bins(64, 48))
    assert abs(np.mean(np.abs(H) ** 2) - 1.0) < 0.05            # CN(0,1) per subcarrier
    tc = synth.channel_taps(0, 256, 10, 4, 8, rho=0.5)
    h = tc.reshape(-1, 8)
    C = (h.conj().T @ h).real / h.shape[0] * 10
    assert abs(C[0, 1] - 0.5) < 0.05 and abs(C[0, 2] - 0.25) < 0.05


def test_pa_spread_and_linear():
    cfg = synth.CONFIGS["m64_k8_n1024"]
    pa = synth.pa_coefficients(0, 64, cfg.pa_nominal, 0.1)
    nom = np.array([cfg.pa_nominal[p] for p in cfg.orders])
    ratio = pa / nom[None]
    assert np.allclose(ratio.imag, 0, atol=1e-12)
    assert ratio.real.min() >= 0.9 - 1e-12 and ratio.real.max() <= 1.1 + 1e-12
    c1 = synth.CONFIGS["m16_k2_n64"]
    p1 = synth.pa_coefficients(0, 16, c1.pa_nominal, 0.1, (3,))
    assert np.all(p1[:, 0, 0] == 1.0) and np.ptp(p1[:, 1, 0].real) > 0


def test_saturation_amplitude_closed_form():
    # |A + a3 A^3| peaks where 1 - 4 Re(a3) t + 3 |a3|^2 t^2 = 0 (t = A^2)
    a3 = -0.08 + 0.02j
    t = (4 * -a3.real - math.sqrt(16 * a3.real ** 2 - 12 * abs(a3) ** 2)) / (6 * abs(a3) ** 2)
    assert abs(synth.saturation_amplitude({1: [1.0], 3: [a3]}) - math.sqrt(t)) < 1e-7   # flat maximum: ~sqrt(eps) resolution


def test_workload_shapes():
    w = synth.make_workload(synth.CONFIGS["m16_k2_n64"])
    assert w.s.shape == (10, 2, 48) and w.H.shape == (1, 48, 2, 16) and w.pa.shape == (16, 2, 1)
    assert w.theta.dtype == np.float32 and w.s.dtype == np.complex64
    w2 = synth.make_workload(synth.CONFIGS["m64_k8_n1024"], S=28, symbol_offset=14)
    w3 = synth.make_workload(synth.CONFIGS["m64_k8_n1024"], S=42)
    assert np.array_equal(w2.s, w3.s[14:]) and np.array_equal(w2.H, w3.H[1:])


def test_channel_estimate_imperfect_csi():
    """Sec. II-A: H_est = sqrt(1 - eta) H + sqrt(eta) H_err, H_err taps CN(0, 1), so the
    per-subcarrier error has variance eta T; eta = 0 returns the true channel."""
    cfg = synth.CONFIGS["m64_k8_n1024"].with_(S=28)
    w = synth.make_workload(cfg, S=28)
    assert np.array_equal(synth.channel_estimate(cfg, 0.0, S=28), w.H)
    eta = 0.2
    d = synth.channel_estimate(cfg, eta, S=28).astype(np.complex128) - math.sqrt(1 - eta) * w.H
    assert abs(np.mean(np.abs(d) ** 2) / (eta * cfg.T) - 1) < 0.02
    assert abs(np.mean(d)) < 0.02 * math.sqrt(eta * cfg.T)
