"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (numpy FFT / pinv, torch conv2d), a closed form (two-tone IM3, pure
tones, ZF identity), brute-force frequency-domain intermodulation sums,
central finite differences of the oracle's own forward, or the paper's
printed FLOP table.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import complexity

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


# --- DFT (Eq. 2 and its unitary forward counterpart) -------------------------
@pytest.mark.parametrize("N", [8, 12, 64, 100])
def test_dft_matches_numpy(N):
    rng = np.random.default_rng(N)
    x = crandn(rng, 3, N)
    assert np.allclose(oracle.dft(x), np.fft.fft(x, axis=-1) / math.sqrt(N), atol=1e-12, rtol=0)
    assert np.allclose(oracle.dft(x, inverse=True), np.fft.ifft(x, axis=-1) * math.sqrt(N), atol=1e-12, rtol=0)


def test_dft_parseval_roundtrip_tone():
    rng = np.random.default_rng(0)
    N = 64
    x = crandn(rng, N)
    X = oracle.dft(x)
    assert abs(np.vdot(X, X).real - np.vdot(x, x).real) < 1e-12 * np.vdot(x, x).real
    assert np.allclose(oracle.dft(X, inverse=True), x, atol=1e-13)
    e = np.zeros(N, complex)
    e[5] = 1.0
    n = np.arange(N)
    assert np.allclose(oracle.dft(e, inverse=True), np.exp(2j * np.pi * 5 * n / N) / math.sqrt(N), atol=1e-15)


# --- ZF precoder (Eq. 6) -------------------------------------------------------
@pytest.mark.parametrize("K,M,rho", [(4, 16, 0.0), (2, 16, 0.0), (16, 128, 0.5), (1, 1, 0.0)])
def test_zf_identity_and_pinv(K, M, rho):
    taps = synth.channel_taps(7, 1, 10, K, M, rho)
    Hk = synth.channel_fd(taps, 64, np.array([3]))[0, 0]
    P_T = 37.5
    W, a = oracle.zf(Hk, P_T)
    assert np.abs(Hk @ W - np.eye(K)).max() <= 1e-12
    assert np.allclose(W, np.linalg.pinv(Hk), atol=1e-12 * np.abs(W).max(), rtol=0)
    assert abs(a * a * np.trace(W.conj().T @ W).real - P_T) < 1e-10 * P_T


def test_zf_singular_rejected():
    rng = np.random.default_rng(1)
    Hk = crandn(rng, 3, 8)
    Hk[2] = Hk[0]
    with pytest.raises(np.linalg.LinAlgError):
        oracle.zf(Hk, 1.0)


# --- PA (Eq. 7 / Eq. 9 diagonal terms) ----------------------------------------
def test_pa_two_tone_im3_closed_form():
    N, A, f1, f2 = 64, 0.7, 5, 8
    a1, a3 = 1.0 + 0.1j, -0.08 + 0.02j
    n = np.arange(N)
    x = A * (np.exp(2j * np.pi * f1 * n / N) + np.exp(2j * np.pi * f2 * n / N))
    X = oracle.dft(oracle.pa(x, [1, 3], [[a1], [a3]]))
    r = math.sqrt(N)
    assert abs(abs(X[2 * f1 - f2]) - r * abs(a3) * A ** 3) < 1e-12
    assert abs(abs(X[2 * f2 - f1]) - r * abs(a3) * A ** 3) < 1e-12
    assert abs(X[f1] - r * (a1 * A + 3 * a3 * A ** 3)) < 1e-12
    others = np.delete(np.abs(X), [f1, f2, 2 * f1 - f2, 2 * f2 - f1])
    assert others.max() < 1e-12


def _brute_cubic(X, a1, a3):
    N = len(X)
    Y = a1 * X.copy()
    for k in range(N):
        acc = 0
        for i in range(N):
            for j in range(N):
                acc += X[i] * X[j] * np.conj(X[(i + j - k) % N])
        Y[k] += a3 * acc / N
    return Y


@pytest.mark.parametrize("N", [16, 32])
def test_pa_frequency_domain_triple_sum(N):
    rng = np.random.default_rng(N)
    X = crandn(rng, N)
    X[N // 2 - 3: N // 2 + 3] = 0                    # guard bins
    c = np.array([[1.0 + 0j, 0.1 - 0.05j, 0.02], [-0.08 + 0.02j, 0.01j, -0.003]])
    Y = oracle.dft(oracle.pa(oracle.dft(X, inverse=True), [1, 3], c))
    k = np.arange(N)
    ref = np.zeros(N, complex)
    for l in range(3):                                 # tap l multiplies bin k by e^{-j 2 pi k l / N}
        ref += np.exp(-2j * np.pi * k * l / N) * _brute_cubic(X, c[0, l], c[1, l])
    assert np.allclose(Y, ref, atol=1e-12, rtol=0)


def test_pa_fifth_order_quintuple_sum():
    N = 8
    rng = np.random.default_rng(5)
    X = crandn(rng, N)
    a5 = 0.3 - 0.2j
    Y = oracle.dft(oracle.pa(oracle.dft(X, inverse=True), [5], [[a5]]))
    ref = np.zeros(N, complex)
    for k in range(N):
        acc = 0
        for a in range(N):
            for b in range(N):
                for c in range(N):
                    for d in range(N):
                        acc += X[a] * X[b] * X[c] * np.conj(X[d]) * np.conj(X[(a + b + c - d - k) % N])
        ref[k] = a5 * acc / N ** 2
    assert np.allclose(Y, ref, atol=1e-12, rtol=0)


# --- FD-CNN (Sec. IV-A) vs torch CPU FP64 conv2d / linear ---------------------
@pytest.mark.parametrize("L_U,K_S,K_C,G,N_d", [(1, 1, 3, 7, 48), (2, 2, 3, 5, 20), (3, 1, 5, 6, 33)])
def test_fdcnn_matches_torch(L_U, K_S, K_C, G, N_d):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    K, N_conv = 3, 2
    d = oracle.make_dims(4, K, 64, N_d, [1, 3], 0, G, 1.0, L_U=L_U, K_C=K_C, K_S=K_S, N_conv=N_conv)
    rng = np.random.default_rng(11)
    th = rng.standard_normal(oracle.theta_len(d)) * 0.3
    s = crandn(rng, K, N_d)
    st, pre, act = oracle.fdcnn(d, s, th)
    Cin, Go = 2 * L_U, -(-G // K_S)
    nw = N_conv * Cin * K_C * K_C
    w = torch.tensor(th[:nw]).reshape(N_conv, Cin, K_C, K_C)
    b = torch.tensor(th[nw:nw + N_conv])
    Fd = N_conv * Go * Go
    fw = torch.tensor(th[nw + N_conv: nw + N_conv + 2 * N_d * Fd]).reshape(2 * N_d, Fd)
    fb = torch.tensor(th[nw + N_conv + 2 * N_d * Fd:])
    grid = np.zeros((K, G * G), complex)
    grid[:, :N_d] = s
    chans = []
    for l in range(L_U):
        g = np.roll(grid, -l, axis=0)
        chans += [g.real, g.imag]
    X = torch.tensor(np.stack(chans, 1).reshape(K, Cin, G, G))
    p = F.conv2d(X, w, b, stride=K_S, padding=K_C // 2)
    assert p.shape[-1] == Go
    assert np.allclose(pre, p.reshape(K, -1).numpy(), atol=1e-12)
    dd = F.linear(F.relu(p).reshape(K, -1), fw, fb).numpy()
    assert np.allclose(st, s + dd[:, :N_d] + 1j * dd[:, N_d:], atol=1e-12)


# --- whole chain ----------------------------------------------------------------
def _small_cfg(**kw):
    base = dict(name="pin", M=6, K=3, N=32, N_d=20, Q=16, S=3, S_per_real=2,
                pa_nominal={1: [1.0, 0.05 - 0.02j, 0.01], 3: [-0.08 + 0.02j, 0.01j, -0.003],
                            5: [-0.002 + 0.0005j, 3e-4, -1e-4]},
                G=5, L_U=2, K_S=2)
    base.update(kw)
    return synth.Config(**base)


def _setup(cfg, fc_scale=0.0, pa=None):
    w = synth.make_workload(cfg, fc_scale=fc_scale, pa_override=pa)
    d = oracle.dims_from_config(cfg, w.P_T)
    W, al = oracle.precode(d, w.H)
    return w, d, W, al


def test_identity_for_linear_pa():
    cfg = synth.CONFIGS["m16_k2_n64"]
    w, d, W, al = _setup(cfg, pa=synth.linear_pa(cfg))
    y, met = oracle.distort(d, w.s, w.H, W, al, w.pa, w.theta)
    assert np.abs(y - w.s).max() < 1e-12
    assert met[0] < 1e-24 and met[3] < 1e-20 * met[4]
    g, _ = oracle.backward(d, w.s, w.H, W, al, w.pa, w.theta)
    assert np.abs(g).max() < 1e-15


def test_linear_pa_with_memory_is_per_bin_gain():
    cfg = _small_cfg()
    taps = np.array([0.9 + 0.1j, 0.2 - 0.1j, 0.05j])
    pa = np.zeros((cfg.M, 3, 3), np.complex64)
    pa[:, 0, :] = taps
    w, d, W, al = _setup(cfg, fc_scale=0.5, pa=pa)
    y, met = oracle.distort(d, w.s, w.H, W, al, w.pa, w.theta)
    k = synth.data_bins(cfg.N, cfg.N_d)
    gain = sum(complex(np.complex64(t)) * np.exp(-2j * np.pi * k * l / cfg.N) for l, t in enumerate(taps))
    for t in range(cfg.S):
        st, _, _ = oracle.fdcnn(d, w.s[t], w.theta)
        assert np.allclose(y[t], gain[None, :] * st, atol=1e-12)


def test_siso_cubic_chain_by_hand():
    cfg = _small_cfg(M=1, K=1, N=16, N_d=16, S=2, S_per_real=2, G=4, L_U=1, K_S=1,
                     pa_nominal={1: [1.0 + 0.05j], 3: [-0.08 + 0.02j]}, pa_spread=0.0)
    w, d, W, al = _setup(cfg)
    y, _ = oracle.distort(d, w.s, w.H, W, al, w.pa, w.theta)
    h = w.H[0, :, 0, 0].astype(complex)
    k = synth.data_bins(cfg.N, cfg.N_d)
    a1, a3 = complex(w.pa[0, 0, 0]), complex(w.pa[0, 1, 0])
    for t in range(2):
        xh = np.zeros(16, complex)
        xh[k] = math.sqrt(w.P_T) * np.exp(-1j * np.angle(h)) * w.s[t, 0]
        Xpa = _brute_cubic(xh, a1, a3)
        ref = h * Xpa[k] / (math.sqrt(w.P_T) * np.abs(h))
        assert np.allclose(y[t, 0], ref, atol=1e-12)


def test_metrics_definitions():
    cfg = _small_cfg()
    w, d, W, al = _setup(cfg, fc_scale=0.2)
    y, met = oracle.distort(d, w.s, w.H, W, al, w.pa, w.theta)
    e = y - w.s
    assert abs(met[1] - np.sum(np.abs(e) ** 2)) < 1e-10 * met[1]
    assert abs(met[2] - np.sum(np.abs(w.s.astype(complex)) ** 2)) < 1e-10 * met[2]
    assert abs(met[0] - met[1] / e.size) < 1e-15
    assert met[3] > 0


# --- adjoint (hand-derived) vs central finite differences ---------------------
def _loss(d, w, W, al, th):
    return oracle.distort(d, w.s, w.H, W, al, w.pa, th)[1][0]


def test_adjoint_central_differences():
    cfg = _small_cfg()
    w, d, W, al = _setup(cfg, fc_scale=0.5)
    th = w.theta.astype(np.float64)
    g, met = oracle.backward(d, w.s, w.H, W, al, w.pa, th)
    assert abs(met[0] - _loss(d, w, W, al, th)) < 1e-15
    rng = np.random.default_rng(2)
    n_conv = d.N_conv * 2 * d.L_U * d.K_C * d.K_C + d.N_conv
    idx = np.concatenate([np.arange(n_conv), rng.choice(np.arange(n_conv, len(th)), 100, replace=False)])
    gmax = np.abs(g).max()
    eps = 1e-5
    for j in idx:
        tp, tm = th.copy(), th.copy()
        tp[j] += eps
        tm[j] -= eps
        fd = (_loss(d, w, W, al, tp) - _loss(d, w, W, al, tm)) / (2 * eps)
        assert abs(fd - g[j]) <= 1e-6 * gmax, (j, fd, g[j])
    for _ in range(10):
        v = rng.standard_normal(len(th))
        v /= np.linalg.norm(v)
        fd = (_loss(d, w, W, al, th + eps * v) - _loss(d, w, W, al, th - eps * v)) / (2 * eps)
        assert abs(fd - g @ v) <= 1e-6 * abs(g @ v) + 1e-9 * gmax


def test_adjoint_paper_literal_mode():
    cfg = _small_cfg(L_U=1, K_S=1)
    w = synth.make_workload(cfg, fc_scale=0.5)
    d = oracle.dims_from_config(cfg, w.P_T, residual=0)
    W, al = oracle.precode(d, w.H)
    th = w.theta.astype(np.float64)
    g, _ = oracle.backward(d, w.s, w.H, W, al, w.pa, th)
    rng = np.random.default_rng(3)
    for j in rng.choice(len(th), 40, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[j] += 1e-5
        tm[j] -= 1e-5
        fd = (_loss(d, w, W, al, tp) - _loss(d, w, W, al, tm)) / 2e-5
        assert abs(fd - g[j]) <= 1e-6 * np.abs(g).max()


# --- update rule ---------------------------------------------------------------
def test_gd_step_exact():
    cfg = _small_cfg()
    w, d, W, al = _setup(cfg, fc_scale=0.3)
    th = w.theta.astype(np.float64)
    g, _ = oracle.backward(d, w.s, w.H, W, al, w.pa, th)
    th1, _ = oracle.update(d, w.s, w.H, W, al, w.pa, th, 1e-3, 1)
    assert np.array_equal(th1, th - 1e-3 * g)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    cfg = _small_cfg()
    w, d, W, al = _setup(cfg, fc_scale=0.3)
    th = w.theta.astype(np.float64)
    st = oracle.AdamState(len(th))
    th_o, _ = oracle.update(d, w.s, w.H, W, al, w.pa, th, 1e-3, 3, adam=st)
    p = torch.nn.Parameter(torch.tensor(th))
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for _ in range(3):
        g, _ = oracle.backward(d, w.s, w.H, W, al, w.pa, p.detach().numpy())
        p.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(th_o, p.detach().numpy(), atol=1e-14, rtol=0)
    assert st.t.value == 3


# --- complexity model vs the printed Fig. 2 -------------------------------------
def _fig2():
    rows = [l for l in open(os.path.join(GOLD, "fig2_flops.csv")) if not l.startswith("#")]
    return np.array([[int(v) for v in r.split(",")] for r in rows[1:]])


def test_fig2_fd_cnn_and_fd_nn_exact():
    t = _fig2()
    for B, _, _, _, fdnn, fdcnn in t:
        assert complexity.fd_nn(4096, 384, 1, B, 3, 15, 1) == fdnn
        assert complexity.fd_nn(4096, 384, 8, B, 3, 15, 1) == fdnn      # per UE: independent of U
        assert complexity.fd_cnn(384, 1, 3, 1, 2, grid_cells=384) == fdcnn
    # with the padded 20 x 20 grid the formula gives 1 256 000, not the printed value
    assert complexity.fd_cnn(384, 1, 3, 1, 2) == 1256000


def test_fig2_td_gmp_structure():
    t = _fig2()
    assert complexity.td_gmp_per_sample(7, 3, 1) == 674                # Eq. (10) as printed
    for B, u1, u4, u8, _, _ in t:                                      # the figure uses 658 / sample
        assert (u1, u4, u8) == tuple(int(complexity.td_gmp(7, 3, 1, 4096, B, U, per_sample=658)) for U in (1, 4, 8))
    # savings quoted in Sec. V-B at B = 32, U = 8 and B = 1024
    r = lambda B: (complexity.fd_nn(4096, 384, 8, B, 3, 15, 1) / 1205760,
                   complexity.td_gmp(7, 3, 1, 4096, B, 8, per_sample=658) / 1205760)
    assert [round(v, 1) for v in r(32)] == [2.2, 8.9]
    assert [int(v) for v in r(1024)] == [26, 286]


def test_chain_rejects_missing_realisations():
    """The chain indexes H, W and alpha by realisation: too few for S symbols is an error."""
    cfg = synth.CONFIGS["m16_k2_n64"]
    w = synth.make_workload(cfg, S=2 * cfg.S_per_real)
    d = oracle.dims_from_config(cfg, w.P_T)
    W, al = oracle.precode(d, w.H[:1])
    with pytest.raises(ValueError):
        oracle.distort(d, w.s, w.H[:1], W, al, w.pa, w.theta)
    with pytest.raises(ValueError):
        oracle.backward(d, w.s, w.H[:1], W, al, w.pa, w.theta[:-1])
    y, _ = oracle.distort(d, w.s[:cfg.S_per_real], w.H[:1], W, al, w.pa, w.theta)
    assert y.shape == (cfg.S_per_real, cfg.K, cfg.N_d)


# --- symbol errors at the users (Sec. V-B; noise of Eq. 4-5) ------------------------
def test_oracle_philox_known_answers():
    """The oracle's own Philox-4x32-10 against the published Random123 vectors."""
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert list(oracle.philox4x32_10(w[:4], w[4:6])) == w[6:10]


def _ser_dims(K=2, N_d=48, Spr=5):
    return oracle.make_dims(M=4, K=K, N=64, N_d=N_d, orders=[1], L=0, G=7, P_T=1.0, S_per_real=Spr)


def test_oracle_ser_noiseless_and_one_step_off():
    d = _ser_dims()
    s = synth.qam_symbols(3, 16, (10, d.K, d.N_d)).astype(np.complex128)
    al = np.ones((2, d.N_d))
    e, n, _, _ = oracle.ser(d, s, s, al, 16, 0.0, 7)
    assert (e, n) == (0, s.size)
    step = 2.0 / math.sqrt(2.0 * 15 / 3.0)                  # one level of unit-power 16-QAM
    y = s + np.where(s.real < 0, step, -step)              # every real part moves to the next level inwards
    e, n, _, _ = oracle.ser(d, y, s, al, 16, 0.0, 7)
    assert (e, n) == (s.size, s.size)
    al[1, 5] = 0.0                                          # a singular subcarrier carries no symbol
    e, n, _, _ = oracle.ser(d, s, s, al, 16, 0.0, 7)
    assert n == s.size - 5 * d.K


def test_oracle_ser_matches_awgn_closed_form():
    """y = s, alpha = 1: square 16-QAM in AWGN, P_s = 1 - (1 - p)^2 with
    p = 2 (1 - 1/4) Q(sqrt(3 SNR / 15)), SNR = E_s / N0 (a textbook closed form)."""
    d = _ser_dims(K=4, N_d=500, Spr=10)
    S = 100
    s = synth.qam_symbols(5, 16, (S, d.K, d.N_d)).astype(np.complex128)
    al = np.ones((10, d.N_d))
    for snr_db in (12.0, 15.0):
        N0 = 10 ** (-snr_db / 10)
        e, n, z, _ = oracle.ser(d, s, s, al, 16, N0, 1234)
        w = z - s
        assert abs(np.mean(np.abs(w) ** 2) / N0 - 1.0) < 0.01        # E|w|^2 = N0
        assert abs(np.mean(w.real ** 2) - np.mean(w.imag ** 2)) < 0.01 * N0
        p = 2 * (1 - 1 / 4) * 0.5 * math.erfc(math.sqrt(3 * 10 ** (snr_db / 10) / 15) / math.sqrt(2))
        ps = 1 - (1 - p) ** 2
        sd = math.sqrt(ps * (1 - ps) / n)
        assert abs(e / n - ps) < 4 * sd, (snr_db, e / n, ps)


def test_oracle_ser_noise_scales_with_alpha():
    """z = y + w / alpha: alpha 2 with 4 N0 reproduces the same z as alpha 1 with N0."""
    d = _ser_dims()
    s = synth.qam_symbols(9, 64, (10, d.K, d.N_d)).astype(np.complex128)
    _, _, z1, w1 = oracle.ser(d, s, s, np.ones((2, d.N_d)), 64, 0.02, 99)
    _, _, z2, w2 = oracle.ser(d, s, s, 2 * np.ones((2, d.N_d)), 64, 0.08, 99)
    assert np.allclose(z1, z2, rtol=0, atol=1e-15) and np.array_equal(w1, w2)


# --- the ideal linear-clipping PA (Sec. V-B, Fig. 3) --------------------------------
def test_clip_pa_definition():
    """|y| = min(|x|, A) with the phase of x; a clipping level above every sample is the
    identity; the drive-level reference is the clipping amplitude."""
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(64) + 1j * rng.standard_normal(64)) * 0.8
    y = oracle.pa(x, [0], np.array([[0.9]]))
    assert np.allclose(np.abs(y), np.minimum(np.abs(x), 0.9), atol=1e-15)
    assert np.allclose(np.angle(y), np.angle(x), atol=1e-12)
    assert np.array_equal(oracle.pa(x, [0], np.array([[1e9]])), x)
    assert synth.saturation_amplitude({0: [1.3]}) == 1.3


def test_clip_pa_adjoint_central_differences():
    """The chain with a clipping PA driven into clipping: hand-derived adjoint (Wirtinger
    derivatives A/(2|x|), -A x^2/(2|x|^3) above A) against central differences."""
    cfg = _small_cfg(pa_nominal=synth.PA_LINEAR_CLIP, ibo_db=0.0)
    w, d, W, al = _setup(cfg, fc_scale=0.5)
    th = w.theta.astype(np.float64)
    g, _ = oracle.backward(d, w.s, w.H, W, al, w.pa, th)
    rng = np.random.default_rng(5)
    gmax = np.abs(g).max()
    for j in rng.choice(len(th), 60, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[j] += 1e-6
        tm[j] -= 1e-6
        fd = (_loss(d, w, W, al, tp) - _loss(d, w, W, al, tm)) / 2e-6
        assert abs(fd - g[j]) <= 1e-5 * gmax, (j, fd, g[j])
    # the PA clips a good share of the time-domain samples at this drive level
    y, met = oracle.distort(d, w.s, w.H, W, al, w.pa, th)
    assert met[3] > 1e-4 * met[4]


# --- the GMP of Eq. (9) with cross terms (the paper's PA model, Sec. V-A: K = 7, L = 3, G = 1)
def _gmp_coef(a, G, scale, seed):
    """[M][P][L+1] memory-polynomial part a plus random lagging / leading cross terms,
    flattened per antenna as a [P][L+1], b [P][L+1][G], c [P][L+1][G]."""
    M, P, L1 = a.shape
    rng = np.random.default_rng(seed)
    bc = scale * (rng.standard_normal((2, M, P, L1, G)) + 1j * rng.standard_normal((2, M, P, L1, G)))
    return np.concatenate([a.reshape(M, -1), bc[0].reshape(M, -1), bc[1].reshape(M, -1)], axis=1)


def test_gmp_single_cross_terms_by_hand():
    """One lagging term b x_{n-1} |x_{n-2}|^2 and one leading term c x_{n-1} |x_n|^2
    (order 3, l = 1, g = 1), circular in n."""
    rng = np.random.default_rng(6)
    x = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    orders, L, G = [1, 3], 1, 1
    a = np.zeros((1, 2, 2), complex)
    for side, ref in ((0, np.roll(x, 1) * np.abs(np.roll(x, 2)) ** 2), (1, np.roll(x, 1) * np.abs(x) ** 2)):
        coef = _gmp_coef(a, G, 0.0, 0)
        # a [2][2] at 0..3, b [2][2][1] at 4..7, c at 8..11: order index 1 (p = 3), l = 1, g = 1
        coef[0, 4 + 4 * side + (1 * 2 + 1) * G + 0] = 0.3 - 0.2j
        y = oracle.pa_gmp(x, orders, coef[0], G)
        assert np.allclose(y, (0.3 - 0.2j) * ref, atol=1e-13), side


def test_gmp_constant_envelope_reduces_to_memory_polynomial():
    """With |x_n| = r for every n the envelope of every cross term is r^{p-1}: the GMP
    equals the memory polynomial with a'_{p,l} = a_{p,l} + sum_g (b_{p,l,g} + c_{p,l,g})."""
    rng = np.random.default_rng(7)
    x = 0.7 * np.exp(2j * np.pi * rng.random(32))
    orders, L, G = [1, 2, 3, 5], 3, 2
    a = rng.standard_normal((1, 4, 4)) + 1j * rng.standard_normal((1, 4, 4))
    coef = _gmp_coef(a, G, 0.2, 8)[0]
    b = coef[16:16 + 32].reshape(4, 4, G)
    c = coef[48:].reshape(4, 4, G)
    a2 = a[0] + np.where(np.array(orders)[:, None] >= 2, (b + c).sum(axis=2), 0)
    assert np.allclose(oracle.pa_gmp(x, orders, coef, G), oracle.pa(x, orders, a2), atol=1e-12)


def test_gmp_adjoint_central_differences():
    """The whole chain with a GMP PA (orders 1..7, L = 3, G = 1): the hand-derived adjoint
    of the cross terms against central differences."""
    cfg = _small_cfg(pa_nominal={1: [1.0, 0.05 - 0.02j, 0.01, 0.002], 2: [0.02j, 0.004, 0.0, 0.0],
                                 3: [-0.08 + 0.02j, 0.01j, -0.003, 0.001], 4: [0.005, 0.0, 0.0, 0.0],
                                 5: [-0.002 + 0.0005j, 3e-4, -1e-4, 0.0], 6: [1e-4, 0.0, 0.0, 0.0],
                                 7: [1e-5j, 0.0, 0.0, 0.0]}, pa_G=1)
    w = synth.make_workload(cfg, fc_scale=0.5)
    pa = _gmp_coef(w.pa.astype(complex), 1, 0.01, 9)
    d = oracle.dims_from_config(cfg, w.P_T)
    W, al = oracle.precode(d, w.H)
    th = w.theta.astype(np.float64)
    loss = lambda t: oracle.distort(d, w.s, w.H, W, al, pa, t)[1][0]
    g, met = oracle.backward(d, w.s, w.H, W, al, pa, th)
    assert abs(met[0] - loss(th)) < 1e-15
    rng = np.random.default_rng(10)
    gmax = np.abs(g).max()
    for j in rng.choice(len(th), 60, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[j] += 1e-5
        tm[j] -= 1e-5
        assert abs((loss(tp) - loss(tm)) / 2e-5 - g[j]) <= 1e-6 * gmax, j
    # the cross terms matter: without them the output differs
    y1, _ = oracle.distort(d, w.s, w.H, W, al, pa, th)
    d0 = oracle.dims_from_config(cfg.with_(pa_G=0), w.P_T)
    y0, _ = oracle.distort(d0, w.s, w.H, W, al, w.pa, th)
    assert np.abs(y1 - y0).max() > 1e-4


# --- per-user FD-CNN parameters theta_u (Sec. IV-A) ------------------------------
@pytest.mark.parametrize("L_U", [1, 2])
def test_per_user_equal_parameters_reduce_to_shared(L_U):
    """K copies of one theta: the same forward chain as the shared network, and the
    per-user gradient slices add up to the shared gradient (the shared gradient is the
    sum of every user's contribution)."""
    cfg = _small_cfg(L_U=L_U)
    w, d, W, al = _setup(cfg, fc_scale=0.5)
    th = w.theta.astype(np.float64)
    dp = oracle.dims_from_config(cfg.with_(per_user=1), w.P_T)
    thK = np.tile(th, cfg.K)
    assert oracle.theta_len(dp) == cfg.K * th.size
    y, m = oracle.distort(d, w.s, w.H, W, al, w.pa, th)
    yp, mp = oracle.distort(dp, w.s, w.H, W, al, w.pa, thK)
    assert np.array_equal(y, yp) and np.array_equal(m, mp)
    g, _ = oracle.backward(d, w.s, w.H, W, al, w.pa, th)
    gp, _ = oracle.backward(dp, w.s, w.H, W, al, w.pa, thK)
    assert np.abs(gp.reshape(cfg.K, -1).sum(axis=0) - g).max() <= 1e-12 * np.abs(g).max()


@pytest.mark.parametrize("L_U", [1, 2])
def test_per_user_outputs_follow_their_own_parameters(L_U):
    """A linear PA and perfect CSI pass s_tilde through unchanged (y = s_tilde), so with
    per-user parameters user u receives exactly the FD-CNN of theta_u applied to its own
    input users (u, ..., u + L_U - 1), whatever the other users' parameters are."""
    cfg = _small_cfg(L_U=L_U, per_user=1)
    w, d, W, al = _setup(cfg, fc_scale=0.5, pa=synth.linear_pa(cfg))
    thK = w.theta.astype(np.float64).reshape(cfg.K, -1)
    assert not np.allclose(thK[0], thK[1])
    y, _ = oracle.distort(d, w.s, w.H, W, al, w.pa, thK.ravel())
    d1 = oracle.dims_from_config(cfg.with_(per_user=0), w.P_T)
    for t in range(cfg.S):
        for u in range(cfg.K):
            st, _, _ = oracle.fdcnn(d1, w.s[t], thK[u])
            assert np.abs(y[t, u] - st[u]).max() < 1e-12


def test_per_user_adjoint_central_differences():
    cfg = _small_cfg(L_U=1, per_user=1)
    w, d, W, al = _setup(cfg, fc_scale=0.5)
    th = w.theta.astype(np.float64)
    g, _ = oracle.backward(d, w.s, w.H, W, al, w.pa, th)
    one = th.size // cfg.K
    n_conv = d.N_conv * 2 * d.K_C * d.K_C + d.N_conv
    rng = np.random.default_rng(5)
    idx = np.concatenate([u * one + np.arange(n_conv) for u in range(cfg.K)] +
                         [rng.choice(np.arange(th.size), 60, replace=False)])
    gmax, eps = np.abs(g).max(), 1e-5
    for j in idx:
        tp, tm = th.copy(), th.copy()
        tp[j] += eps
        tm[j] -= eps
        fd = (_loss(d, w, W, al, tp) - _loss(d, w, W, al, tm)) / (2 * eps)
        assert abs(fd - g[j]) <= 1e-6 * gmax, (j, fd, g[j])
