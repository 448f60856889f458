"""Pins of the oracle's FD-NN comparison workload (Sec. III-C) and of its guard-bin power.

- The network of one symbol against the same definition built from library routines
  (numpy FFTs for the unitary DFTs, np.roll for the tapped delay lines, torch FP64
  linear layers and ReLU), with one and two hidden layers.
- Zero output weights with the residual form make the FD-NN the identity; the FD-NN chain
  (every bin precoded) then equals the FD-CNN chain with the identity predistorter.
- With a linear PA the users receive exactly the FD-NN output at the data bins (ZF
  identity of Eq. 6), and the guard- and data-bin powers have the closed form
  sum_k alpha_k^2 s_k^H (H_k H_k^H)^{-1} s_k.
- The guard-bin power of the FD-CNN chain against a numpy FFT of the PA output for a
  nonlinear PA (the ACPR sums).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _cfg(**kw):
    base = dict(name="fdnn_pin", M=6, K=3, N=32, N_d=20, Q=16, S=3, S_per_real=2,
                pa_nominal={1: [1.0, 0.05 - 0.02j, 0.01], 3: [-0.08 + 0.02j, 0.01j, -0.003],
                            5: [-0.002 + 0.0005j, 3e-4, -1e-4]},
                G=5, nn_L4=3, nn_D=7, nn_layers=1)
    base.update(kw)
    return synth.Config(**base)


def _fdnn_ref(cfg, s_sym, theta, residual=1):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    U, N, L1, D = cfg.K, cfg.N, cfg.nn_L4 + 1, cfg.nn_D
    bins = synth.data_bins(N, cfg.N_d)
    full = np.zeros((U, N), complex)
    full[:, bins] = s_sym
    t = np.fft.ifft(full, axis=1) * math.sqrt(N)                 # unitary IDFT
    taps = np.stack([np.roll(t, l, axis=1) for l in range(L1)], axis=2)   # [U][N][L1]: s_u[n-l]
    x = np.concatenate([taps.real.transpose(1, 0, 2).reshape(N, -1),
                        taps.imag.transpose(1, 0, 2).reshape(N, -1)], axis=1)   # [N][2U L1]
    th = torch.from_numpy(theta.astype(np.float64))
    o, nin = 0, 2 * U * L1
    h = torch.from_numpy(x)
    for k in range(cfg.nn_layers):
        n_in = nin if k == 0 else D
        Wk = th[o:o + D * n_in].reshape(D, n_in); o += D * n_in
        bk = th[o:o + D]; o += D
        h = F.relu(F.linear(h, Wk, bk))
    Wo = th[o:o + 2 * U * D].reshape(2 * U, D); o += 2 * U * D
    bo = th[o:o + 2 * U]
    out = F.linear(h, Wo, bo).numpy()                             # [N][2U]
    y = out[:, :U] + 1j * out[:, U:]
    y = y.T + (t if residual else 0)
    return np.fft.fft(y, axis=1) / math.sqrt(N)                   # unitary DFT, every bin


@pytest.mark.parametrize("layers,residual", [(1, 1), (2, 1), (2, 0)])
def test_fdnn_matches_library_definition(layers, residual):
    cfg = _cfg(nn_layers=layers)
    w = synth.make_workload(cfg)
    d = oracle.dims_from_config(cfg, w.P_T, residual=residual)
    th = synth.fdnn_theta_init(cfg, 3, out_scale=0.7)
    assert th.size == oracle.fdnn_theta_len(d) == synth.fdnn_theta_len(cfg)
    for t in range(cfg.S):
        got = oracle.fdnn(d, w.s[t], th)
        ref = _fdnn_ref(cfg, w.s[t].astype(complex), th, residual)
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def _all_bins(cfg, w, d):
    H_all = synth.channel_all_bins(cfg)
    Wa, ala = oracle.precode(oracle.all_bins_dims(d), H_all)
    return H_all, Wa, ala


def test_fdnn_identity_equals_plain_chain():
    cfg = _cfg()
    w = synth.make_workload(cfg)                                  # FD-CNN theta: identity (fc = 0)
    d = oracle.dims_from_config(cfg, w.P_T)
    H_all, Wa, ala = _all_bins(cfg, w, d)
    assert np.array_equal(H_all[:, synth.data_bins(cfg.N, cfg.N_d)], w.H)
    th0 = synth.fdnn_theta_init(cfg, 3, out_scale=0.0)
    sd = oracle.fdnn(d, w.s[0], th0)
    bins = synth.data_bins(cfg.N, cfg.N_d)
    assert np.abs(sd[:, bins] - w.s[0]).max() < 1e-12
    assert np.abs(np.delete(sd, bins, axis=1)).max() < 1e-12
    W, al = oracle.precode(d, w.H)
    y1, m1 = oracle.fdnn_distort(d, w.s, w.H, Wa, ala, w.pa, th0)
    y2, m2 = oracle.distort(d, w.s, w.H, W, al, w.pa, w.theta)
    assert np.abs(y1 - y2).max() < 1e-10
    assert np.allclose(m1, m2, rtol=1e-10, atol=0)


def test_fdnn_linear_pa_closed_forms():
    cfg = _cfg()
    w = synth.make_workload(cfg, pa_override=synth.linear_pa(cfg))
    d = oracle.dims_from_config(cfg, w.P_T)
    H_all, Wa, ala = _all_bins(cfg, w, d)
    th = synth.fdnn_theta_init(cfg, 5, out_scale=0.5)
    y, met = oracle.fdnn_distort(d, w.s, w.H, Wa, ala, w.pa, th)
    bins = synth.data_bins(cfg.N, cfg.N_d)
    guard = np.setdiff1d(np.arange(cfg.N), bins)
    gp = dp = 0.0
    for t in range(cfg.S):
        r = t // cfg.S_per_real
        sd = oracle.fdnn(d, w.s[t], th)
        assert np.abs(y[t] - sd[:, bins]).max() < 1e-10      # H W = I at every data bin
        assert np.abs(np.delete(sd, bins, axis=1)).max() > 1e-3   # the guard bins are filled
        for k in range(cfg.N):
            Hk = H_all[r, k].astype(complex)
            e = ala[r, k] ** 2 * np.real(sd[:, k].conj() @ np.linalg.solve(Hk @ Hk.conj().T, sd[:, k]))
            if k in guard:
                gp += e
            else:
                dp += e
    assert abs(met[3] - gp) <= 1e-9 * gp and abs(met[4] - dp) <= 1e-9 * dp


def test_guard_power_against_numpy_fft_nonlinear_pa():
    """The FD-CNN chain's guard- and data-bin power sums (ACPR) for a nonlinear PA with
    memory: the PA output from the pinned oracle PA, its unitary DFT by numpy, summed by
    bin class here."""
    cfg = _cfg(L_U=1, K_S=1)
    w = synth.make_workload(cfg)                                  # identity predistorter
    d = oracle.dims_from_config(cfg, w.P_T)
    W, al = oracle.precode(d, w.H)
    _, met = oracle.distort(d, w.s, w.H, W, al, w.pa, w.theta)
    bins = synth.data_bins(cfg.N, cfg.N_d)
    is_data = np.zeros(cfg.N, bool)
    is_data[bins] = True
    gp = dp = 0.0
    for t in range(cfg.S):
        r = t // cfg.S_per_real
        for m in range(cfg.M):
            xh = np.zeros(cfg.N, complex)
            xh[bins] = al[r] * np.einsum("ik,ki->i", W[r, :, m, :], w.s[t])
            x = np.fft.ifft(xh) * math.sqrt(cfg.N)
            X = np.fft.fft(oracle.pa(x, cfg.orders, w.pa[m])) / math.sqrt(cfg.N)
            p = np.abs(X) ** 2
            gp += p[~is_data].sum()
            dp += p[is_data].sum()
    assert gp > 1e-6 * dp                                         # a nonlinear PA leaks
    assert abs(met[3] - gp) <= 1e-10 * gp and abs(met[4] - dp) <= 1e-10 * dp
