#!/usr/bin/env python3
"""Throughput of the FD-DPD downlink chain on one GB300: DPD'd OFDM symbols/s.

Workload: M=128 antennas, K=16 users, N=2048 with N_d=1200 data subcarriers,
256-QAM, exponentially correlated (rho=0.5) Rayleigh channel with a new
realisation every 14 symbols, memory-polynomial PAs (orders 1,3,5, taps 0..3),
FD-CNN G=35, N_conv=2, K_C=3; 2000 symbols per step (143 realisations).

One step = the whole hot path once over the 2000 symbols: zero-forcing build for
every realisation, FD-CNN, precoding, IFFT, PA, FFT, combining, loss, the adjoint
of all of it, and one gradient-descent update of theta.  Inputs are resident in
HBM and larger than L2 (H alone is 2.8 GB).  `value` is device-timed with CUDA
events; `e2e` runs the same step through fddpd_update_host from pinned host memory.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|bf16|fp16]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DPD'd OFDM symbols/s at M=128,K=16,N=2048; % roofline; EVM vs FP64 oracle"
UNIT = "symbols/s"
SER_SNR_DB = 30.0   # mean per-subcarrier SNR at the users for the SER line
WORKLOAD = ("m128_k16_n2048: M=128 K=16 N=2048 N_d=1200 256-QAM rho=0.5, 14 symbols/realisation, orders 1,3,5 taps 0..3, "
            "FD-CNN G=35 N_conv=2 K_C=3")
LR = 1e-4
ARITHMETIC = ("ZF Gram FP32, Cholesky + triangular inverse FP64; FD-CNN dense layer, precoding and combining "
              "on tcgen05 with BF16 operands and FP32 accumulation; FFT, PA and its adjoint FP32 with x(t) "
              "recomputed in the adjoint")
FAST_ARITHMETIC = ("as the headline but Cholesky + triangular inverse FP32 and x(t) kept from the forward in BF16 "
                   "(FDDPD_OPT_FACTOR_FP64 = 0, FDDPD_OPT_KEEP_PA_INPUT = 1)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--symbols", type=int, default=2000)
    ap.add_argument("--cpu-sample", type=int, default=20, help="symbols in the oracle's cpu_baseline sample")
    ap.add_argument("--ref-sample", type=int, default=2, help="symbols per step of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-fast-variant", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-fdnn", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-regime", action="store_true", help="skip the symbols-per-realisation sweep")
    ap.add_argument("--train-steps", type=int, default=TRAIN_STEPS)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return mp, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peaks(fd, stream):
    """FP32 and FP64 pipe peaks measured now by the library's FMA loop (TFLOP/s): the
    FP32 peak is the better of the scalar and the packed-pair fma loops."""
    p = {k: fd.alu_peak(k, stream) for k in ("fp32", "fp32x2", "fp64")}
    p["fp32_peak"] = max(p["fp32"], p["fp32x2"])
    return p


# ---------------------------------------------------------------------------
# algorithmic work per launch of each stage (bytes or flops)
# ---------------------------------------------------------------------------
def stage_work(cfg, S: int, prec: str, fp64_factor: bool = True, kept_xt: bool = False):
    M, K, Nd, F, L_U = cfg.M, cfg.K, cfg.N_d, cfg.N_conv * (-(-cfg.grid // cfg.K_S)) ** 2, cfg.L_U
    R = -(-S // cfg.S_per_real)
    cols = S * K
    c8 = 8
    opb = 8 if prec == "fp32" else 4          # bytes of one complex H / W operand
    ab = 4 if prec == "bf16" else 8           # bytes of one complex X^PA, gX, g_xhat entry
    fc_bound = "alu" if prec == "fp32" else "tensor"
    theta_len = cfg.N_conv * 2 * L_U * cfg.K_C ** 2 + cfg.N_conv + 2 * Nd * F + 2 * Nd
    return {
        # Gram: read H (+ write its 16-bit copy and, with the precoder kept as its factors,
        # the 16-bit H^H); factor: K^3/3 complex MACs per subcarrier (Cholesky + triangular
        # inverse, 4 FMA = 8 flop each), FP64 unless a 16-bit plan selects FP32; apply: read
        # H, write W
        "zf_gram": ("hbm", R * Nd * K * M * (c8 + (0 if prec == "fp32" else 8))),
        "zf_factor": ("fp64" if (prec == "fp32" or fp64_factor) else "alu", R * Nd * 8.0 * (K ** 3 / 3.0)),
        "zf_apply": ("hbm", R * Nd * K * M * (2 * c8 + (0 if prec == "fp32" else 4)) + R * Nd * 4),
        "conv_fwd": ("hbm", cols * Nd * c8 * L_U + cols * F * 4),
        "fc_fwd": (fc_bound, 2.0 * cols * 2 * Nd * F),
        "precode": ("hbm", R * Nd * M * K * opb + S * K * Nd * c8 + S * M * Nd * c8),
        # the row kernels are bound by FP32 arithmetic: per row two N-point transforms at the
        # conventional 5 N log2 N flops each, plus the PA (4 taps x 19 flops: |x|^2, the
        # Horner polynomial in |x|^2, the complex multiply-add) or its adjoint (three 4-tap
        # complex filters, 96 flops, plus ~26 for the two Horner evaluations and x^2)
        "fftpa_fwd": ("alu", S * M * (2 * 5.0 * cfg.N * math.log2(cfg.N) + cfg.N * (cfg.L + 1) * 19.0)),
        "combine": ("hbm", R * Nd * K * M * opb + S * M * Nd * ab + 2 * S * K * Nd * c8),
        "adj_combine": ("hbm", R * Nd * K * M * opb + S * K * Nd * c8 + S * M * Nd * ab),
        # adjoint: the transform of g_X and the final one, plus (x(t) recomputed) the inverse
        # transform of x_hat
        "fftpa_adj": ("alu", S * M * ((2 if kept_xt else 3) * 5.0 * cfg.N * math.log2(cfg.N)
                                      + cfg.N * (24.0 * (cfg.L + 1) + 26.0))),
        "adj_precode": ("hbm", R * Nd * M * K * opb + S * M * Nd * ab + S * K * Nd * c8),
        "fc_bwd_w": (fc_bound, 2.0 * 2 * Nd * F * cols),
        "fc_bwd_b": ("hbm", cols * 2 * Nd * 4),
        "fc_bwd_d": (fc_bound, 2.0 * cols * F * 2 * Nd),
        "conv_bwd": ("hbm", cols * (Nd * c8 * L_U + F * 4)),
        "step": ("hbm", 3 * theta_len * 4),
        # Z x per (symbol, subcarrier) from the factor's Y (one of two launches: precode side,
        # adjoint side): Y's lower triangles in, x in, result out
        "zmul": ("hbm", R * Nd * (K * (K + 1) // 2) * 8 + 2 * S * K * Nd * c8),
    }


def roofline_of(bound, amount, per_launch_ms, mp, src, alu):
    """(achieved, peak, unit, peak source) of `amount` bytes / flops done in per_launch_ms."""
    sec = per_launch_ms / 1e3
    if bound == "hbm":
        return amount / sec / 1e9, mp["hbm_gbs"], "GB/s", f"{src} hbm_gbs (copy)"
    if bound == "tensor":
        return amount / sec / 1e12, mp["bf16_tflops_sustained"], "TFLOP/s", f"{src} bf16_tflops_sustained"
    if bound == "fp64":
        return amount / sec / 1e12, alu["fp64"], "TFLOP/s", "measured now: FP64 fma loop (fddpd_alu_peak)"
    return (amount / sec / 1e12, alu["fp32_peak"], "TFLOP/s",
            "measured now: FP32 fma loop, the better of scalar and packed-pair (fddpd_alu_peak)")


def step_lower_bounds(work, mp, alu):
    """Milliseconds each resource needs for the whole step's algorithmic work (the stages'
    bytes through HBM as this staged design moves them; flops per pipe)."""
    tot = {"hbm": 0.0, "tensor": 0.0, "alu": 0.0, "fp64": 0.0}
    for bound, amount in work.values():
        tot[bound] += amount
    return {"hbm": tot["hbm"] / (mp["hbm_gbs"] * 1e9) * 1e3,
            "tensor": tot["tensor"] / (mp["bf16_tflops_sustained"] * 1e12) * 1e3,
            "fp32_alu": tot["alu"] / (alu["fp32_peak"] * 1e12) * 1e3,
            "fp64": tot["fp64"] / (alu["fp64"] * 1e12) * 1e3}


def source_files(stage: str, prec: str):
    """Sources of the kernel(s) a stage launches in a plan of precision `prec`."""
    p16 = prec != "fp32"
    bins = ("tcbin.cu", "tc_ptx.cuh") if p16 else ("bingemm.cu", "bingemm.cuh", "bingemm_f32.cu")
    fc = ("tc_gemm.cu", "tc_ptx.cuh", "pack16.cu") if p16 else ("fdcnn.cu",)
    files = {"zf_gram": ("zf.cu",), "zf_factor": ("zf.cu",),
             "zf_apply": ("tczf.cu", "tc_ptx.cuh") if p16 else ("zf.cu",),
             "fftpa_fwd": ("fftpa.cu", "fftpa.cuh", "fftpa_n11.cu"),
             "fftpa_adj": ("fftpa.cu", "fftpa.cuh", "fftpa_n11.cu"),
             "precode": bins, "combine": bins, "adj_combine": bins, "adj_precode": bins,
             "fc_fwd": fc, "fc_bwd_w": fc, "fc_bwd_d": fc, "fc_bwd_b": ("fdcnn.cu",),
             "conv_fwd": ("fdcnn.cu",), "conv_bwd": ("fdcnn.cu",), "step": ("update.cu",), "zmul": ("zf.cu",)}
    return files.get(stage, ("api.cu",))


def source_hash(stage: str, prec: str) -> str:
    h = hashlib.sha256()
    for f in source_files(stage, prec):
        with open(os.path.join(ROOT, "paper_2205_05158_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(stage: str, prec: str):
    """DRAM bytes per launch of `stage` from a committed ncu summary, if it was taken
    on the current source of that kernel (profiles/traffic.txt: stage precision
    source-hash bytes-per-launch)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    h = source_hash(stage, prec)
    for line in open(path):
        t = line.split()
        if len(t) >= 4 and not line.startswith("#") and t[0] == stage and t[1] == prec and t[2] == h:
            return float(t[3])
    return None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            t = [x.strip() for x in line.split(",")]
            if len(t) < 9:
                continue
            try:
                sm.append(float(t[1]))
                mx = max(mx, float(t[2]))
            except ValueError:
                continue
            for n, v in zip(names, t[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# training run of the 128 x 16 system (Sec. V-A: theta learned by gradient descent through
# the PA model): per-user FD-CNN parameters from the identity predistorter, 256 symbols
# per step, each step's mini-batch with its own symbols and channel realisations (drawn
# from a pool of `pool` distinct batches), the ZF build of that batch's channel inside
# the step; EVM / ACPR before and after on a training batch and on a held-out batch
# ---------------------------------------------------------------------------
TRAIN_STEPS = 500
TRAIN_POOL = 16   # distinct mini-batches (symbols and channel realisations) the run cycles through


def train_run(fd, torch, prec, optimizer, lr, steps, pool, stream, per_user=1, eval_every=50):
    import numpy as np

    import synth
    cfg = synth.CONFIGS["m128_k16_n2048_train"].with_(per_user=per_user)
    S = cfg.S
    stride = -(-S // cfg.S_per_real) * cfg.S_per_real       # batches start on realisation boundaries
    P_T = synth.transmit_power(cfg)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    plan = fd.Plan.from_config(cfg, P_T, max_symbols=S, precision=prec, stream=stream)
    theta0 = dev(synth.theta_init(cfg, cfg.seed, 0.0))      # the identity predistorter
    pa = dev(synth.pa_coefficients(cfg.seed, cfg.M, cfg.pa_nominal, cfg.pa_spread, cfg.pa_spread_orders)
             .astype(np.complex64))
    data = [tuple(dev(a) for a in synth.batch(cfg, S, b * stride)) for b in range(pool + 1)]   # last: held out
    R = data[0][1].shape[0]
    W = torch.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=torch.complex64, device="cuda") \
        if prec == fd.FDDPD_FP32 else None
    al = torch.empty((R, cfg.N_d), dtype=torch.float32, device="cuda")
    met = torch.zeros(5, dtype=torch.float64, device="cuda")

    def quality(theta, b):
        s_b, H_b = data[b]
        plan.precode(H_b, W, al)
        plan.distort(s_b, H_b, W, al, pa, theta, None, met)
        m = met.cpu().numpy()
        return {"evm_db": 10 * math.log10(m[1] / m[2]), "acpr_db": 10 * math.log10(m[3] / m[4])}

    before = {"train": quality(theta0, 0), "held_out": quality(theta0, pool)}
    theta = theta0.clone()
    plan.reset_optimizer()
    hist = torch.zeros((steps // eval_every + 1, 5), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        s_b, H_b = data[i % pool]
        plan.precode(H_b, W, al)
        plan.update(s_b, H_b, W, al, pa, theta, lr, 1, optimizer, met)
        if i % eval_every == 0:
            hist[i // eval_every].copy_(met)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    h = hist.cpu().numpy()
    after = {"train": quality(theta, 0), "held_out": quality(theta, pool)}
    return plan, cfg, data, W, al, pa, theta0, {
        "precision": {fd.FDDPD_FP32: "fp32", fd.FDDPD_BF16: "bf16", fd.FDDPD_FP16: "fp16"}[prec],
        "per_user": per_user, "optimizer": "adam" if optimizer == fd.FDDPD_ADAM else "gd", "lr": lr,
        "steps": steps, "symbols_per_step": S, "distinct_batches": pool, "ms_per_step": ms,
        "steps_per_s": 1e3 / ms, "before": before, "after": after,
        "evm_db_of_step": {str(j * eval_every): 10 * math.log10(h[j, 1] / h[j, 2])
                           for j in range(len(h)) if j * eval_every < steps}}


def fdnn_run(fd, torch, stream, S=560, reps=10):
    """The FD-NN comparison workload (Sec. III-C) on the 128 x 16, N = 2048 system: its
    forward chain (FP32 plan; every bin precoded) against the FD-CNN forward chain of an
    FP32 plan on the same symbols, both timed with CUDA events; and the running cost per
    UE and symbol of both DPDs from the paper's FLOP formulas (FD-NN: its network, U
    IDFT/DFT pairs and the guard-bin precoding; FD-CNN: convolution and dense layer)."""
    import numpy as np

    import synth
    cfg = synth.CONFIGS["m128_k16_n2048"].with_(S=S)
    w = synth.make_workload(cfg, fc_scale=0.05)
    H_all = synth.channel_all_bins(cfg)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s, Hd, Ha, pa = dev(w.s), dev(w.H), dev(H_all), dev(w.pa)
    R = w.H.shape[0]
    out = {"workload": f"m128_k16_n2048, {S} symbols, FP32 plans", "fdnn": {"L4": cfg.nn_L4, "D": cfg.nn_D,
                                                                          "layers": cfg.nn_layers}}
    met = torch.zeros(5, dtype=torch.float64, device="cuda")

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    pn = fd.Plan.fdnn_from_config(cfg, w.P_T, max_symbols=S, stream=stream)
    th = dev(synth.fdnn_theta_init(cfg, cfg.seed, out_scale=0.1))
    Wa = torch.empty((R, cfg.N, cfg.M, cfg.K), dtype=torch.complex64, device="cuda")
    ala = torch.empty((R, cfg.N), dtype=torch.float32, device="cuda")
    pn.precode(Ha, Wa, ala)
    pn.profile(True)
    pn.profile_read()
    ms_nn = timed(lambda: pn.distort(s, Hd, Wa, ala, pa, th, None, met))
    prof = pn.profile_read()
    m = met.cpu().numpy()
    out["fdnn_forward"] = {"value": S / (ms_nn / 1e3), "unit": UNIT, "ms": ms_nn,
                           "evm_db": 10 * math.log10(m[1] / m[2]), "acpr_db": 10 * math.log10(m[3] / m[4]),
                           "stages_ms": {k: v[0] / (reps + 1) for k, v in prof.items() if v[1] > 0}}
    pn.close()
    del Wa, ala, Ha
    pc = fd.Plan.from_config(cfg, w.P_T, max_symbols=S, precision=fd.FDDPD_FP32, stream=stream)
    W = torch.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=torch.complex64, device="cuda")
    al = torch.empty((R, cfg.N_d), dtype=torch.float32, device="cuda")
    pc.precode(Hd, W, al)
    thc = dev(w.theta)
    ms_cnn = timed(lambda: pc.distort(s, Hd, W, al, pa, thc, None, met))
    out["fdcnn_forward_fp32"] = {"value": S / (ms_cnn / 1e3), "unit": UNIT, "ms": ms_cnn}
    pc.close()
    # running cost per UE per OFDM symbol (the paper's counts, Sec. III-C and IV-B)
    U, N, B, Nd, L, D, Knn = cfg.K, cfg.N, cfg.M, cfg.N_d, cfg.nn_L4, cfg.nn_D, cfg.nn_layers
    nn_flops = (N * (4 * U * (L + 1) * D + 2 * (Knn - 1) * D * D + 4 * D * U) + 10 * U * N * math.log2(N)
                + 8 * (N - Nd) * U * B) / U
    cells = math.ceil(math.sqrt(Nd)) ** 2
    cnn_flops = 2 * cfg.N_conv * cfg.L_U * (2 * cfg.K_C ** 2 - 1) * cells + 8 * Nd * cfg.L_U * cells
    out["flops_per_ue_symbol"] = {"fdnn": nn_flops, "fdcnn": cnn_flops}
    return out


def regime_run(fd, torch, stream, S=1792, reps=5):
    """The per-subcarrier contractions as the symbols per channel realisation grow (14, 64,
    256; S = 1792 symbols in each case, the 128 x 16 x 2048 system, BF16 plan, precoder
    kept as its factors, forward chain): per contraction stage its milliseconds, its
    algorithmic bytes and flops (a complex multiply-add = 8 flops) as fractions of the
    measured HBM and sustained BF16 peaks.  Symbols and i.i.d. Rayleigh channel taps are
    drawn on the device from a seeded torch generator."""
    import numpy as np

    import synth
    base = synth.CONFIGS["m128_k16_n2048"]
    mp, _ = peaks()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    rows = []
    for Sr in (14, 64, 256):
        cfg = base.with_(S=S, S_per_real=Sr)
        R = -(-S // Sr)
        side = int(round(math.sqrt(cfg.Q)))
        lv = torch.tensor(synth.qam_levels(cfg.Q), dtype=torch.float32, device="cuda")
        idx = torch.randint(0, side, (2, S, cfg.K, cfg.N_d), device="cuda", generator=gen)
        s = torch.complex(lv[idx[0]], lv[idx[1]]).contiguous()
        del idx
        taps = torch.randn((R, cfg.T, cfg.K, cfg.M, 2), device="cuda", generator=gen) * math.sqrt(0.5 / cfg.T)
        taps = torch.complex(taps[..., 0], taps[..., 1]).to(torch.complex128)
        bins = torch.tensor(synth.data_bins(cfg.N, cfg.N_d), device="cuda", dtype=torch.float64)
        ph = torch.exp(-2j * math.pi * bins[:, None] * torch.arange(cfg.T, device="cuda", dtype=torch.float64)[None] / cfg.N)
        H = torch.einsum("bt,rtkm->rbkm", ph, taps).to(torch.complex64).contiguous()
        del taps, ph
        pa = torch.from_numpy(synth.pa_coefficients(cfg.seed, cfg.M, cfg.pa_nominal, 0.1).astype(np.complex64)).cuda()
        theta = torch.from_numpy(synth.theta_init(cfg, cfg.seed, 0.0)).cuda()
        plan = fd.Plan.from_config(cfg, synth.transmit_power(cfg), max_symbols=S, precision=fd.FDDPD_BF16,
                                   stream=stream)
        al = torch.empty((R, cfg.N_d), dtype=torch.float32, device="cuda")
        met = torch.zeros(5, dtype=torch.float64, device="cuda")
        plan.precode(H, None, al)
        plan.distort(s, H, None, al, pa, theta, None, met)
        torch.cuda.synchronize()
        plan.profile(True)
        plan.profile_read()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            plan.distort(s, H, None, al, pa, theta, None, met)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        prof = plan.profile_read()
        plan.profile(False)
        plan.close()
        work = stage_work(cfg, S, "bf16")
        flops = 8.0 * cfg.M * cfg.K * cfg.N_d * S
        entry = {"S_per_real": Sr, "realisations": R, "forward_ms": ms, "symbols_per_s": S / (ms / 1e3)}
        for st in ("precode", "combine", "zmul"):
            if st in prof and prof[st][1] > 0:
                t = prof[st][0] / prof[st][1] / 1e3
                e = {"ms": t * 1e3, "hbm_bytes": work[st][1], "hbm_frac": work[st][1] / t / (mp["hbm_gbs"] * 1e9)}
                if st != "zmul":
                    e["tflops"] = flops / t / 1e12
                    e["tensor_frac"] = flops / t / (mp["bf16_tflops_sustained"] * 1e12)
                entry[st] = e
        rows.append(entry)
        del s, H, pa, theta, al
        torch.cuda.empty_cache()
    return {"symbols": S, "system": "M=128 K=16 N=2048 N_d=1200, BF16, forward chain", "rows": rows}


def batched_run(fd, torch, stream, n=512, S=50, lanes=8, reps=3):
    """The batched uneven workload: n independent instances (M 32..256, K 4..32 with
    K <= M / 4, N 512..4096 with about 58 % of the bins occupied, 64-QAM, i.i.d. Rayleigh
    taps, orders {1,3} or {1,3,5}), BF16 plans with the precoder kept as its factors, each
    autotuned (choices stored per shape), the forward chain of every instance recorded on
    `lanes` concurrent lanes of one CUDA graph and replayed as one launch; against the same
    calls one by one on one stream.  The symbols and channel taps of this timing run are
    drawn on the device from a seeded torch generator (shapes and PA sets from synth)."""
    import numpy as np

    import synth
    cfgs = synth.uneven_instances(n, S=S)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    free0 = torch.cuda.mem_get_info()[0]
    insts = []
    for cfg in cfgs:
        if torch.cuda.mem_get_info()[0] < 0.12 * free0:   # keep well inside the device memory
            break
        R = -(-S // cfg.S_per_real)
        side = int(round(math.sqrt(cfg.Q)))
        lv = torch.tensor(synth.qam_levels(cfg.Q), dtype=torch.float32, device="cuda")
        idx = torch.randint(0, side, (2, S, cfg.K, cfg.N_d), device="cuda", generator=gen)
        s = torch.complex(lv[idx[0]], lv[idx[1]]).contiguous()
        taps = torch.randn((R, cfg.T, cfg.K, cfg.M, 2), device="cuda", generator=gen) * math.sqrt(0.5 / cfg.T)
        taps = torch.complex(taps[..., 0], taps[..., 1]).to(torch.complex128)
        bins = torch.tensor(synth.data_bins(cfg.N, cfg.N_d), device="cuda", dtype=torch.float64)
        ph = torch.exp(-2j * math.pi * bins[:, None] * torch.arange(cfg.T, device="cuda", dtype=torch.float64)[None] / cfg.N)
        H = torch.einsum("bt,rtkm->rbkm", ph, taps).to(torch.complex64).contiguous()
        pa = torch.from_numpy(synth.pa_coefficients(cfg.seed, cfg.M, cfg.pa_nominal, 0.1).astype(np.complex64)).cuda()
        theta = torch.from_numpy(synth.theta_init(cfg, cfg.seed, 0.0)).cuda()
        try:
            plan = fd.Plan.from_config(cfg, synth.transmit_power(cfg), max_symbols=S, precision=fd.FDDPD_BF16,
                                       stream=stream)
        except fd.FddpdError:
            break
        al = torch.empty((R, cfg.N_d), dtype=torch.float32, device="cuda")
        plan.precode(H, None, al)
        insts.append((cfg, plan, s, H, al, pa, theta))
    fd.autotune_forget()
    t0 = time.perf_counter()
    for cfg, plan, s, H, al, pa, theta in insts:
        plan.autotune(s, H, None, al, pa, theta, reps=2)
    tune_s = time.perf_counter() - t0
    ys = [torch.empty_like(x[2]) for x in insts]

    def one_by_one():
        for (cfg, plan, s, H, al, pa, theta), y in zip(insts, ys):
            plan.distort(s, H, None, al, pa, theta, y)

    one_by_one()
    torch.cuda.synchronize()
    ref = [y.clone() for y in ys]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        one_by_one()
    b.record(stream)
    torch.cuda.synchronize()
    ms_seq = a.elapsed_time(b) / reps
    main = torch.cuda.Stream()
    t0 = time.perf_counter()
    with fd.Graph.record_lanes(main, lanes) as (g, lane_streams):
        for i, (cfg, plan, s, H, al, pa, theta) in enumerate(insts):
            plan.set_stream(lane_streams[i % lanes])
            plan.distort(s, H, None, al, pa, theta, ys[i])
    rec_s = time.perf_counter() - t0
    g.launch()
    main.synchronize()
    a.record(main)
    for _ in range(reps):
        g.launch()
    b.record(main)
    main.synchronize()
    ms_graph = a.elapsed_time(b) / reps
    same = all(torch.equal(y, r) for y, r in zip(ys, ref))
    shapes = {(c.M, c.K, c.N) for c, *_ in insts}
    tc = sum(p.get_option(fd.FDDPD_OPT_TENSOR_CONTRACTIONS) for _, p, *_ in insts)
    one_cta = sum(p.get_option(fd.FDDPD_OPT_ROW_CTAS) == 1 for _, p, *_ in insts)
    one_bin_cta = sum(p.get_option(fd.FDDPD_OPT_CONTRACTION_CTAS) == 1 and p.get_option(fd.FDDPD_OPT_TENSOR_CONTRACTIONS)
                      for _, p, *_ in insts)
    half_items = sum(p.get_option(fd.FDDPD_OPT_CONTRACTION_ITEM) == 1 and p.get_option(fd.FDDPD_OPT_TENSOR_CONTRACTIONS)
                     for _, p, *_ in insts)
    nsym = len(insts) * S
    for _, p, *_ in insts:
        p.close()
    del g
    return {"instances": len(insts), "requested": n, "symbols_per_instance": S, "distinct_shapes": len(shapes),
            "lanes": lanes, "graph": {"value": nsym / (ms_graph / 1e3), "unit": UNIT, "ms": ms_graph},
            "one_by_one": {"value": nsym / (ms_seq / 1e3), "unit": UNIT, "ms": ms_seq},
            "graph_equals_one_by_one": same, "autotune_s": tune_s, "record_s": rec_s,
            "autotuned": {"tensor_core_contractions": tc, "row_kernels_one_cta_per_sm": one_cta,
                          "contractions_one_cta_per_sm": one_bin_cta, "contractions_half_items": half_items},
            "precision": "bf16", "data": "device-drawn seeded symbols and channel taps"}


def torch_optim_run(fd, torch, plan, data, W, al, pa, theta0, steps=20, lr=1e-3):
    """The same plan trained through the autograd wrapper (fddpd_loss) by torch.optim.Adam,
    against fddpd_update's own Adam over the same steps on the first batch."""
    s_b, H_b = data[0]
    plan.precode(H_b, W, al)
    th = torch.nn.Parameter(theta0.clone())
    opt = torch.optim.Adam([th], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    losses = []
    for _ in range(steps):
        opt.zero_grad()
        loss = fd.fddpd_loss(th, plan, s_b, H_b, W, al, pa)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    ref = theta0.clone()
    plan.reset_optimizer()
    plan.update(s_b, H_b, W, al, pa, ref, lr, steps, fd.FDDPD_ADAM)
    torch.cuda.synchronize()
    d = (th.detach() - ref).double().norm() / (ref - theta0).double().norm()
    return {"steps": steps, "lr": lr, "loss_first": losses[0], "loss_last": losses[-1],
            "rel_diff_vs_library_adam": float(d)}


# ---------------------------------------------------------------------------
# the reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_step(cfg, w, n_sym: int):
    """ZF of the realisations of the first n_sym symbols + one update iteration over them."""
    import oracle
    d = oracle.dims_from_config(cfg, w.P_T)
    R = -(-n_sym // cfg.S_per_real)
    W, al = oracle.precode(d, w.H[:R])
    th, met = oracle.update(d, w.s[:n_sym], w.H[:R], W, al, w.pa, w.theta, LR, 1)
    return met


def run_reference(args):
    rank, _, _ = rank_env()
    if rank != 0:
        return
    import oracle
    import synth
    cfg = synth.CONFIGS["m128_k16_n2048"]
    n = max(1, args.ref_sample)
    w = synth.make_workload(cfg, S=n, fc_scale=0.05)
    oracle.build()
    for _ in range(args.warmup):
        oracle_step(cfg, w, n)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(cfg, w, n)
        t.append(time.perf_counter() - t0)
    sec = sum(t) / len(t)
    value = n / sec
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD,
                      "sample": f"{n} symbols per step"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"ZF of the {-(-n // cfg.S_per_real)} 1200-subcarrier realisation(s) of "
                                      f"{n} symbols + forward, adjoint and GD step over them"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# ranks: one process per GPU running an independent replica (symbols and channel
# realisations are independent units, so the data path exchanges nothing); a rank draws
# its own symbols and channels, the timing is the maximum over ranks, and the value
# counts every rank's symbols
# ---------------------------------------------------------------------------
def rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_config(rank: int, symbols: int):
    import synth
    return synth.CONFIGS["m128_k16_n2048"].with_(seed=rank, S=symbols)


def max_over_ranks(x: float, dist, device) -> float:
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, symbols: int, seconds: float) -> float:
    return world * symbols / seconds


def data_parallel_step(backward, all_reduce, apply, world: int):
    """One data-parallel training step, the one exchange the path has on more than one
    GPU: this rank's gradient over its own symbols (backward() returns it), summed over
    the ranks in place by all_reduce, then the same step -- the sum scaled by 1 / world,
    the gradient of the mean loss over every rank's symbols -- applied on every rank."""
    g = backward()
    if world > 1:
        all_reduce(g)
    apply(g, 1.0 / world)
    return g


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import synth
    import paper_2205_05158_gb300 as fd

    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    prec_name = args.precision or "bf16"
    prec = {"fp32": fd.FDDPD_FP32, "bf16": fd.FDDPD_BF16, "fp16": fd.FDDPD_FP16}[prec_name]
    cfg = rank_config(rank, args.symbols)
    S = cfg.S
    w = synth.make_workload(cfg, fc_scale=0.05)
    R = w.H.shape[0]
    stream = torch.cuda.current_stream()
    alu = alu_peaks(fd, stream)
    plan = fd.Plan.from_config(cfg, w.P_T, max_symbols=S, precision=prec, stream=stream)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s, H, pa, theta0 = dev(w.s), dev(w.H), dev(w.pa), dev(w.theta)
    theta = theta0.clone()
    W = torch.empty((R, cfg.N_d, cfg.M, cfg.K), dtype=torch.complex64, device="cuda")
    al = torch.empty((R, cfg.N_d), dtype=torch.float32, device="cuda")
    met = torch.zeros(5, dtype=torch.float64, device="cuda")

    # W is not formed on the training path: fddpd_precode keeps the precoder as its factors
    # and the chain applies alpha H^H (Z s) (16-bit plans; FP32 plans form W)
    Wt = W if prec == fd.FDDPD_FP32 else None

    # one training step of a plan: on one GPU fddpd_update (forward, adjoint, GD step); on
    # several, data-parallel: fddpd_backward on this rank's symbols, the gradients summed
    # over the ranks (NCCL all-reduce on the plan's stream), the same averaged step on
    # every rank (fddpd_apply_gradient)
    def train_step(p, th, mt, Wx, alx, gbuf):
        p.precode(H, Wx, alx)
        if world == 1:
            p.update(s, H, Wx, alx, pa, th, LR, 1, fd.FDDPD_GD, mt)
            return
        data_parallel_step(lambda: (p.backward(s, H, Wx, alx, pa, th, gbuf, mt), gbuf)[1], dist.all_reduce,
                           lambda g, sc: p.apply_gradient(th, g, LR, fd.FDDPD_GD, sc), world)

    gbuf = torch.empty(plan.theta_len, dtype=torch.float32, device="cuda") if world > 1 else None

    def step():
        train_step(plan, theta, met, Wt, al, gbuf)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier()

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    plan.profile(True)
    plan.profile_read()
    launches0 = plan.launch_count
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    prof = plan.profile_read()
    plan.profile(False)
    launches = plan.launch_count - launches0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    value = job_rate(world, S, ms / 1e3)

    # forward-only (running mode) throughput on the same inputs, informational
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        plan.distort(s, H, Wt, al, pa, theta, None, met)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1) / args.steps
    m = met.cpu().numpy()
    evm_db = 10 * math.log10(m[1] / m[2])
    acpr_db = 10 * math.log10(m[3] / m[4])

    # symbol errors at the users: forward chain, receiver noise at a mean per-subcarrier
    # SNR of SER_SNR_DB, nearest-point decisions (informational)
    y_ser = torch.empty_like(s)
    ser_counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    N0 = float((al.double() ** 2).mean()) * 10 ** (-SER_SNR_DB / 10)
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for it in range(args.steps):
        plan.distort(s, H, Wt, al, pa, theta, y_ser, None)
        plan.ser(y_ser, s, al, cfg.Q, N0, 1000 + it, ser_counts)
    q1.record(stream)
    torch.cuda.synchronize()
    ser_ms = q0.elapsed_time(q1) / args.steps
    sc = ser_counts.cpu().numpy()

    # roofline of the dominant stage
    mp, src = peaks()
    work = stage_work(cfg, S, prec_name)
    stage, (tot_ms, cnt) = max(((k, v) for k, v in prof.items() if k in work and v[1] > 0), key=lambda kv: kv[1][0])
    bound, amount = work[stage]
    per_launch_ms = tot_ms / cnt
    achieved, peak, unit, peak_src = roofline_of(bound, amount, per_launch_ms, mp, src, alu)
    traffic = measured_traffic(stage, prec_name)
    stages_out = {}
    for k, v in prof.items():
        if v[1] <= 0:
            continue
        stages_out[k] = {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
        if k in work:
            a, pk, u, _ = roofline_of(work[k][0], work[k][1], v[0] / v[1], mp, src, alu)
            stages_out[k].update({"bound": work[k][0], "achieved": a, "unit": u, "frac": a / pk})
    # step-level roofline: the largest resource lower bound of the whole step over its time
    lb = step_lower_bounds(work, mp, alu)
    plan.precode(H, W, al)               # W itself, for the final FP64 check of H_k W_k = I
    zf_res = plan.zf_residual(H, W, 1)   # (all subcarriers) and the oracle comparison
    plan.precode(H, Wt, al)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if prec_name == "fp32" else f"{prec_name}+f32",
           "data": "synthetic",
           "config": {"workload": WORKLOAD,
                      "symbols_per_step": S, "realisations_per_step": R, "precision": prec_name,
                      "arithmetic": ARITHMETIC if prec_name == "bf16" else "default options of the plan",
                      "step": "ZF (Gram + factor; the precoder applied through its factors, W not formed) + FD-CNN + "
                              "precode + IFFT/PA/FFT + combine + loss + adjoint + GD update",
                      "l2": "inputs larger than L2 (H 2.8 GB), no flush",
                      "parallelism": (f"data-parallel x{world}: each rank its own symbols and channels, "
                                      "gradients summed by an NCCL all-reduce, the same step on every rank")
                                     if world > 1 else "single GPU"},
           "roofline": {"kernel": stage, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                        "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                        "work_per_launch": amount},
           "step_roofline": {"lower_bounds_ms": lb, "binding": max(lb, key=lb.get),
                             "frac": max(lb.values()) / ms},
           "alu_peaks_tflops": alu,
           "zf_residual_fp64": zf_res,
           "stages": stages_out,
           "forward_only": {"value": world * S / (fwd_ms / 1e3), "unit": UNIT, "ms": fwd_ms},
           "quality": {"evm_db": evm_db, "acpr_db": acpr_db},
           "ser": {"value": world * S / (ser_ms / 1e3), "unit": UNIT, "ms": ser_ms, "snr_db": SER_SNR_DB,
                   "ser": float(sc[0]) / max(1, int(sc[1])), "symbols": int(sc[1])},
           "gpu_launches": launches,
           "clocks": clk}

    # the faster arithmetic beside the headline: FP32 Gram factor and x(t) kept in BF16
    if prec_name == "bf16" and not args.no_fast_variant:
        plan.set_option(fd.FDDPD_OPT_FACTOR_FP64, 0)
        plan.set_option(fd.FDDPD_OPT_KEEP_PA_INPUT, 1)
        thf = theta0.clone()
        metf = torch.zeros(5, dtype=torch.float64, device="cuda")

        def stepf():
            train_step(plan, thf, metf, Wt, al, gbuf)

        for _ in range(max(3, args.warmup)):
            stepf()
        torch.cuda.synchronize()
        plan.profile(True)
        plan.profile_read()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for _ in range(args.steps):
            stepf()
        v1.record(stream)
        torch.cuda.synchronize()
        proff = plan.profile_read()
        plan.profile(False)
        msf = max_over_ranks(v0.elapsed_time(v1) / args.steps, dist, "cuda")
        plan.distort(s, H, Wt, al, pa, theta0, None, metf)
        mf = metf.cpu().numpy()
        out["fast_variant"] = {"arithmetic": FAST_ARITHMETIC, "value": job_rate(world, S, msf / 1e3), "unit": UNIT,
                               "ms_per_step": msf, "evm_db": 10 * math.log10(mf[1] / mf[2]),
                               "acpr_db": 10 * math.log10(mf[3] / mf[4]),
                               "stages_ms": {k: v[0] / args.steps for k, v in proff.items() if v[1] > 0}}
        plan.set_option(fd.FDDPD_OPT_FACTOR_FP64, 1)
        plan.set_option(fd.FDDPD_OPT_KEEP_PA_INPUT, 0)

    # end to end through the C-ABI with host buffers (pinned), copies inside the timed region
    if not args.no_e2e:
        hs = torch.from_numpy(w.s).pin_memory().numpy()
        hH = torch.from_numpy(w.H).pin_memory().numpy()
        hpa = torch.from_numpy(w.pa).pin_memory().numpy()
        hth = torch.from_numpy(w.theta.copy()).pin_memory().numpy()
        hmet = torch.zeros(5, dtype=torch.float64).pin_memory().numpy()
        if world > 1:   # the data-parallel step from host buffers: copies in, step, theta and metrics out
            ts, tH, tpa, tth = (torch.from_numpy(a) for a in (hs, hH, hpa, hth))
            ds, dH, dpa, dth = (torch.empty_like(a, device="cuda") for a in (ts, tH, tpa, tth))
            dmet = torch.zeros(5, dtype=torch.float64, device="cuda")

            def host_step():
                for dst, src in ((ds, ts), (dH, tH), (dpa, tpa), (dth, tth)):
                    dst.copy_(src, non_blocking=True)
                plan.precode(dH, Wt, al)
                data_parallel_step(lambda: (plan.backward(ds, dH, Wt, al, dpa, dth, gbuf, dmet), gbuf)[1],
                                   dist.all_reduce, lambda g, sc: plan.apply_gradient(dth, g, LR, fd.FDDPD_GD, sc),
                                   world)
                tth.copy_(dth, non_blocking=True)
                torch.from_numpy(hmet).copy_(dmet, non_blocking=True)
                torch.cuda.synchronize()
        else:
            def host_step():
                plan.update_host(hs, hH, hpa, hth, LR, 1, fd.FDDPD_GD, hmet)
        for _ in range(max(1, args.warmup)):
            host_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        sec = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, "cuda")
        out["e2e"] = {"value": job_rate(world, S, sec), "unit": UNIT,
                      "h2d_bytes_per_step": int(hs.nbytes + hH.nbytes + hpa.nbytes + hth.nbytes),
                      "d2h_bytes_per_step": int(hth.nbytes + 5 * 8)}

    # the plain FP32 plan on the same inputs and the same step (the mixed-precision plan's
    # comparison point), timed the same way
    if prec_name != "fp32" and not args.no_fp32_compare:
        plan32 = fd.Plan.from_config(cfg, w.P_T, max_symbols=S, precision=fd.FDDPD_FP32, stream=stream)
        th32 = theta0.clone()
        met32 = torch.zeros(5, dtype=torch.float64, device="cuda")
        W32 = torch.empty_like(W)
        al32 = torch.empty_like(al)

        def step32():
            train_step(plan32, th32, met32, W32, al32, gbuf)

        for _ in range(2):
            step32()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n32 = max(2, args.steps // 2)
        g0.record(stream)
        for _ in range(n32):
            step32()
        g1.record(stream)
        torch.cuda.synchronize()
        ms32 = g0.elapsed_time(g1) / n32
        plan32.distort(s, H, W32, al32, pa, theta, None, met32)
        m32 = met32.cpu().numpy()
        out["fp32_plan"] = {"value": world * S / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32,
                            "evm_db": 10 * math.log10(m32[1] / m32[2]), "acpr_db": 10 * math.log10(m32[3] / m32[4])}
        del plan32

    # the informational sections below report their own failure instead of losing the line
    def section(name, fn):
        try:
            out[name] = fn()
        except Exception as exc:   # noqa: BLE001
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    if rank == 0 and not args.no_fdnn:
        section("fdnn_comparison", lambda: fdnn_run(fd, torch, stream))

    # the contractions as the symbols per realisation grow (rank 0, informational)
    if rank == 0 and not args.no_regime:
        section("regime_sweep", lambda: regime_run(fd, torch, stream))

    # the batched uneven workload: 512 instances in one graph launch (rank 0, informational)
    if rank == 0 and not args.no_batched:
        section("batched_uneven", lambda: batched_run(fd, torch, stream))

    # the training run of the 128 x 16 system (rank 0; informational, outside the timed step)
    def training():
        runs = []
        # per-user parameters (the configuration's own), mixed precision, the paper's Adam and
        # plain GD; the shared network for comparison; FP32 with torch.optim beside it
        for prec_, pu_, opt_, lr_ in ((fd.FDDPD_BF16, 1, fd.FDDPD_ADAM, 1e-3), (fd.FDDPD_BF16, 1, fd.FDDPD_GD, 30.0),
                                      (fd.FDDPD_BF16, 0, fd.FDDPD_ADAM, 1e-3), (fd.FDDPD_FP32, 1, fd.FDDPD_ADAM, 1e-3)):
            tp, tcfg, tdata, tW, tal, tpa, tth0, res = train_run(fd, torch, prec_, opt_, lr_, args.train_steps,
                                                                 TRAIN_POOL, stream, per_user=pu_)
            if prec_ == fd.FDDPD_FP32:
                res["torch_optim"] = torch_optim_run(fd, torch, tp, tdata, tW, tal, tpa, tth0)
            runs.append(res)
            tp.close()
            del tdata
        return runs

    if rank == 0 and not args.no_train:
        section("training", training)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        plan.precode(H, W, al)
        out["cpu_baseline"] = cpu_baseline(cfg, w, args.cpu_sample, plan, s, H, W, al, pa, theta0)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def cpu_baseline(cfg, w, n_sym, plan, s, H, W, al, pa, theta0):
    """Oracle (as it stands) on a bounded sample; also the EVM delta of the GPU on it."""
    import numpy as np
    import torch

    import oracle
    oracle.build()
    t0 = time.perf_counter()
    met_o = oracle_step(cfg, w, n_sym)
    sec = time.perf_counter() - t0
    d = oracle.dims_from_config(cfg, w.P_T)
    R = -(-n_sym // cfg.S_per_real)
    Wo, alo = oracle.precode(d, w.H[:R])
    _, meto = oracle.distort(d, w.s[:n_sym], w.H[:R], Wo, alo, w.pa, w.theta)
    met = torch.zeros(5, dtype=torch.float64, device="cuda")
    plan.distort(s[:n_sym], H, W, al, pa, theta0, None, met, S=n_sym)
    m = met.cpu().numpy()
    return {"value": n_sym / sec, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"ZF of the {R} 1200-subcarrier realisation(s) of {n_sym} symbols + forward, adjoint and "
                      f"GD step over them",
            "seconds": sec,
            "evm_db_oracle": 10 * math.log10(meto[1] / meto[2]),
            "evm_db_gpu": 10 * math.log10(m[1] / m[2]),
            "acpr_db_oracle": 10 * math.log10(meto[3] / meto[4]),
            "acpr_db_gpu": 10 * math.log10(m[3] / m[4])}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
