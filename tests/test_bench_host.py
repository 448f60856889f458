"""Host-side logic of bench.py (no GPU): the algorithmic work per launch behind the
roofline fractions, and the rule that a committed DRAM-traffic figure is reported only
while the kernel's sources are the ones it was measured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402

STAGES = ["zf_gram", "zf_factor", "zf_apply", "conv_fwd", "fc_fwd", "precode", "fftpa_fwd", "combine",
          "adj_combine", "fftpa_adj", "adj_precode", "fc_bwd_w", "fc_bwd_b", "fc_bwd_d", "conv_bwd", "step", "zmul"]


def test_stage_work_of_the_benchmark_step():
    """128 antennas, 16 users, N = 2048 (1200 data bins), 2000 symbols over 143
    realisations, F = 2 x 35^2 = 2450 dense inputs, BF16 plan: figures worked out by hand
    from the per-stage formulas (dense layer 2 x cols x 2N_d x F; row kernels two
    5 N log2 N transforms plus 19 flops per tap and sample forward, 24 per tap and 26 per
    sample for the adjoint, which transforms three times when it recomputes x(t); the
    contractions' operand and plane bytes)."""
    w = bench.stage_work(synth.CONFIGS["m128_k16_n2048"], 2000, "bf16")
    assert set(w) == set(STAGES)
    assert w["fc_fwd"] == ("tensor", 376_320_000_000)
    assert w["fc_bwd_w"][1] == w["fc_bwd_d"][1] == w["fc_fwd"][1]
    assert w["fftpa_fwd"] == ("alu", 2000 * 128 * (10 * 2048 * 11 + 2048 * 4 * 19))
    # the adjoint recomputes x(t) (three transforms); with x(t) kept, two
    assert w["fftpa_adj"] == ("alu", 2000 * 128 * (3 * 5 * 2048 * 11 + 2048 * (24 * 4 + 26)))
    assert bench.stage_work(synth.CONFIGS["m128_k16_n2048"], 2000, "bf16", kept_xt=True)["fftpa_adj"] == \
        ("alu", 121_634_816_000)
    # the Gram factor in FP64 by default, FP32 when the plan selects it
    assert w["zf_factor"][0] == "fp64"
    assert bench.stage_work(synth.CONFIGS["m128_k16_n2048"], 2000, "bf16", fp64_factor=False)["zf_factor"][0] == "alu"
    # alpha W s: W's 16-bit copy per realisation, s_tilde in, x_hat out (FP32)
    assert w["precode"] == ("hbm", 143 * 1200 * 128 * 16 * 4 + 2000 * 16 * 1200 * 8 + 2000 * 128 * 1200 * 8)
    # H's copy, the BF16 X^PA plane, s in and y out
    assert w["combine"] == ("hbm", 3_248_947_200)
    assert w["zf_apply"] == ("hbm", 143 * 1200 * 16 * 128 * 20 + 143 * 1200 * 4)
    # theta, its gradient and the update's write: 5,882,438 parameters
    assert w["step"] == ("hbm", 12 * 5_882_438)


def test_fp32_plans_count_fp32_operands():
    cfg = synth.CONFIGS["m64_k8_n1024"]
    w16, w32 = bench.stage_work(cfg, 100, "bf16"), bench.stage_work(cfg, 100, "fp32")
    R = -(-100 // cfg.S_per_real)
    # H / W operands: 8 bytes in FP32 plans, 4 in 16-bit ones; the planes 8 and 4
    assert w32["precode"][1] - w16["precode"][1] == R * cfg.N_d * cfg.M * cfg.K * 4
    assert w32["combine"][1] - w16["combine"][1] == R * cfg.N_d * cfg.M * cfg.K * 4 + 100 * cfg.M * cfg.N_d * 4
    assert w32["fc_fwd"][0] == "alu" and w32["zf_factor"][0] == "fp64"


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_every_stage_names_existing_sources(prec):
    for st in STAGES:
        for f in bench.source_files(st, prec):
            assert os.path.exists(os.path.join(ROOT, "paper_2205_05158_gb300", "csrc", f)), (st, f)


def test_committed_traffic_lines_parse():
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        stage, prec, h, nbytes = line.split()[:4]
        assert stage in STAGES and prec in ("fp32", "bf16", "fp16")
        assert len(h) == 12 and int(h, 16) >= 0 and float(nbytes) > 0


def test_traffic_is_reported_only_for_the_measured_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2205_05158_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "update.cu").write_text("// version 1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.source_hash("step", "fp32")
    (tmp_path / "profiles" / "traffic.txt").write_text(f"# stage precision hash bytes\nstep fp32 {h} 12345\n")
    assert bench.measured_traffic("step", "fp32") == 12345.0
    assert bench.measured_traffic("step", "bf16") is None          # another precision
    (csrc / "update.cu").write_text("// version 2\n")              # the kernel changed
    assert bench.measured_traffic("step", "fp32") is None
