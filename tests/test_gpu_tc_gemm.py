"""The tcgen05 tensor-core GEMM against a plain PyTorch FP32 matmul of the same
16-bit operands (products of 16-bit values are exact in FP32, so only the
summation order differs)."""
import pytest

pytestmark = pytest.mark.gpu


def _mk(rows, K, dtype, gen):
    import torch
    ld = (K + 7) // 8 * 8 + 8          # padded rows: the padding must never be read
    full = torch.randn(rows, ld, generator=gen, device="cuda").to(dtype)
    full[:, K:] = float("nan")
    return full, full[:, :K]


@pytest.mark.parametrize("M,N,K,splits,dtype", [
    (128, 256, 64, 1, "bf16"), (300, 520, 200, 1, "bf16"), (1000, 2400, 2450, 1, "bf16"),
    (256, 512, 4096, 4, "bf16"), (130, 260, 1000, 3, "fp16"), (2400, 2450, 3000, 4, "bf16")])
def test_tc_gemm_matches_fp32_matmul(M, N, K, splits, dtype):
    import torch
    dt = torch.bfloat16 if dtype == "bf16" else torch.float16
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    Af, A = _mk(M, K, dt, g)
    Bf, B = _mk(N, K, dt, g)
    C = torch.zeros(M, N + 5, device="cuda")
    from paper_2205_05158_gb300 import binding
    L = binding.load()
    rc = L.fddpd_tc_gemm(M, N, K, Af.data_ptr(), Af.stride(0), Bf.data_ptr(), Bf.stride(0), C.data_ptr(), C.stride(0),
                         1 if dt == torch.bfloat16 else 0, splits, torch.cuda.current_stream().cuda_stream)
    assert rc == 0, L.fddpd_last_error(None)
    ref = A.float() @ B.float().T
    err = (C[:, :N] - ref).abs().max().item()
    scale = (A.float().abs() @ B.float().abs().T).max().item()
    assert err <= 1e-5 * scale, (err, scale)
    assert torch.all(C[:, N:] == 0)
