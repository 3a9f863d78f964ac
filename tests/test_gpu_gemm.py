"""The hand-written tcgen05 BF16 GEMM (C = A B^T, FP32 accumulation in
tensor memory) against a plain PyTorch fp32 matmul of the same bf16
operands, for every fused epilogue and for ragged shapes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(128, 256, 64), (300, 512, 288), (512, 16, 4096), (1000, 100, 40), (4096, 512, 512),
          (130, 17, 24)]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2608_07580_b300 import firert
    return torch, firert


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("epi", [0, 1, 2, 3])
def test_gemm_matches_fp32_reference(env, M, N, K, epi):
    torch, fr = env
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K + epi)
    A = (torch.randn(M, K, device="cuda", generator=g) * 0.5).to(torch.bfloat16)
    B = (torch.randn(N, K, device="cuda", generator=g) * 0.5).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g) if epi in (0, 1, 2) else None
    mask = (torch.randn(M, N, device="cuda", generator=g)).to(torch.bfloat16) if epi == 3 else None
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    ref = A.float() @ B.float().T
    if bias is not None:
        ref = ref + bias
    if epi == 1:
        ref = torch.relu(ref)
    elif epi == 2:
        ref = torch.tanh(ref)
    elif epi == 3:
        ref = ref * (mask.float() > 0)
    Cf = torch.full((M, N), float("nan"), device="cuda")
    Cb = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
    CbT = torch.empty((N, M), dtype=torch.bfloat16, device="cuda")
    fr.gemm_bf16(A, B, epi=epi, bias=bias, mask=mask, Cf=Cf, Cb=Cb, CbT=CbT, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    scale = (A.float().abs() @ B.float().abs().T).clamp_min(1e-3)
    assert torch.max((Cf - ref).abs() / scale).item() < 1e-5
    assert torch.max((Cb.float() - ref).abs() / (ref.abs() + scale * 1e-3)).item() < 1e-2
    assert torch.equal(CbT, Cb.T.contiguous())


def test_gemm_accumulate(env):
    torch, fr = env
    A = torch.randn(256, 64, device="cuda").to(torch.bfloat16)
    B = torch.randn(32, 64, device="cuda").to(torch.bfloat16)
    Cf = torch.ones(256, 32, device="cuda")
    fr.gemm_bf16(A, B, Cf=Cf, accumulate=True)
    torch.cuda.synchronize()
    ref = 1.0 + A.float() @ B.float().T
    assert torch.allclose(Cf, ref, atol=1e-3, rtol=1e-5)


def test_gemm_rejects_unaligned_operands(env):
    """Operand bases must be 16-byte aligned (TMA and the 16-byte copies):
    a base 8 bytes off is refused before any launch."""
    torch, fr = env
    flat = torch.zeros(64 * 64 + 4, device="cuda", dtype=torch.bfloat16)
    A = flat[4:].view(64, 64)             # contiguous, 8 bytes past a 16-byte boundary
    assert A.is_contiguous() and A.data_ptr() % 16 == 8
    B = torch.zeros(16, 64, device="cuda", dtype=torch.bfloat16)
    Cf = torch.zeros(64, 16, device="cuda")
    with pytest.raises(fr.FireError):
        fr.gemm_bf16(A, B, Cf=Cf)
