"""The tcgen05 GEMM (TMA + tensor memory) against a plain PyTorch fp32 matmul of the same bf16 data."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 64, 192), (8192, 256, 256), (256, 16, 1024),
                                   (1000, 128, 64), (256, 256, 8192)])
def test_gemm_matches_fp32_reference(M, N, K):
    import torch

    import paper_2604_05794_b300 as hf
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    a = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    b = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    c = hf.gemm_bf16(a, b)
    torch.cuda.synchronize()
    ref = a.float() @ b.float().T
    err = (c - ref).abs().max().item()
    scale = ref.abs().max().item()
    # bf16 products are exact in fp32; only the summation order differs
    assert err <= 2e-5 * scale + 1e-4 * (K / 64) ** 0.5, (err, scale)


def test_gemm_rejects_bad_shapes():
    import torch

    import paper_2604_05794_b300 as hf
    a = torch.zeros((128, 100), device="cuda", dtype=torch.bfloat16)
    b = torch.zeros((16, 100), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(hf.HairFuseError):
        hf.gemm_bf16(a, b)
