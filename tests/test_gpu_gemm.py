"""The tensor-core BF16 GEMM of the surrogate against a plain PyTorch FP32
matmul of the same BF16-rounded operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2102_01887_b300 import build, llama
    build.build()
    llama.load()
    return llama


@pytest.mark.parametrize("m,n,k", [(128, 64, 64), (128, 256, 64), (256, 128, 128), (384, 256, 256),
                                   (200, 256, 512), (1000, 128, 64), (8192, 256, 256), (130, 384, 192)])
@pytest.mark.parametrize("relu", [False, True])
def test_gemm_matches_fp32_reference(L, m, n, k, relu):
    import torch
    g = torch.Generator(device="cpu").manual_seed(m * 7 + n + k)
    a = (torch.randn(m, k, generator=g) * 0.5).to(torch.bfloat16).cuda()
    b = (torch.randn(n, k, generator=g) * 0.5).to(torch.bfloat16).cuda()
    bias = torch.randn(n, generator=g).float().cuda()
    c16 = torch.empty(m, n, dtype=torch.bfloat16, device="cuda")
    c32 = torch.empty(m, n, dtype=torch.float32, device="cuda")
    L.llama_gemm_error(True)
    L.llama_gemm_bf16(a, b, bias, c16, c32, L.GEMM_RELU if relu else 0)
    torch.cuda.synchronize()
    assert L.llama_gemm_error(True) == L.OK
    ref = a.float() @ b.float().T + bias
    if relu:
        ref = ref.clamp_min(0)
    # FP32 accumulation of BF16 products: only the summation order differs
    tol = 1e-4 * k ** 0.5 * (ref.abs().max().item() + 1)
    assert (c32 - ref).abs().max().item() <= tol
    # BF16 output: rounding of the FP32 result (relative 2^-8)
    assert torch.allclose(c16.float(), c32, rtol=2 ** -8, atol=1e-6)


def test_gemm_rejects_bad_shapes(L):
    import torch
    a = torch.zeros(128, 96, dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(128, 96, dtype=torch.bfloat16, device="cuda")
    c = torch.zeros(128, 128, dtype=torch.float32, device="cuda")
    with pytest.raises(L.LlamaError):  # k not a multiple of 64
        L.llama_gemm_bf16(a, b, None, None, c)
    with pytest.raises(L.LlamaError):  # no output
        L.llama_gemm_bf16(a[:, :64].contiguous(), b[:, :64].contiguous(), None, None, None)
