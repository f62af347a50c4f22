"""The tcgen05 tensor-core GEMM (the dense coupling's building block) against torch."""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(128, 128, 64), (256, 384, 512), (128, 256, 1024)])
def test_tc_gemm_matches_matmul(shape):
    require_gpu()
    import torch
    from paper_2505_22631_gb300 import capi
    M, N, K = shape
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.zeros(M, N, device="cuda", dtype=torch.float32)
    capi.oim_debug_tc_gemm(A, B, D, M, N, K)
    ref = A.double() @ B.double().T
    err = (D.double() - ref).abs().max().item()
    assert err <= 1e-4 * K ** 0.5, err
