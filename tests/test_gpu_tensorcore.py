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


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    """Failure detection by a bounded device wait: the producer withholds one K block,
    so the MMA thread's wait for it runs out after a short poll limit.  The call
    reports OIM_ETIMEOUT (no fault, no hang), and the same process then runs the
    self-test normally, with a result equal to the matrix product."""
    require_gpu()
    import torch
    from paper_2505_22631_gb300 import capi
    M, N, K = 256, 128, 512
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    for withhold in (1, 5):   # a block of the first loads, and one of the refills
        D = torch.zeros(M, N, device="cuda", dtype=torch.float32)
        with pytest.raises(capi.OimError) as ei:
            capi.oim_debug_tc_gemm_withhold(A, B, D, M, N, K, withhold, 1 << 16)
        assert ei.value.code == capi.OIM_ETIMEOUT
    # nothing withheld, the same short limit: the pipeline completes
    D = torch.zeros(M, N, device="cuda", dtype=torch.float32)
    capi.oim_debug_tc_gemm_withhold(A, B, D, M, N, K, -1, 1 << 20)
    assert (D.double() - ref).abs().max().item() <= 1e-4 * K ** 0.5
    D = torch.zeros(M, N, device="cuda", dtype=torch.float32)
    capi.oim_debug_tc_gemm(A, B, D, M, N, K)
    torch.cuda.synchronize()
    assert (D.double() - ref).abs().max().item() <= 1e-4 * K ** 0.5
