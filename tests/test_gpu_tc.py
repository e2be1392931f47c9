"""The tensor-core building block alone: D = A B^T through tcgen05 (TMEM accumulator,
K-major shared-memory operands) against a float64 product of the same operands.

* 3xTF32: within a few FP32 ulps of the exact product of the FP32 inputs.
* TF32 once: within TF32 rounding (2^-11 relative per operand).
* BF16: exact products of the BF16 inputs summed in FP32.
Shapes cover one and several 128-row tiles, N from 16 to 128 and K from one MMA
step to the largest accepted; invalid shapes are refused on the host.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ab(M, N, K, seed, dtype=torch.float32):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn((M, K), generator=g, dtype=torch.float64)
    B = torch.randn((N, K), generator=g, dtype=torch.float64)
    return A.to(dtype).cuda(), B.to(dtype).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 16, 8), (128, 64, 56), (256, 64, 56), (384, 128, 64),
                                   (128, 48, 24)])
def test_tf32x3_matches_fp32_product(M, N, K):
    from paper_1203_2394_gb300 import dpf
    A, B = _ab(M, N, K, M + N + K)
    D = dpf.tc_matmul(A, B, dpf.DPF_TC_TF32X3).double().cpu()
    ref = A.double().cpu() @ B.double().cpu().T
    scale = A.double().abs().cpu() @ B.double().abs().cpu().T
    err = (D - ref).abs() / scale
    assert float(err.max()) < 2e-6, float(err.max())


@pytest.mark.parametrize("M,N,K", [(128, 64, 56), (256, 32, 16)])
def test_tf32_once_within_tf32_rounding(M, N, K):
    from paper_1203_2394_gb300 import dpf
    A, B = _ab(M, N, K, 7 * M + K)
    D = dpf.tc_matmul(A, B, dpf.DPF_TC_TF32).double().cpu()
    ref = A.double().cpu() @ B.double().cpu().T
    scale = A.double().abs().cpu() @ B.double().abs().cpu().T
    err = (D - ref).abs() / scale
    assert float(err.max()) < 2.0 ** -10
    # and visibly coarser than 3xTF32 (the split is doing its job)
    D3 = dpf.tc_matmul(A, B, dpf.DPF_TC_TF32X3).double().cpu()
    assert float(((D3 - ref).abs() / scale).max()) < float(err.max()) / 16


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (256, 128, 128), (128, 80, 48)])
def test_bf16_products_summed_in_fp32(M, N, K):
    from paper_1203_2394_gb300 import dpf
    A, B = _ab(M, N, K, 3 * M + N, torch.bfloat16)
    D = dpf.tc_matmul(A, B, dpf.DPF_TC_BF16).double().cpu()
    ref = A.double().cpu() @ B.double().cpu().T  # BF16 products are exact in FP32
    scale = A.double().abs().cpu() @ B.double().abs().cpu().T
    err = (D - ref).abs() / scale
    assert float(err.max()) < 1e-6, float(err.max())


def test_rows_and_columns_not_transposed():
    # A = e_i rows, B = distinct rows: D must pick B's rows in order
    from paper_1203_2394_gb300 import dpf
    M, N, K = 128, 32, 32
    A = torch.zeros((M, K), dtype=torch.float32)
    for r in range(M):
        A[r, r % K] = 1.0
    B = torch.arange(N * K, dtype=torch.float32).reshape(N, K) / 64.0
    D = dpf.tc_matmul(A.cuda(), B.cuda(), dpf.DPF_TC_TF32X3).cpu()
    np.testing.assert_array_equal(D.numpy(), (A @ B.T).numpy())


@pytest.mark.parametrize("M,N,K,mode", [(100, 16, 8, 1), (128, 8, 8, 1), (128, 144, 8, 1),
                                        (128, 16, 12, 1), (128, 16, 72, 0), (128, 16, 8, 2),
                                        (128, 16, 16, 5)])
def test_bad_shapes_refused(M, N, K, mode):
    from paper_1203_2394_gb300 import dpf
    A = torch.zeros((max(M, 1), K), dtype=torch.float32, device="cuda")
    B = torch.zeros((max(N, 1), K), dtype=torch.float32, device="cuda")
    with pytest.raises(dpf.DpfError):
        dpf.tc_matmul(A, B, mode)
