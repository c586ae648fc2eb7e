"""Tensor-core dense kernels (tcgen05 kind::tf32) through the C ABI: the GEMM
against an FP64 product, the blocked Cholesky against the matrix it factors.

TF32 keeps 10 mantissa bits of each FP32 operand, so one product carries a
relative error of at most about 2 * 2^-10; a K-term sum is bounded by
3e-3 * sum_k |a_k| |b_k| elementwise (FP32 accumulation adds far less)."""
import numpy as np
import pytest

from paper_2510_13310_b300 import ba

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.mark.parametrize("M,N,K", [(128, 256, 32), (300, 500, 200), (1024, 1024, 1024), (129, 7, 100),
                                   (2048, 384, 4096)])
@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_tc_gemm_matches_fp64_within_tf32_bound(M, N, K, beta):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float32)
    B = torch.randn(N, K, generator=g, dtype=torch.float32)
    C0 = torch.randn(M, N, generator=g, dtype=torch.float32)
    dev = torch.device("cuda")
    Cd = C0.to(dev).clone()
    ba.tc_gemm_nt(A.to(dev), B.to(dev), Cd, alpha=-0.5, beta=beta)
    ref = -0.5 * (A.double() @ B.double().T) + beta * C0.double()
    bound = 3e-3 * 0.5 * (A.double().abs() @ B.double().abs().T) + 1e-6 * (1 + ref.abs())
    err = (Cd.cpu().double() - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())
    # an honest TF32 product is not exact: the tensor cores did the work
    if K >= 32:
        assert float(err.max()) > 0.0


def spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, 1.0 / cond, n)
    A = (Q * ev) @ Q.T
    d = np.sqrt(np.diag(A))
    return A / d[:, None] / d[None, :]  # Jacobi-scaled like S^


@pytest.mark.parametrize("n", [100, 128, 300, 1000, 1791, 2100, 4000])
def test_dense_cholesky_reconstructs(n):
    """Orders from one tile to 32 tiles (four panels of eight: the look-ahead's split
    trailing updates, the rest on the low-priority stream, run for three of them)."""
    A = spd(n, 1e3, seed=n)
    L, flags = ba.dense_cholesky(A.astype(np.float32))
    assert flags == 0
    assert np.all(np.triu(L, 1) == 0)
    assert np.all(np.diag(L) > 0)
    rec = L.astype(np.float64) @ L.astype(np.float64).T
    # backward error of a TF32 factorisation: ~ a few 1e-3 of |A| (|L||L^T| = O(1) after Jacobi scaling)
    assert np.abs(rec - A).max() <= 1e-2, np.abs(rec - A).max()
    Lref = np.linalg.cholesky(A)
    assert np.abs(L - Lref).max() <= 5e-2 * np.abs(Lref).max()


def test_dense_cholesky_reports_indefinite():
    A = spd(256, 10.0, seed=3)
    A[200, 200] = -1.0
    _, flags = ba.dense_cholesky(A.astype(np.float32))
    assert flags & 32
