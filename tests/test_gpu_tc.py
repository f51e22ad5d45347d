"""Tensor-core matrix update (cs_tc_gemm_update: tcgen05, operands split into two TF32
terms, three products accumulated in FP32) against the FP64 product.

Bar: normwise, |C - (C0 + alpha A B)| <= 4e-6 (|C0| + |alpha| |A| |B|) elementwise
maximum, about what FP32 inner products reach; a single TF32 product would be off by
~1e-3 and fail it.  Shapes cover one exact tile, ragged edges in every dimension, a
batch, and inner dimensions that are not multiples of the staged block."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_08465_gb300 import cs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("batch,M,N,K,alpha", [(1, 128, 64, 32, 1.0), (1, 300, 200, 70, -1.0),
                                               (3, 257, 65, 33, 0.5), (2, 1000, 700, 32, -1.0),
                                               (1, 5, 3, 1, 2.0)])
def test_tc_gemm_update_matches_fp64(batch, M, N, K, alpha):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = torch.Generator(device=DEV).manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(batch, M, K, device=DEV, generator=g)
    B = torch.randn(batch, K, N, device=DEV, generator=g)
    C = torch.randn(batch, M, N, device=DEV, generator=g)
    ref = C.double() + alpha * (A.double() @ B.double())
    scale = C.double().abs() + abs(alpha) * (A.double().abs() @ B.double().abs())
    ctx = cs.Context()
    cs.tc_gemm_update(A, B, C, alpha, ctx=ctx)
    ctx.sync()
    err = ((C.double() - ref).abs() / scale).max().item()
    assert err <= 4e-6, err
    ctx.close()


@pytest.mark.parametrize("n,batch", [(3, 1), (40, 2), (130, 1), (374, 2)])
def test_blocked_hessenberg_matches_the_fp64_reduction(n, batch):
    """cs_hessenberg_tc (panels of 32 columns, trailing updates on the tensor cores)
    against LAPACK's FP64 reduction of the same matrices: upper Hessenberg with exact
    zeros below the subdiagonal, the same entries up to FP32 rounding (both use
    reflectors with beta = -sign(alpha) |x|), and the similarity invariants (trace,
    Frobenius norm) kept.  Orders cover one partial panel, several panels and a ragged
    last one, and the 300-bus network's state order (374)."""
    scipy = pytest.importorskip("scipy.linalg")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(n)
    A = rng.standard_normal((batch, n, n)).astype(np.float32)
    T = torch.as_tensor(A, device=DEV)
    ctx = cs.Context()
    ctx.hessenberg_tc(T)
    ctx.sync()
    H = T.cpu().numpy().astype(np.float64)
    for b in range(batch):
        A64 = A[b].astype(np.float64)
        H64 = scipy.hessenberg(A64)
        assert np.all(np.tril(H[b], -2) == 0.0)
        fro = np.linalg.norm(A64)
        assert abs(np.linalg.norm(H[b]) - fro) <= 1e-5 * fro
        assert abs(np.trace(H[b]) - np.trace(A64)) <= 1e-5 * fro
        err = np.abs(np.abs(H[b]) - np.abs(H64)).max()
        assert err <= 5e-5 * fro, (b, err, fro)
    ctx.close()
