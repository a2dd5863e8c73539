"""FP64-class products on the BF16 tensor cores (hodlr_dgemm_slices, the product of the
HODLR_MIXED_BF16 path) against FP64 products of the same operands.

  * exactness: integer operands whose products and sums are exact in FP64 give bit-exact results,
    with K inside one 512-long chunk (exact FP32 accumulation of the digit groups in tensor
    memory) and across chunks (split K, FP64 reduction of exact partials);
  * accuracy: random operands with rows and columns scaled over six decades, every layout
    (transposes, batches with strides, a shared A, paired B operands, alpha and beta), ragged
    sizes; the error is checked against the slicing bound K 2^-44 max|A_i.| max|B_.j| and
    normwise against 5e-13 (seven 7-bit digits; measured about 2e-13 on these operands);
  * zero rows and columns give exact zeros.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def slices(A, B, M, N, K, batch=1, lda=None, sA=None, tA=0, ldb=None, sB=None, tB=0, bmap=0, alpha=1.0, beta=0.0,
           C=None, ldc=None, sC=None, work_mb=256):
    from paper_2303_10102_gb300 import lib as plib
    lib = plib.load()
    work = torch.empty(work_mb << 20, dtype=torch.uint8, device=DEV)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hodlr_dgemm_slices(M, N, K, batch, ctypes.c_void_p(A.data_ptr()), lda, sA, tA,
                                ctypes.c_void_p(B.data_ptr()), ldb, sB, tB, bmap, alpha, beta,
                                ctypes.c_void_p(C.data_ptr()), ldc, sC, ctypes.c_void_p(work.data_ptr()),
                                work.numel(), st)
    torch.cuda.synchronize()
    return rc


def colmajor(x):
    """device buffer holding the column-major storage of a 2-D array"""
    return torch.as_tensor(np.asfortranarray(x).ravel(order="F"), device=DEV)


@pytest.mark.parametrize("K", [37, 512, 1000, 2048])
def test_integer_operands_are_exact(K):
    rng = np.random.default_rng(K)
    M, N = 150, 130
    A = rng.integers(-1000, 1001, size=(M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(K, N)).astype(np.float64)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    C = torch.zeros(M * N, dtype=torch.float64, device=DEV)
    assert slices(colmajor(A), colmajor(B), M, N, K, 1, M, 0, 0, K, 0, 0, 0, 1.0, 0.0, C, M, 0) == 0
    got = C.cpu().numpy().reshape(N, M).T
    assert np.array_equal(got, ref)


def _bound(A, B):
    K = A.shape[1]
    return K * 2.0 ** -44 * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]


def _scaled(rng, m, n):
    return (rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-3, 3, size=(m, 1))
            * 10.0 ** rng.uniform(-3, 3, size=(1, n)))


@pytest.mark.parametrize("tA,tB,inner", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1)])
def test_random_scaled_operands_all_layouts(tA, tB, inner):
    """Rows of A and columns of B scaled over six decades each (inner = 0); with inner = 1 the
    columns of A and the rows of B are scaled as well, independently, so that max|A_i.| max|B_.j|
    can exceed |C_ij| by orders of magnitude and only the slicing bound applies."""
    rng = np.random.default_rng(10 + 2 * tA + tB + 4 * inner)
    M, N, K = 200, 300, 777
    if inner:
        A = _scaled(rng, M, K)
        B = _scaled(rng, K, N)
    else:
        A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-3, 3, size=(M, 1))
        B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-3, 3, size=(1, N))
    C0 = rng.standard_normal((M, N))
    Ast = colmajor(A.T if tA else A)
    Bst = colmajor(B.T if tB else B)
    C = colmajor(C0)
    alpha, beta = -1.5, 0.5
    rc = slices(Ast, Bst, M, N, K, 1, K if tA else M, 0, tA, N if tB else K, 0, tB, 0, alpha, beta, C, M, 0)
    assert rc == 0
    got = C.cpu().numpy().reshape(N, M).T
    ref = alpha * (A @ B) + beta * C0
    err = np.abs(got - ref)
    assert np.all(err <= 1.5 * _bound(A, B) + 1e-15 * np.abs(ref)), err.max()
    if not inner:
        # seven digits: the representation and the dropped digit groups give about 4e-14 here; the
        # tensor cores' FP32 accumulation of the shared tail groups (t = 4..6) about 2e-13
        assert np.linalg.norm(got - ref) <= 5e-13 * np.linalg.norm(ref)


def test_batched_strided_shared_and_paired_operands():
    rng = np.random.default_rng(3)
    M, N, K, nb = 130, 70, 600, 4
    As = [_scaled(rng, M, K) for _ in range(nb)]
    Bs = [_scaled(rng, K, N) for _ in range(nb)]
    # products b use B_(b^1): stored as K x N blocks
    A = torch.cat([colmajor(a) for a in As])
    B = torch.cat([colmajor(b) for b in Bs])
    C = torch.zeros(nb * M * N, dtype=torch.float64, device=DEV)
    assert slices(A, B, M, N, K, nb, M, M * K, 0, K, K * N, 0, 1, 1.0, 0.0, C, M, M * N) == 0
    got = C.cpu().numpy().reshape(nb, N, M).transpose(0, 2, 1)
    for b in range(nb):
        ref = As[b] @ Bs[b ^ 1]
        assert np.all(np.abs(got[b] - ref) <= 1.5 * _bound(As[b], Bs[b ^ 1])), b
    # one A shared by the batch (sA = 0), B_(b>>1)
    C2 = torch.zeros(nb * M * N, dtype=torch.float64, device=DEV)
    assert slices(A, B, M, N, K, nb, M, 0, 0, K, K * N, 0, 2, 1.0, 0.0, C2, M, M * N) == 0
    got = C2.cpu().numpy().reshape(nb, N, M).transpose(0, 2, 1)
    for b in range(nb):
        ref = As[0] @ Bs[b >> 1]
        assert np.all(np.abs(got[b] - ref) <= 1.5 * _bound(As[0], Bs[b >> 1])), b


def test_zero_rows_columns_and_chunked_workspace():
    rng = np.random.default_rng(4)
    M, N, K = 257, 1000, 300
    A = _scaled(rng, M, K)
    B = _scaled(rng, K, N)
    A[5] = 0.0
    B[:, 17] = 0.0
    C = torch.full((M * N,), float("nan"), dtype=torch.float64, device=DEV)
    # a workspace this small forces column chunks of the B planes
    rc = slices(colmajor(A), colmajor(B), M, N, K, 1, M, 0, 0, K, 0, 0, 0, 1.0, 0.0, C, M, 0, work_mb=64)
    assert rc == 0
    got = C.cpu().numpy().reshape(N, M).T
    ref = A @ B
    assert np.all(got[5] == 0.0) and np.all(got[:, 17] == 0.0)
    assert np.all(np.abs(got - ref) <= 1.5 * _bound(A, B))


def test_long_k_split_into_ranges_and_short_k_tiles():
    """K = 40000 with a 64 MiB workspace: the operands' planes do not fit at once, so K is cut into
    ranges whose partial products are summed in FP64; K = 100 takes the 32-column short-K tiles
    (two CTAs per SM) with a ragged N."""
    rng = np.random.default_rng(5)
    for M, N, K in [(130, 130, 40000), (300, 203, 100)]:
        A = rng.standard_normal((M, K))
        B = rng.standard_normal((K, N))
        C = torch.zeros(M * N, dtype=torch.float64, device=DEV)
        Ast = colmajor(A.T)      # A given transposed (K contiguous), as the Gram products are
        rc = slices(Ast, colmajor(B), M, N, K, 1, K, 0, 1, K, 0, 0, 0, 1.0, 0.0, C, M, 0, work_mb=64)
        assert rc == 0
        got = C.cpu().numpy().reshape(N, M).T
        ref = A @ B
        assert np.all(np.abs(got - ref) <= 1.5 * _bound(A, B)), (M, N, K)
        assert np.linalg.norm(got - ref) <= 5e-13 * np.linalg.norm(ref), (M, N, K)


# ---------------------------------------------------------------- fused products
# Short-K A B with column-major A (K <= 64, M x batch >= 4096) and long-K A^T B with M <= 128
# (K >= 1024) make their digit planes in shared memory (oz_ab_kernel / oz_atb_kernel) instead of
# reading sliced planes; the long-K product scales each 512-long chunk of K by its own exponents.

@pytest.mark.parametrize("M,N,K", [(5000, 130, 37), (4096 + 17, 136, 64), (300, 50, 8)])
def test_fused_short_k_integer_operands_are_exact(M, N, K):
    rng = np.random.default_rng(M + K)
    nb = 1 if M * 1 >= 4096 else 16   # 300 x 16 rows: the batch reaches the fused path
    As = [rng.integers(-1000, 1001, size=(M, K)).astype(np.float64) for _ in range(nb)]
    Bs = [rng.integers(-1000, 1001, size=(K, N)).astype(np.float64) for _ in range(nb)]
    A = torch.cat([colmajor(a) for a in As])
    B = torch.cat([colmajor(b) for b in Bs])
    C = torch.zeros(nb * M * N, dtype=torch.float64, device=DEV)
    assert slices(A, B, M, N, K, nb, M, M * K, 0, K, K * N, 0, 0, 1.0, 0.0, C, M, M * N) == 0
    got = C.cpu().numpy().reshape(nb, N, M).transpose(0, 2, 1)
    for b in range(nb):
        ref = (As[b].astype(np.int64) @ Bs[b].astype(np.int64)).astype(np.float64)
        assert np.array_equal(got[b], ref), b


def test_fused_short_k_scaled_operands_layouts_and_batches():
    rng = np.random.default_rng(21)
    # one product: rows of A and columns of B over six decades, B given transposed, alpha / beta
    M, N, K = 3 * 4096 + 5, 136, 61
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-3, 3, size=(M, 1))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-3, 3, size=(1, N))
    C0 = rng.standard_normal((M, N))
    C = colmajor(C0)
    assert slices(colmajor(A), colmajor(B.T), M, N, K, 1, M, 0, 0, N, 0, 1, 0, -1.5, 0.5, C, M, 0) == 0
    got = C.cpu().numpy().reshape(N, M).T
    ref = -1.5 * (A @ B) + 0.5 * C0
    assert np.all(np.abs(got - ref) <= 1.5 * 1.5 * _bound(A, B) + 1e-15 * np.abs(ref))
    assert np.linalg.norm(got - ref) <= 5e-13 * np.linalg.norm(ref)
    # batches: paired B operands (b^1) and one shared A, with ragged M and a C leading dimension
    # larger than M
    M, N, K, nb, ldc = 1030, 70, 33, 6, 1040
    As = [_scaled(rng, M, K) for _ in range(nb)]
    Bs = [_scaled(rng, K, N) for _ in range(nb)]
    A = torch.cat([colmajor(a) for a in As])
    B = torch.cat([colmajor(b) for b in Bs])
    for bmap, sA, pick in [(1, M * K, lambda b: (As[b], Bs[b ^ 1])), (2, 0, lambda b: (As[0], Bs[b >> 1]))]:
        C = torch.zeros(nb * ldc * N, dtype=torch.float64, device=DEV)
        assert slices(A, B, M, N, K, nb, M, sA, 0, K, K * N, 0, bmap, 1.0, 0.0, C, ldc, ldc * N) == 0
        got = C.cpu().numpy().reshape(nb, N, ldc).transpose(0, 2, 1)
        for b in range(nb):
            a, bb = pick(b)
            assert np.all(np.abs(got[b, :M] - a @ bb) <= 1.5 * _bound(a, bb)), (bmap, b)
            assert np.all(got[b, M:] == 0.0)


@pytest.mark.parametrize("M,N,K", [(64, 136, 40000), (100, 130, 5000), (1, 7, 1024)])
def test_fused_long_k_integer_operands_are_exact(M, N, K):
    """Integer operands whose products and partial sums are exact in FP64: each 512-long chunk
    with its own exponents, the chunks of a CTA summed in FP64, the CTAs' partials reduced."""
    rng = np.random.default_rng(M * 7 + N)
    A = rng.integers(-1000, 1001, size=(M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(K, N)).astype(np.float64)
    A[:, 1000:1700] *= 1024.0      # chunks of very different magnitude
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    C = torch.zeros(M * N, dtype=torch.float64, device=DEV)
    assert slices(colmajor(A.T), colmajor(B), M, N, K, 1, K, 0, 1, K, 0, 0, 0, 1.0, 0.0, C, M, 0) == 0
    got = C.cpu().numpy().reshape(N, M).T
    assert np.array_equal(got, ref)


def test_fused_long_k_scaled_operands_ragged_and_batched():
    rng = np.random.default_rng(22)
    for M, N, K in [(64, 136, 33333), (128, 48, 2049), (37, 200, 100001)]:
        A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-3, 3, size=(M, 1))
        B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-3, 3, size=(1, N))
        C0 = rng.standard_normal((M, N))
        C = colmajor(C0)
        assert slices(colmajor(A.T), colmajor(B), M, N, K, 1, K, 0, 1, K, 0, 0, 0, 2.0, -1.0, C, M, 0) == 0
        got = C.cpu().numpy().reshape(N, M).T
        ref = 2.0 * (A @ B) - C0
        assert np.all(np.abs(got - ref) <= 2 * 1.5 * _bound(A, B) + 1e-15 * np.abs(ref)), (M, N, K)
        assert np.linalg.norm(got - ref) <= 5e-13 * np.linalg.norm(ref), (M, N, K)
    # batch of 5 with one shared B and with B_(b>>1)
    M, N, K, nb = 45, 136, 4096, 5
    As = [_scaled(rng, M, K) for _ in range(nb)]
    Bs = [_scaled(rng, K, N) for _ in range(nb)]
    A = torch.cat([colmajor(a.T) for a in As])
    B = torch.cat([colmajor(b) for b in Bs])
    for bmap, sB, pick in [(0, 0, lambda b: Bs[0]), (2, K * N, lambda b: Bs[b >> 1])]:
        C = torch.zeros(nb * M * N, dtype=torch.float64, device=DEV)
        assert slices(A, B, M, N, K, nb, K, M * K, 1, K, sB, 0, bmap, 1.0, 0.0, C, M, M * N) == 0
        got = C.cpu().numpy().reshape(nb, N, M).transpose(0, 2, 1)
        for b in range(nb):
            assert np.all(np.abs(got[b] - As[b] @ pick(b)) <= 1.5 * _bound(As[b], pick(b))), (bmap, b)


@pytest.mark.parametrize("plan", [(0, 0, 1), (0, 1, 1), (0, 2, 1), (1, 0, 1), (1, 1, 1), (1, 0, 4)])
def test_every_kernel_plan_is_exact_and_accurate(plan):
    """Each plan the autotuner can choose (slice planes with 128 x 96, two-CTA 128 x 48 or persistent
    warp-specialised 128 x 48 tiles, fused with
    either tile and more chunks per CTA), forced for this thread, on a long-K A^T B, a short-K A B
    and a general A B: integer operands bit-exact, scaled operands within the slicing bound."""
    from paper_2303_10102_gb300 import lib as plib
    lib = plib.load()
    assert lib.hodlr_dgemm_slices_plan(*plan) == 0
    try:
        rng = np.random.default_rng(sum(plan))
        for M, N, K, tA in [(100, 150, 3000, 1), (5000, 70, 40, 0), (300, 200, 700, 0)]:
            for integer in (True, False):
                if integer:
                    A = rng.integers(-1000, 1001, size=(M, K)).astype(np.float64)
                    B = rng.integers(-1000, 1001, size=(K, N)).astype(np.float64)
                else:
                    A = _scaled(rng, M, K)
                    B = _scaled(rng, K, N)
                Ast = colmajor(A.T if tA else A)
                C = torch.zeros(M * N, dtype=torch.float64, device=DEV)
                assert slices(Ast, colmajor(B), M, N, K, 1, K if tA else M, 0, tA, K, 0, 0, 0, 1.0, 0.0, C, M, 0) == 0
                got = C.cpu().numpy().reshape(N, M).T
                if integer:
                    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
                    assert np.array_equal(got, ref), (plan, M, N, K)
                else:
                    assert np.all(np.abs(got - A @ B) <= 1.5 * _bound(A, B)), (plan, M, N, K)
    finally:
        lib.hodlr_dgemm_slices_plan(-1, 0, 1)
