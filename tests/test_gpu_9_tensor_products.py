"""The split-BF16 product on the tensor cores (the operator products of the
Woodbury form, Sec. III-C) against exact rational sums: random, wide-range and
adversarial (every digit at its largest) operands, with ragged sizes that leave
partial 128 x 64 tiles and K stages."""
import ctypes
from fractions import Fraction

import numpy as np
import pytest

from paper_2110_01585_gb300 import _lib

from ._parity import cuda

pytestmark = pytest.mark.gpu


def _tc_product(A, B, slices=8):
    torch = cuda()
    lib = _lib.load()
    a = torch.as_tensor(np.ascontiguousarray(A), device="cuda")
    b = torch.as_tensor(np.ascontiguousarray(B), device="cuda")
    c = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float64, device="cuda")
    code = lib.ep_tv_tc_gemm_f64(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                 ctypes.c_void_p(c.data_ptr()), A.shape[0], B.shape[0], A.shape[1], slices,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, _lib.load().ep_tv_status_str(code)
    return c.cpu().numpy()


# (truncation, tail) coefficients of the bound below for each slice count: eight
# 7-bit digits leave 2^-57 of the row scale and an FP32 tail from s + t = 7; ten
# digits leave 2^-71 and a tail from s + t = 9 (7 + 7 bits smaller)
_BOUND = {8: (2.0 ** -55, 2.0 ** -52), 10: (2.0 ** -69, 2.0 ** -66)}


def _check(A, B, C, n_samples=40, seed=0, slices=8):
    """Every entry against numpy, and sampled entries against exact rational sums
    within the split form's bound.  With e_i the row scale (2^e_i <= 2 max_k |a_ik|)
    and eight round-to-nearest 7-bit digits, each operand entry is off by at most
    2^-57 2^e_i, i.e. 2^-56 of its row's largest entry; the dropped slice pairs
    (s + t >= 10) and the FP32 tail accumulator add at most about 2^-53 of
    2^(e_i + f_j) per value of k; the result is rounded once.  So
      |C_ij - sum_k a_ik b_jk| <= 2^-55 (amax_i sum|b_j| + bmax_j sum|a_i|)
                                  + 2^-52 k amax_i bmax_j + 2^-51 |sum_k a_ik b_jk|
    (with a factor of two to spare), relative to the rows' largest entries as for
    every split of this kind (with ten slices the two coefficients are 2^-69 and
    2^-66).  Returns the largest error / bound and the mean error / sum_k |a_ik b_jk|."""
    c_trunc, c_tail = _BOUND[slices]
    rng = np.random.default_rng(seed)
    m, n = C.shape
    k = A.shape[1]
    worst, rel = 0.0, []
    picks = [(0, 0), (m - 1, n - 1)] + [tuple(x) for x in zip(rng.integers(0, m, n_samples),
                                                              rng.integers(0, n, n_samples))]
    for i, j in picks:
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i], B[j]))
        amax, bmax = float(np.max(np.abs(A[i]))), float(np.max(np.abs(B[j])))
        bound = (c_trunc * (amax * float(np.sum(np.abs(B[j]))) + bmax * float(np.sum(np.abs(A[i]))))
                 + c_tail * k * amax * bmax + 2.0 ** -51 * abs(float(exact)))
        err = float(abs(Fraction(float(C[i, j])) - exact))
        worst = max(worst, err / bound if bound > 0 else err)
        absum = float(np.sum(np.abs(A[i] * B[j])))
        if absum > 0:
            rel.append(err / absum)
    assert worst <= 1.0, worst
    # all entries against numpy's FP64 product (its own error <= k 2^-53 sum|a b|)
    ref = A @ B.T
    aa, ab_ = np.abs(A), np.abs(B)
    amax, bmax = aa.max(axis=1), ab_.max(axis=1)
    bound = (c_trunc * (np.outer(amax, ab_.sum(axis=1)) + np.outer(aa.sum(axis=1), bmax))
             + c_tail * k * np.outer(amax, bmax) + 2.0 ** -51 * np.abs(ref)
             + k * 2.0 ** -53 * (aa @ ab_.T))
    assert np.all(np.abs(C - ref) <= bound)
    return worst, float(np.mean(rel)) if rel else 0.0


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (128, 64, 16), (200, 77, 300), (300, 130, 1000),
                                   (130, 257, 4101)])
def test_random_normal(m, n, k):
    rng = np.random.default_rng(m + n + k)
    A, B = rng.standard_normal((m, k)), rng.standard_normal((n, k))
    _, mean_rel = _check(A, B, _tc_product(A, B))
    # entries of one scale: as accurate as an FP64 product on average
    assert mean_rel <= 2.0 ** -50, mean_rel


def test_wide_range_rows_and_columns():
    """Entries spread over 2^-40 .. 2^40 within rows (the cavity variances of
    Sec. III-C span 1e-2 .. 1e8) and zero rows."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((150, 2000)) * np.exp2(rng.uniform(-40, 40, (150, 2000)))
    B = rng.standard_normal((90, 2000)) * np.exp2(rng.uniform(-20, 20, 2000))
    A[7] = 0.0
    C = _tc_product(A, B)
    assert np.all(C[7] == 0.0)
    _check(A, B, C)


def test_largest_digits_exact_over_long_k():
    """All entries just below the row scale: every leading digit is 128, so the
    exact partial sums reach 2^22 in every chunk of 256 values of k."""
    rng = np.random.default_rng(9)
    A = 1.0 - rng.random((130, 8192)) * 2.0 ** -10
    B = 1.0 - rng.random((70, 8192)) * 2.0 ** -10
    _check(A, B, _tc_product(A, B), n_samples=10)


def test_symmetric_product_lower_half_matches_full():
    """G G^T (the form of K = A C A^T): both halves of the product agree."""
    rng = np.random.default_rng(11)
    G = rng.standard_normal((260, 700)) * np.sqrt(np.exp(rng.uniform(-5, 18, 700)))
    C = _tc_product(G, G)
    # the exact slice sums agree bit for bit; the FP32 tail adds in another order
    amax = np.max(np.abs(G), axis=1)
    assert np.all(np.abs(C - C.T) <= 2.0 ** -50 * G.shape[1] * np.outer(amax, amax))
    _check(G, G, C, n_samples=20)


@pytest.mark.parametrize("m,n,k", [(130, 257, 4101), (300, 70, 8192)])
def test_ten_slices_random_and_wide_range(m, n, k):
    """The form of the Cholesky factorisation's products (ten slices, seven exact
    diagonals): random operands and rows spanning 2^+-30, within its bound."""
    rng = np.random.default_rng(m * n)
    A, B = rng.standard_normal((m, k)), rng.standard_normal((n, k))
    _, mean_rel = _check(A, B, _tc_product(A, B, 10), slices=10)
    assert mean_rel <= 2.0 ** -50, mean_rel
    A = A * np.exp2(rng.uniform(-30, 30, (m, k)))
    _check(A, B, _tc_product(A, B, 10), slices=10)


def test_ten_slices_largest_digits_and_cancellation():
    """Every leading digit at its largest over k = 8192 (the exact chunk sums at
    their bound), and the diagonal of L L^T within 5e-13 of its exact value, far
    below the 1e-9 a Schur complement K22 - L21 L21^T may cancel to."""
    rng = np.random.default_rng(21)
    A = 1.0 - rng.random((130, 8192)) * 2.0 ** -10
    B = 1.0 - rng.random((70, 8192)) * 2.0 ** -10
    _check(A, B, _tc_product(A, B, 10), n_samples=8, slices=10)
    L = rng.standard_normal((60, 1000))
    D = _tc_product(L, L, 10)
    for i in range(60):
        exact = sum(Fraction(float(v)) ** 2 for v in L[i])
        err = float(abs(Fraction(float(D[i, i])) - exact))
        assert err <= 2.0 ** -66 * 1000 * float(np.max(np.abs(L[i]))) ** 2 + 2.0 ** -51 * float(exact), (i, err)
        assert err <= 5e-13


def test_slice_count_is_checked():
    lib = _lib.load()
    cuda()
    for slices in (7, 9, 12):
        assert lib.ep_tv_tc_gemm_f64(ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 1, 1, 1, slices,
                                     None) == 1
    assert lib.ep_tv_tc_gemm_f64(ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 1, 1, 8193, 10,
                                 None) == 1

