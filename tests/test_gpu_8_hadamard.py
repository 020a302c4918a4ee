"""Compressive sensing with subsampled 2-D Hadamard patterns (Sec. II-A (iii)):
the fast-transform Woodbury site on the GPU against the FP64 oracle, which
forms the M x N matrix from the definition of the Walsh functions and runs the
same Woodbury site as for the dense Gaussian matrix."""
import numpy as np
import pytest

from oracle import operators
from oracle.ep import EPOracle
from paper_2110_01585_gb300 import EPTV, OP_HADAMARD
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import assert_parity, cuda

pytestmark = pytest.mark.gpu


def _run(h, w, ratio, sweeps, em_every, seed, periodic=1, xi_plane=None):
    torch = cuda()
    p = syn.hadamard_cs_problem(h, w, ratio=ratio, sigma=0.01, beta0=2.0, seed=seed)
    y32 = p.y.astype(np.float32)
    A = operators.hadamard_matrix(h, w, p.patterns)
    kw = {}
    xi = p.xi
    if xi_plane is not None:
        xi = xi_plane.astype(np.float32).astype(np.float64)
        kw["xi_plane"] = torch.as_tensor(xi_plane.astype(np.float32), device="cuda")
    with EPTV(torch.as_tensor(y32, device="cuda"), p.xi, p.beta, op=OP_HADAMARD,
              patterns=p.patterns, height=h, width=w, periodic=periodic, **kw) as ep:
        ep.sweep(sweeps, em_every=em_every)
        mu, var = (t.cpu().numpy() for t in ep.posterior())
        beta_gpu, _ = ep.em_beta()
        assert ep.status() == 0
    o = EPOracle("cs", y32.astype(np.float64), xi, p.beta, h, w, A=A, site0="woodbury",
                 periodic=bool(periodic))
    o.run(sweeps, em_every=em_every)
    mu_r, var_r = o.posterior()
    return mu, var, mu_r, var_r, A.T @ p.y, beta_gpu, o


@pytest.mark.parametrize("h,w,sweeps,em", [(16, 16, 6, 3), (32, 32, 10, 5), (16, 64, 8, 4),
                                           (64, 64, 8, 4)])
def test_hadamard_cs_matches_oracle(h, w, sweeps, em):
    mu, var, mu_r, var_r, ref, _, _ = _run(h, w, 0.3, sweeps, em, seed=h + w)
    assert_parity(mu, var, mu_r, var_r, ref)


def test_hadamard_rows_longer_than_one_shared_memory_transform():
    """128 x 256 (N = 32768): the row transforms take their last stride in a
    global pass after the shared-memory chunks of 16384."""
    mu, var, mu_r, var_r, ref, _, _ = _run(128, 256, 0.03, 4, 2, seed=7)
    assert_parity(mu, var, mu_r, var_r, ref)


def test_hadamard_free_boundary_and_diagonal_noise():
    """The free boundary with one noise variance per measurement
    (K = diag(xi) + A C A^T)."""
    m = int(np.floor(0.3 * 32 * 32))
    xi = 1e-4 * np.exp(np.random.default_rng(3).uniform(0.0, 3.0, m))
    mu, var, mu_r, var_r, ref, _, _ = _run(32, 32, 0.3, 6, 3, seed=11, periodic=0, xi_plane=xi)
    assert_parity(mu, var, mu_r, var_r, ref)


def test_hadamard_cs_128_full_size():
    """The compressive-sensing size with Hadamard patterns: 128 x 128, M =
    floor(0.3 N) = 4915 uniformly drawn patterns, sigma 0.01, six sweeps with EM
    after the third and the sixth."""
    mu, var, mu_r, var_r, ref, beta_gpu, o = _run(128, 128, 0.3, 6, 3, seed=0)
    assert_parity(mu, var, mu_r, var_r, ref)
    beta_ref = o.em_update()
    assert abs(beta_gpu / beta_ref - 1.0) < 1e-4, (beta_gpu, beta_ref)
