"""Compressive sensing (dense Gaussian sensing matrix): the FP64 Woodbury
likelihood site on the GPU against the FP64 oracle."""
import numpy as np
import pytest

from oracle.ep import EPOracle
from paper_2110_01585_gb300 import EPTV, OP_DENSE
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import assert_parity, cuda

pytestmark = pytest.mark.gpu


def _run(side, m, sweeps, em_every, seed, width=None, periodic=1, order="prior_first"):
    torch = cuda()
    h, w = side, (width or side)
    p = syn.cs_problem(h, w, m=m, seed=seed, beta0=2.0)
    # both sides see the same float32 data
    A32 = p.A.astype(np.float32)
    y32 = p.y.astype(np.float32)
    At = torch.as_tensor(A32, device="cuda")
    yt = torch.as_tensor(y32, device="cuda")
    with EPTV(yt, p.xi, p.beta, op=OP_DENSE, dense=At, height=h, width=w, periodic=periodic,
              order_mode=1 if order == "q0_first" else 0) as ep:
        ep.sweep(sweeps, em_every=em_every)
        mu, var = (t.cpu().numpy() for t in ep.posterior())
        assert ep.status() == 0
    o = EPOracle("cs", y32.astype(np.float64), p.xi, p.beta, h, w,
                 A=A32.astype(np.float64), site0="woodbury", periodic=bool(periodic), order=order)
    o.run(sweeps, em_every=em_every)
    mu_r, var_r = o.posterior()
    return mu, var, mu_r, var_r, p


@pytest.mark.parametrize("side,m,sweeps,em", [(16, 77, 6, 3), (32, 307, 10, 5), (64, 1228, 8, 4)])
def test_cs_matches_oracle(side, m, sweeps, em):
    mu, var, mu_r, var_r, p = _run(side, m, sweeps, em, seed=side)
    # y is not an image here; scale the mean tolerance by the range of the back-projection
    ref = p.A.T @ p.y
    assert_parity(mu, var, mu_r, var_r, ref)


def test_cs_free_boundary_odd_size_q0_first():
    """A 21 x 34 image with the free boundary (odd height), Algorithm 1's listed
    order (likelihood site first) and EM."""
    mu, var, mu_r, var_r, p = _run(21, 214, 6, 3, seed=5, width=34, periodic=0, order="q0_first")
    assert_parity(mu, var, mu_r, var_r, p.A.T @ p.y)


def test_cs_config_128_full_size():
    """The compressive-sensing configuration at its stated size: 128 x 128 image
    (N = 16384), M = floor(0.3 N) = 4915 Gaussian rows of variance 1/M, noise
    sigma 0.01, beta0 = 1 (Sec. V-C), six sweeps with EM after the third and
    sixth.  The oracle forms the Woodbury site in FP64 with one 4915 x 4915
    Cholesky factorisation per sweep (Sec. III-C)."""
    torch = cuda()
    h = w = 128
    p = syn.cs_problem(h, w, ratio=0.3, sigma=0.01, beta0=1.0, seed=0)
    assert p.A.shape == (4915, 16384)
    A32 = p.A.astype(np.float32)
    y32 = p.y.astype(np.float32)
    At = torch.as_tensor(A32, device="cuda")
    yt = torch.as_tensor(y32, device="cuda")
    with EPTV(yt, p.xi, p.beta, op=OP_DENSE, dense=At, height=h, width=w) as ep:
        ep.sweep(6, em_every=3)
        mu, var = (t.cpu().numpy() for t in ep.posterior())
        beta_gpu, _ = ep.em_beta()
        assert ep.status() == 0
    del At
    o = EPOracle("cs", y32.astype(np.float64), p.xi, p.beta, h, w, A=A32.astype(np.float64),
                 site0="woodbury")
    o.run(6, em_every=3)
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, p.A.T @ p.y)
    # beta of the last EM step (N / a_u of the sixth sweep, recomputed on both sides)
    beta_ref = o.em_update()
    assert abs(beta_gpu / beta_ref - 1.0) < 1e-4, (beta_gpu, beta_ref)


def test_cs_diagonal_noise_matches_oracle():
    """Compressive sensing with one noise variance per measurement: the Woodbury
    site with K = diag(xi) + A C A^T (Sec. III-C)."""
    torch = cuda()
    h = w = 32
    p = syn.cs_problem(h, w, m=307, seed=32, beta0=2.0)
    m = p.A.shape[0]
    xi = 1e-4 * np.exp(np.random.default_rng(33).uniform(0.0, 3.0, m))
    y = p.A @ p.x.reshape(-1) + np.sqrt(xi) * np.random.default_rng(34).standard_normal(m)
    A32, y32, xi32 = p.A.astype(np.float32), y.astype(np.float32), xi.astype(np.float32)
    At = torch.as_tensor(A32, device="cuda")
    with EPTV(torch.as_tensor(y32, device="cuda"), 0.0, p.beta, op=OP_DENSE, dense=At, height=h,
              width=w, xi_plane=torch.as_tensor(xi32, device="cuda")) as ep:
        ep.sweep(8, em_every=4)
        mu, var = (t.cpu().numpy() for t in ep.posterior())
        assert ep.status() == 0
    o = EPOracle("cs", y32.astype(np.float64), xi32.astype(np.float64), p.beta, h, w,
                 A=A32.astype(np.float64), site0="woodbury")
    o.run(8, em_every=4)
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, p.A.T @ y)
