"""Compressive sensing (dense Gaussian sensing matrix): the FP64 Woodbury
likelihood site on the GPU against the FP64 oracle."""
import numpy as np
import pytest

from oracle.ep import EPOracle
from paper_2110_01585_gb300 import EPTV, OP_DENSE
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import assert_parity, cuda

pytestmark = pytest.mark.gpu


def _run(side, m, sweeps, em_every, seed):
    torch = cuda()
    p = syn.cs_problem(side, side, m=m, seed=seed, beta0=2.0)
    # both sides see the same float32 data
    A32 = p.A.astype(np.float32)
    y32 = p.y.astype(np.float32)
    At = torch.as_tensor(A32, device="cuda")
    yt = torch.as_tensor(y32, device="cuda")
    with EPTV(yt, p.xi, p.beta, op=OP_DENSE, dense=At, height=side, width=side) as ep:
        ep.sweep(sweeps, em_every=em_every)
        mu, var = (t.cpu().numpy() for t in ep.posterior())
        assert ep.status() == 0
    o = EPOracle("cs", y32.astype(np.float64), p.xi, p.beta, side, side,
                 A=A32.astype(np.float64), site0="woodbury")
    o.run(sweeps, em_every=em_every)
    mu_r, var_r = o.posterior()
    return mu, var, mu_r, var_r, p


@pytest.mark.parametrize("side,m,sweeps,em", [(16, 77, 6, 3), (32, 307, 10, 5), (64, 1228, 8, 4)])
def test_cs_matches_oracle(side, m, sweeps, em):
    mu, var, mu_r, var_r, p = _run(side, m, sweeps, em, seed=side)
    # y is not an image here; scale the mean tolerance by the range of the back-projection
    ref = p.A.T @ p.y
    assert_parity(mu, var, mu_r, var_r, ref)
