"""Each deconvolution parity case is well conditioned at the mean tolerance:
the FP64 oracle itself moves by less than half of it when the float32
observation is perturbed by 1e-7 relative (about one float32 rounding), so a
GPU result outside the tolerance points at the GPU path, not at the instance."""
import numpy as np
import pytest

from ._cases import (DECONV_CASES, MOG2_DECONV, mog2_deconv_problem, mog2_oracle_run, oracle_run,
                     probes, y32)
from ._parity import RTOL_MEAN, parity_errors


@pytest.mark.parametrize("name", sorted(DECONV_CASES))
def test_case_stable_under_float32_rounding(name):
    make, (S, seed), sweeps, em_every, order, _ = DECONV_CASES[name]
    p = make()
    y = y32(p)
    pr = probes(p, S, seed)
    mu0, var0 = oracle_run(p, y, pr, sweeps, em_every, order)
    rng = np.random.default_rng(0)
    mu, var = oracle_run(p, y * (1 + 1e-7 * rng.standard_normal(y.shape)), pr, sweeps, em_every,
                         order)
    e_mu, _ = parity_errors(mu, var, mu0, var0, p.y)
    assert e_mu < 0.5 * RTOL_MEAN, e_mu


def test_mog2_case_stable_under_float32_rounding():
    """The same admission rule for the MoG2-TV deconvolution case."""
    p = mog2_deconv_problem()
    y = y32(p)
    pr = probes(p, MOG2_DECONV["S"], MOG2_DECONV["probe_seed"])
    mu0, var0, capped = mog2_oracle_run(p, y, pr)
    assert capped > 1000  # the variance cap is exercised
    rng = np.random.default_rng(0)
    mu, var, _ = mog2_oracle_run(p, y * (1 + 1e-7 * rng.standard_normal(y.shape)), pr)
    e_mu, _ = parity_errors(mu, var, mu0, var0, p.y)
    assert e_mu < 0.5 * RTOL_MEAN, e_mu
