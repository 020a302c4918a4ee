"""Shared helpers for GPU-vs-oracle parity tests."""
import numpy as np

# Tolerances stated for this method: after the same fixed number of sweeps the
# FP32 GPU path must match the FP64 oracle to 1e-4 relative on posterior means
# (relative to max(|mu|, 1e-3 * range(y)), since a mean can be ~0) and 1e-3
# relative on posterior variances.
RTOL_MEAN = 1e-4
RTOL_VAR = 1e-3


def parity_errors(mu, var, mu_ref, var_ref, y):
    mu, var = np.asarray(mu, np.float64), np.asarray(var, np.float64)
    y = np.asarray(y, np.float64)
    scale = np.maximum(np.abs(mu_ref), 1e-3 * (y.max() - y.min()))
    e_mu = float(np.max(np.abs(mu - mu_ref) / scale))
    e_var = float(np.max(np.abs(var - var_ref) / var_ref))
    return e_mu, e_var


def assert_parity(mu, var, mu_ref, var_ref, y, rtol_mean=RTOL_MEAN, rtol_var=RTOL_VAR):
    e_mu, e_var = parity_errors(mu, var, mu_ref, var_ref, y)
    print(f"parity: mean {e_mu:.3e} (tol {rtol_mean:.0e}), variance {e_var:.3e} (tol {rtol_var:.0e})")
    assert e_mu <= rtol_mean and e_var <= rtol_var, (e_mu, e_var)
    return e_mu, e_var


def cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")
    return torch
