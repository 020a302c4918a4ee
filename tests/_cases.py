"""Deconvolution parity cases shared by the GPU parity tests and the CPU test
that checks each case is well conditioned at the parity tolerance.

A parity case is only meaningful if the FP64 oracle itself is stable under
perturbations at FP32 rounding level: the GPU works from the float32 copy of y
and rounds at every step.  Near-zero posterior means of a deconvolution can
move by more than the mean tolerance when y is perturbed by 1e-7 relative, and
such an instance cannot separate a correct FP32 path from a wrong one; the CPU
test rejects it.  Both sides are given the same float32-rounded observation.
"""
import numpy as np

from paper_2110_01585_gb300 import synthetic as syn


def _nonsep_kernel():
    rng = np.random.default_rng(4)
    k = rng.random((5, 3)) ** 2
    return k / k.sum()


# name: (problem, RBMC probes (S, seed), sweeps, EM every, order, GPU options)
DECONV_CASES = {
    "uniform9_32_em": (lambda: syn.deconv_problem(32, 32, kernel=syn.uniform_kernel(9), bsnr_db=40.0,
                                                  beta0=1.0, seed=3, grf_length=8.0),
                       (8, 1), 10, 5, "prior_first", {}),
    "uniform5_48x80_em": (lambda: syn.deconv_problem(48, 80, kernel=syn.uniform_kernel(5), bsnr_db=30.0,
                                                     beta0=3.0, seed=2, grf_length=8.0),
                          (4, 3), 6, 3, "prior_first", {"cg_max_iter": 20000}),
    "nonseparable_40x36": (lambda: syn.deconv_problem(40, 36, kernel=_nonsep_kernel(), bsnr_db=35.0,
                                                      beta0=5.0, seed=5, grf_length=6.0),
                           (6, 6), 5, 0, "prior_first", {"cg_max_iter": 20000}),
    "gaussian15_48": (lambda: syn.deconv_problem(48, 48, kernel=syn.gaussian_kernel(15, 2.0), bsnr_db=30.0,
                                                 beta0=2.0, seed=7, grf_length=8.0),
                      (4, 8), 4, 0, "prior_first", {"cg_max_iter": 20000}),
    "uniform3_32_q0_first": (lambda: syn.deconv_problem(32, 32, kernel=syn.uniform_kernel(3), bsnr_db=30.0,
                                                        beta0=4.0, seed=9, grf_length=8.0),
                             (4, 10), 5, 0, "q0_first", {"order_mode": 1}),
}


# The MoG2-TV deconvolution case (Sec. II-B): 32 x 32, 5 x 5 uniform blur,
# BSNR 30 dB, theta = (omega, s1^2, s2^2), 4 probes, 5 sweeps; thousands of its
# site updates hit the variance cap.  (The same blur on seed 23 is not admitted:
# there the oracle moves by up to 1.2e-4 under float32 rounding of y.)
MOG2_DECONV = dict(seed=5, theta=(0.3, 0.1, 1e-3), S=4, probe_seed=24, sweeps=5)


def mog2_deconv_problem():
    c = MOG2_DECONV
    return syn.deconv_problem(32, 32, kernel=syn.uniform_kernel(5), bsnr_db=30.0, beta0=0.0,
                              seed=c["seed"], grf_length=8.0)


def mog2_oracle_run(p, y, pr):
    from oracle.ep import EPOracle
    c = MOG2_DECONV
    o = EPOracle("deconv", y, p.xi, 0.0, 32, 32, kernel=p.kernel, site0="rbmc", probes=pr,
                 prior="mog2", theta=c["theta"])
    o.run(c["sweeps"])
    return o.posterior() + (o.n_capped,)


def y32(p):
    """The observation as both sides see it: rounded to float32."""
    return p.y.astype(np.float32).astype(np.float64)


def probes(p, S, seed):
    n = p.shape[0] * p.shape[1]
    return syn.rbmc_probes(S, n, n, seed=seed)


def oracle_run(p, y, pr, sweeps, em_every, order):
    from oracle.ep import EPOracle
    h, w = p.shape
    o = EPOracle("deconv", y, p.xi, p.beta, h, w, kernel=p.kernel, site0="rbmc", probes=pr,
                 order=order)
    o.run(sweeps, em_every=em_every)
    return o.posterior()
