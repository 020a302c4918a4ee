"""Writes deconv512_oracle.npz: the FP64 oracle on the 512 x 512 deconvolution
workload, sampled.

Workload: seeded image of rectangles, discs and a Gaussian random field (length
32 px), 9 x 9 uniform periodic blur, Gaussian noise at BSNR 40 dB, beta0 = 1,
32 RBMC probes (standard normals, seed 21), six sweeps of Algorithm 1 with the
EM update of Algorithm 2 after the fifth.  The oracle sees the observation
rounded to float32, as the GPU does.  Stored: the posterior mean and variance
at 8192 sampled pixels, the image-wide sums of both, beta and a_u after the EM
step, and checksums of the inputs so that a test can confirm it regenerated the
same inputs.

Only the oracle and the input generators are called.  Run from the repository
root (about 20 minutes with 8 worker processes):

    python -m tests.golden.make_deconv512 --workers 8
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import multiprocessing as mp
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "deconv512_oracle.npz")
SIDE = 512
S = 32
PROBE_SEED = 21
SWEEPS = 6
EM_EVERY = 5
N_SAMPLES = 8192
SAMPLE_SEED = 512


def inputs():
    """The workload's inputs, exactly as the GPU test regenerates them."""
    from paper_2110_01585_gb300 import synthetic as syn
    p = syn.deconv_problem(SIDE, SIDE, kernel=syn.uniform_kernel(9), bsnr_db=40.0, beta0=1.0, seed=0)
    eps1, eps2 = syn.rbmc_probes(S, SIDE * SIDE, SIDE * SIDE, seed=PROBE_SEED)
    y32 = p.y.astype(np.float32).astype(np.float64)
    return p, y32, eps1, eps2


def checksums(y32, eps1, eps2):
    return np.array([y32.sum(), (y32 ** 2).sum(), eps1.sum(), (eps1 ** 2).sum(), eps2.sum(),
                     (eps2 ** 2).sum()])


def sample_indices():
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(SIDE * SIDE, N_SAMPLES, replace=False))


def main():
    from oracle.ep import EPOracle
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=8)
    args = ap.parse_args()
    p, y32, eps1, eps2 = inputs()
    pool = cf.ProcessPoolExecutor(max_workers=args.workers, mp_context=mp.get_context("spawn"))
    o = EPOracle("deconv", y32, p.xi, p.beta, SIDE, SIDE, kernel=p.kernel, site0="rbmc_cg",
                 probes=(eps1, eps2), pool=pool)
    t0 = time.time()
    beta = abar = None
    for t in range(SWEEPS):
        o.sweep()
        if (t + 1) % EM_EVERY == 0:
            abar = o.abar
            beta = o.em_update()
        print(f"sweep {t + 1}: {time.time() - t0:.0f} s", flush=True)
    pool.shutdown()
    mu, var = (a.reshape(-1) for a in o.posterior())
    idx = sample_indices()
    np.savez_compressed(OUT, idx=idx, mean=mu[idx], var=var[idx], mean_sum=mu.sum(),
                        var_sum=var.sum(), beta=beta, abar=abar, xi=p.xi,
                        checksums=checksums(y32, eps1, eps2), sweeps=SWEEPS, em_every=EM_EVERY)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
