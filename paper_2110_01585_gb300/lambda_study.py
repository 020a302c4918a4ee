"""Synthetic analogue of the paper's Fig. 3 (Sec. IV): which approximation of
a_0 (Eq. a_0) makes the EM estimate of the TV parameter land nearest the value
that minimises the MSE of the posterior mean.

For a denoising problem with known ground truth x: the posterior mean after a
fixed number of EP sweeps is computed on a grid of beta values (the paper's
lambda), giving the MSE-optimal beta on the grid; then the fast EP-EM of Sec. V
(one sweep per EM iteration, from beta0) runs with each of Options 1, 2 and 3
and reports its final beta and MSE.  The paper finds Option 3 best on its test
images; the inputs here are the seeded synthetic piecewise-constant images.

    python -m paper_2110_01585_gb300.lambda_study [--size 256] [--sigmas 0.05 0.1 0.2]
"""
from __future__ import annotations

import argparse

import numpy as np

from . import EPTV
from . import synthetic as syn


def study(problem, grid, sweeps: int = 40, em_iterations: int = 40, beta0: float = 1.0):
    """Returns (beta_opt, mse_opt, mse_on_grid, {option: (beta, mse)})."""
    import torch
    y = torch.as_tensor(problem.y.astype(np.float32), device="cuda")
    x = problem.x.astype(np.float64)

    def mse(ep):
        mu, _ = ep.posterior()
        return float(np.mean((mu.cpu().numpy().astype(np.float64) - x) ** 2))

    curve = []
    for beta in grid:
        with EPTV(y, problem.xi, float(beta)) as ep:
            ep.sweep(sweeps)
            curve.append(mse(ep))
    i = int(np.argmin(curve))
    options = {}
    for option in (1, 2, 3):
        with EPTV(y, problem.xi, beta0, em_option=option) as ep:
            ep.sweep(em_iterations, em_every=1)
            beta, _ = ep.em_beta()
            options[option] = (beta, mse(ep))
    return float(grid[i]), curve[i], curve, options


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--sigmas", type=float, nargs="+", default=[0.05, 0.1, 0.2])
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args()
    grid = np.exp(np.linspace(np.log(1.0), np.log(400.0), 41))
    print(f"{'sigma':>6} {'beta_opt':>9} {'mse_opt':>10} | " +
          " | ".join(f"option {k}: beta, mse" for k in (1, 2, 3)))
    for sigma in args.sigmas:
        p = syn.denoise_problem(args.size, args.size, sigma=sigma, beta=1.0, seed=args.seed)
        b_opt, m_opt, _, opts = study(p, grid)
        print(f"{sigma:6.3f} {b_opt:9.2f} {m_opt:10.3e} | " +
              " | ".join(f"{opts[k][0]:8.2f}, {opts[k][1]:.3e}" for k in (1, 2, 3)))


if __name__ == "__main__":
    main()
