"""Train the warm-start network on posteriors of plain cold-start EP, and
measure what it gains.

    python -m paper_2110_01585_gb300.train_warmstart --out net.npz [--images 512]

Labels: ``--images`` seeded 128 x 128 problems of the warm-start workload
(synthetic.warmstart_problem: 15 x 15 Gaussian blur, std 2 px, BSNR 30 dB),
each run through plain EP from the cold start for ``--label-sweeps`` sweeps at a
fixed TV parameter.  That parameter is the EM fixed point (Algorithm 2) of one
separate problem of the same workload, found first.  Training: Adam on
minibatches of the eight torus symmetries (rotations and flips, under which the
workload is invariant) of the labelled images.  Everything runs on the GPU
through libeptv; the network file records the TV parameter and the settings.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np


_TRANSPOSED_SITES = [0, 3, 4, 1, 2]


def _sym(a, k, sites: bool = False):
    """k-th of the 8 symmetries of the square torus (last two axes): row flip
    (k & 1), column flip (k & 2), transpose (k & 4).  Flips map each matching V_k
    onto itself (even sides); the transpose swaps horizontal and vertical ones,
    so a stack of five site planes has V1 <-> V3 and V2 <-> V4 exchanged."""
    import torch
    if k & 1:
        a = torch.flip(a, dims=(-2,))
    if k & 2:
        a = torch.flip(a, dims=(-1,))
    if k & 4:
        a = a.transpose(-1, -2)
        if sites:
            a = a[_TRANSPOSED_SITES]
    return a


def fixed_beta(side: int, sweeps: int, probes: int, seed: int = 999) -> float:
    """EM fixed point of beta on one problem of the workload."""
    import torch
    from . import EPTV, OP_CONV_PERIODIC
    from . import synthetic as syn
    p = syn.warmstart_problem(side, side, seed=seed, beta=1.0)
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(yt, p.xi, 1.0, op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=probes,
              cg_max_iter=20000, cg_rtol=CG_RTOL) as ep:
        ep.sweep(sweeps - 5, em_every=5)
        ep.sweep(5)
        return float(ep.em_beta()[0])


# Mean solves of labelling and evaluation stop at a relative residual of 1e-9,
# as in the parity tests: with looser solves the EP map depends on the solver's
# history, and runs from different starts settle at different states.
CG_RTOL = 1e-9


def label(seeds, side: int, beta: float, sweeps: int, probes: int, group: int = 32, log=print):
    """(y, mean, tau, xi) of plain cold-start EP for each seed: observation,
    posterior mean, the five site precisions (CUDA tensors) and noise variance.
    A problem is kept when the likelihood-site solves of its last sweep met their
    tolerances (the badly conditioned first solves of a cold start may not, which
    the context's status records); the others are left out."""
    import torch
    from . import EPTV, OP_CONV_PERIODIC, Batch
    from . import synthetic as syn
    ys, means, vars_, xis = [], [], [], []
    stream = torch.cuda.current_stream()
    for g0 in range(0, len(seeds), group):
        probs = [syn.warmstart_problem(side, side, seed=s, beta=beta) for s in seeds[g0:g0 + group]]
        eps = [EPTV(torch.as_tensor(p.y.astype(np.float32), device="cuda"), p.xi, beta,
                    op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=probes, cg_max_iter=20000,
                    cg_rtol=CG_RTOL, stream=stream) for p in probs]
        with Batch(eps) as b:
            b.sweep(sweeps)
        for p, ep in zip(probs, eps):
            rep = ep.solver_report()
            if ep.status() not in (0, 5) or rep["relres_mean"] > 1e-8 or rep["relres_probe_max"] > 1e-5:
                log(f"seed {p.seed}: EP status {ep.status()}, last solve {rep}, left out")
                ep.close()
                continue
            m, _ = ep.posterior()
            tau, _ = ep.sites()
            ys.append(torch.as_tensor(p.y.astype(np.float32), device="cuda"))
            means.append(m)
            vars_.append(tau)
            xis.append(p.xi)
            ep.close()
    return torch.stack(ys), torch.stack(means), torch.stack(vars_), np.asarray(xis)


def train(net, y, mean, tau, xi, epochs: int, batch: int, lr: float, blur_std: float, seed: int = 0,
          log=print):
    import torch
    n = y.shape[0]
    rng = np.random.default_rng(seed)
    log_xi_all = torch.as_tensor(np.log(xi), dtype=torch.float32, device="cuda")
    steps_per_epoch = (8 * n) // batch
    total = epochs * steps_per_epoch
    step = 0
    hist = []
    for ep in range(epochs):
        order = rng.permutation(8 * n)
        acc = 0.0
        for s in range(steps_per_epoch):
            idx = order[s * batch:(s + 1) * batch]
            img = torch.as_tensor(idx // 8, device="cuda")
            yb = torch.stack([_sym(y[i // 8], i % 8) for i in idx]).contiguous()
            mb = torch.stack([_sym(mean[i // 8], i % 8) for i in idx]).contiguous()
            tb = torch.stack([_sym(tau[i // 8], i % 8, sites=True) for i in idx]).contiguous()
            lb = log_xi_all[img].contiguous()
            x = net.features(yb, xi[idx // 8], blur_std)
            out = net.forward(x, keep=True)
            loss, dout = net.loss(out, yb, mb, tb, lb)
            grads = net.backward(dout)
            # cosine decay of the learning rate
            step += 1
            net.adam(grads, lr=lr * 0.5 * (1.0 + math.cos(math.pi * step / total)))
            acc += float(loss.item())
        hist.append(acc / steps_per_epoch)
        log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.5f}")
    return hist


def rel_errors(mean, var, ref_mean, ref_var, y):
    """Largest relative errors of mean and variance against a reference (the
    parity metric: the mean scale is floored at 1e-3 of the observation range)."""
    import torch
    floor = 1e-3 * float(y.max() - y.min())
    e_mu = float(torch.max(torch.abs(mean - ref_mean) / torch.clamp(torch.abs(ref_mean), min=floor)))
    e_var = float(torch.max(torch.abs(var - ref_var) / ref_var))
    return e_mu, e_var


def control_constants(beta: float, probes: int, side: int = 128, images: int = 8,
                      sweeps: int = 100, seed: int = 770000):
    """The non-learned warm start's constants: for each of the five sites the
    median over labelled images and pixels of the network's target log(tau_s) +
    log(xi) (the training labels of the same workload; seeds apart from the
    training and evaluation sets)."""
    import torch
    y, mean, tau, xi = label(list(range(seed, seed + images)), side, beta, sweeps, probes,
                             log=lambda s: None)
    t = torch.log(tau.double()) + torch.as_tensor(np.log(xi), device=tau.device).view(-1, 1, 1, 1)
    return [float(torch.median(t[:, s_].reshape(-1))) for s_ in range(5)]


def control_output(y, consts):
    """The 6-plane output a warm start takes, without a network: posterior mean
    y (residual 0) and the constant site log-precisions consts."""
    import torch
    h, w = y.shape[-2:]
    out = torch.zeros((6, h, w), dtype=torch.float32, device=y.device)
    for s_ in range(5):
        out[1 + s_] = consts[s_]
    return out


def sweeps_to_match(problem, beta: float, probes: int, net=None, blur_std: float = 2.0,
                    ref_sweeps: int = 250, max_sweeps: int = 150, tol_mean: float = 1e-4,
                    tol_var: float = 1e-3, warm_mode: int = 0, control=None):
    """Sweeps and device seconds plain EP needs, from the cold start, from the
    network's warm start ("warm") and from the non-learned control start
    (control_output of the constants control, if given), until its posterior is
    within (tol_mean, tol_var) of the converged cold-start posterior (ref_sweeps
    sweeps; by default the parity tolerances of the oracle tests).  Seconds
    count the network or control and the warm start, and the sweeps, timed with
    CUDA events; the checks between sweeps are not timed."""
    import torch
    from . import EPTV, OP_CONV_PERIODIC, warm_start
    p = problem
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")

    def make():
        return EPTV(yt, p.xi, beta, op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=probes,
                    cg_max_iter=20000, cg_rtol=CG_RTOL)

    with make() as ref:
        ref.sweep(ref_sweeps)
        rm, rv = ref.posterior()
        rm, rv = rm.clone(), rv.clone()
    out = {}
    for mode in ("cold", "warm", "control"):
        if (mode == "warm" and net is None) or (mode == "control" and control is None):
            continue
        ep = make()
        seconds = 0.0
        if mode != "cold":
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pred = net.predict(yt, p.xi, blur_std) if mode == "warm" else control_output(yt, control)
            warm_start(ep, pred, warm_mode)
            e1.record()
            e1.synchronize()
            seconds += e0.elapsed_time(e1) / 1e3
        hit = None
        for n in range(1, max_sweeps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ep.stream)
            ep.sweep(1)
            e1.record(ep.stream)
            e1.synchronize()
            seconds += e0.elapsed_time(e1) / 1e3
            m, v = ep.posterior()
            e = rel_errors(m, v, rm, rv, yt)
            if e[0] <= tol_mean and e[1] <= tol_var:
                hit = n
                break
        ep.close()
        out[mode] = {"sweeps": hit, "seconds": seconds if hit else None}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--images", type=int, default=512)
    ap.add_argument("--side", type=int, default=128)
    ap.add_argument("--label-sweeps", type=int, default=100)
    ap.add_argument("--probes", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=24)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    import torch
    from .warmstart import WarmStartNet
    from . import synthetic as syn
    t0 = time.time()
    beta = fixed_beta(args.side, 60, args.probes)
    print(f"fixed beta {beta:.4f} ({time.time() - t0:.1f} s)", flush=True)
    seeds = list(range(10000 + args.seed * 100000, 10000 + args.seed * 100000 + args.images))
    y, mean, tau, xi = label(seeds, args.side, beta, args.label_sweeps, args.probes,
                             log=lambda s: print(s, flush=True))
    torch.cuda.synchronize()
    print(f"labelled {y.shape[0]} of {len(seeds)} images ({time.time() - t0:.1f} s)", flush=True)
    net = WarmStartNet(seed=args.seed)
    hist = train(net, y, mean, tau, xi, args.epochs, args.batch, args.lr, syn.WARMSTART_BLUR_STD,
                 seed=args.seed, log=lambda s: print(s, flush=True))
    net.save(args.out, beta=beta, blur_std=syn.WARMSTART_BLUR_STD, images=args.images, side=args.side,
             label_sweeps=args.label_sweeps, probes=args.probes, epochs=args.epochs,
             final_loss=hist[-1])
    print(f"saved {args.out} ({time.time() - t0:.1f} s)", flush=True)


if __name__ == "__main__":
    main()
