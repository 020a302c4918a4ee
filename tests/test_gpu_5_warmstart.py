"""Learned warm start on the GPU: the network kernels (convolution forward and
backward, loss, Adam) against the FP64 oracle of oracle/cnn.py, the site
mapping of ep_tv_warm_start, training that lowers the loss, and what the
trained network gains over the cold start."""
import ctypes
import math

import numpy as np
import pytest

from oracle import cnn
from paper_2110_01585_gb300 import EPTV, OP_CONV_PERIODIC, warm_start
from paper_2110_01585_gb300 import synthetic as syn
from paper_2110_01585_gb300.warmstart import WarmStartNet

from ._parity import cuda

pytestmark = pytest.mark.gpu

# FP32 kernels against FP64: sums of up to 288 products per output, relative to
# the output scale
RTOL = 2e-5


def _close(a, ref, rtol=RTOL):
    a = np.asarray(a, np.float64)
    scale = max(1e-30, float(np.max(np.abs(ref))))
    err = float(np.max(np.abs(a - ref))) / scale
    assert err <= rtol, err


def _t(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("n,cin,cout,h,w,relu", [(2, 3, 32, 37, 45, 1), (1, 32, 32, 16, 16, 1),
                                                 (3, 32, 2, 20, 33, 0), (1, 5, 7, 1, 3, 1)])
def test_conv_forward_backward_match_oracle(n, cin, cout, h, w, relu):
    torch = cuda()
    from paper_2110_01585_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(n * 100 + cin)
    x = rng.standard_normal((n, cin, h, w)).astype(np.float32)
    wt = (rng.standard_normal((cout, cin, 3, 3)) / math.sqrt(cin * 9)).astype(np.float32)
    b = rng.standard_normal(cout).astype(np.float32)
    dy = rng.standard_normal((n, cout, h, w)).astype(np.float32)
    z = cnn.conv3x3(x.astype(np.float64), wt.astype(np.float64), b.astype(np.float64))
    yref = np.maximum(z, 0.0) if relu else z
    xd, wd, bd, dyd = _t(torch, x), _t(torch, wt), _t(torch, b), _t(torch, dy)
    yd = torch.empty((n, cout, h, w), dtype=torch.float32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p()
    assert lib.ep_tv_conv3x3_forward(n, cin, cout, h, w, P(xd), P(wd), P(bd), relu, P(yd), s) == 0
    _close(yd.cpu().numpy(), yref)
    work_bytes = lib.ep_tv_conv3x3_backward_work(n, cin, cout, h, w)
    work = torch.empty(work_bytes // 4 + 1, dtype=torch.float32, device="cuda")
    dx = torch.empty_like(xd)
    dw = torch.empty_like(wd)
    db = torch.empty_like(bd)
    assert lib.ep_tv_conv3x3_backward(n, cin, cout, h, w, P(xd), P(wd), P(yd if relu else None), P(dyd),
                                      P(dx), P(dw), P(db), P(work), ctypes.c_size_t(work.numel() * 4), s) == 0
    g = dy.astype(np.float64) * (z > 0) if relu else dy.astype(np.float64)
    dxr, dwr, dbr = cnn.conv3x3_backward(x.astype(np.float64), wt.astype(np.float64), g)
    _close(dx.cpu().numpy(), dxr)
    _close(dw.cpu().numpy(), dwr)
    _close(db.cpu().numpy(), dbr)


def test_network_step_matches_oracle():
    """Forward, loss, backward and two Adam steps of the whole network."""
    torch = cuda()
    net = WarmStartNet(seed=3)
    rng = np.random.default_rng(4)
    n, h, w = 2, 24, 40
    y = rng.random((n, h, w)).astype(np.float32)
    mean = (y + 0.05 * rng.standard_normal((n, h, w))).astype(np.float32)
    tau = np.exp(rng.standard_normal((n, 5, h, w)) + 8.0).astype(np.float32)
    xi = np.array([1e-4, 3e-5])
    log_xi = np.log(xi).astype(np.float32)
    params = [(w_.cpu().numpy().astype(np.float64), b_.cpu().numpy().astype(np.float64)) for w_, b_ in net.params]
    yt = _t(torch, y)
    x = net.features(yt, xi, 2.0)
    xr = x.cpu().numpy().astype(np.float64)
    for step in (1, 2):
        out = net.forward(x, keep=True)
        loss, dout = net.loss(out, yt, _t(torch, mean), _t(torch, tau), _t(torch, log_xi))
        grads = net.backward(dout)
        outr, acts, pres = cnn.forward(params, xr)
        lossr, gr = cnn.warmstart_loss(outr, y.astype(np.float64), mean.astype(np.float64),
                                       tau.astype(np.float64), log_xi.astype(np.float64), 100.0)
        gradsr = cnn.backward(params, acts, pres, gr)
        _close(out.cpu().numpy(), outr, 1e-4)
        assert abs(float(loss.item()) - lossr) <= 1e-4 * lossr
        for (dw, db), (dwr, dbr) in zip(grads, gradsr):
            _close(dw.cpu().numpy(), dwr, 2e-4)
            _close(db.cpu().numpy(), dbr, 2e-4)
        net.adam(grads, lr=1e-3)
        if step == 1:
            state = [(np.zeros_like(p), np.zeros_like(p), np.zeros_like(b), np.zeros_like(b)) for p, b in params]
        for (p, b), (dwr, dbr), (mw, vw, mb, vb) in zip(params, gradsr, state):
            cnn.adam_step(p, dwr, mw, vw, step, 1e-3)
            cnn.adam_step(b, dbr, mb, vb, step, 1e-3)
        for (w_, b_), (p, b) in zip(net.params, params):
            _close(w_.cpu().numpy(), p, 1e-4)


def test_warm_start_sets_sites_from_prediction():
    torch = cuda()
    rng = np.random.default_rng(5)
    for kind in ("denoise", "deconv"):
        if kind == "denoise":
            p = syn.denoise_problem(32, 48, sigma=0.1, beta=5.0, seed=6)
            ep = EPTV(_t(torch, p.y), p.xi, p.beta)
        else:
            p = syn.warmstart_problem(32, 48, seed=7)
            ep = EPTV(_t(torch, p.y), p.xi, p.beta, op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=2)
        out = rng.standard_normal((6, 32, 48)).astype(np.float32)
        out[0] *= 0.1
        out[5] -= 30.0     # site 4 below the variance cap: capped
        warm_start(ep, _t(torch, out))
        tau, nu = (a.cpu().numpy().astype(np.float64) for a in ep.sites())
        ep.close()
        mean = p.y.astype(np.float32).astype(np.float64) + out[0]
        for s_ in range(5):
            if s_ == 0 and kind == "denoise":
                np.testing.assert_allclose(tau[0], 1 / p.xi, rtol=1e-6)
                continue
            t = np.exp(out[1 + s_].astype(np.float64) - math.log(p.xi))
            if s_ > 0:
                t = np.maximum(t, 1e-8)
            np.testing.assert_allclose(tau[s_], t, rtol=2e-5)
            np.testing.assert_allclose(nu[s_], t * mean, rtol=2e-5, atol=1e-6 * np.abs(t * mean).max())


def test_training_lowers_the_loss():
    torch = cuda()
    net = WarmStartNet(seed=8)
    rng = np.random.default_rng(9)
    n, h, w = 4, 32, 32
    y = rng.random((n, h, w)).astype(np.float32)
    mean = y + 0.02 * np.sin(np.arange(w) / 3.0)[None, None, :].astype(np.float32)
    tau = np.full((n, 5, h, w), 3e3, np.float32)
    tau[:, 0] = 1e4
    xi = np.full(n, 1e-4)
    yt, mt, vt, lt = _t(torch, y), _t(torch, mean), _t(torch, tau), _t(torch, np.log(xi))
    x = net.features(yt, xi, 2.0)
    losses = []
    for _ in range(60):
        out = net.forward(x, keep=True)
        loss, dout = net.loss(out, yt, mt, vt, lt)
        losses.append(float(loss.item()))
        net.adam(net.backward(dout), lr=3e-3)
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_trained_network_against_cold_start_and_control():
    """The network shipped in the package (trained on the GPU by
    train_warmstart on 256 labelled 128^2 problems of the warm-start workload)
    against plain cold-start EP and against a non-learned control start (mean
    y, each site at the median of the training targets) on a held-out problem:
    sweeps and device seconds until the posterior is within the parity
    tolerances (1e-4 on means, 1e-3 on variances) of the converged cold-start
    posterior.  Measured on GB300 on three held-out seeds: cold 48/59/60 sweeps,
    network 40/50/50, control 43/53/54; in time both warm starts are 20-45x
    faster than the cold start (whose first likelihood-site solves, with a flat
    cavity, take thousands of CG iterations) and within a few percent of each
    other.  So most of the gain is that of any sensible initial state; the
    network adds about 7% fewer sweeps at its training size (none at 512^2)."""
    import os
    import paper_2110_01585_gb300 as pkg
    from paper_2110_01585_gb300.train_warmstart import control_constants, sweeps_to_match
    cuda()
    path = os.path.join(os.path.dirname(pkg.__file__), "data", "warmstart_gauss15_128.npz")
    net, meta = WarmStartNet.load(path)
    beta, probes = float(meta["beta"]), int(meta["probes"])
    p = syn.warmstart_problem(128, 128, seed=900002, beta=beta)
    r = sweeps_to_match(p, beta, probes, net=net, control=control_constants(beta, probes))
    cold, warm, ctrl = r["cold"], r["warm"], r["control"]
    assert None not in (cold["sweeps"], warm["sweeps"], ctrl["sweeps"]), r
    assert warm["sweeps"] < ctrl["sweeps"] < cold["sweeps"], r
    assert warm["seconds"] < 0.1 * cold["seconds"] and ctrl["seconds"] < 0.1 * cold["seconds"], r
