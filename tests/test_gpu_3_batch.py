"""Batched sweeps (ep_tv_batch_*): one prior-site launch over all images plus
concurrent likelihood-site updates must give exactly what the same contexts
give when swept one by one."""
import numpy as np
import pytest

from oracle.ep import EPOracle
from paper_2110_01585_gb300 import EPTV, OP_CONV_PERIODIC, Batch
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import assert_parity, cuda

pytestmark = pytest.mark.gpu


def _problems():
    return [
        ("denoise", syn.denoise_problem(64, 96, sigma=0.1, beta=1.0, seed=1), {}),
        ("denoise", syn.denoise_problem(48, 48, sigma=0.05, beta=1.0, seed=2), {}),
        ("denoise", syn.denoise_problem(37, 71, sigma=0.1, beta=1.0, seed=3), {"periodic": 0}),
        ("deconv", syn.deconv_problem(64, 64, kernel=syn.uniform_kernel(5), sigma=0.05, seed=4,
                                      grf_length=8.0), {}),
        ("deconv", syn.deconv_problem(40, 36, kernel=syn.uniform_kernel(3), sigma=0.1, seed=5,
                                      grf_length=6.0), {}),
    ]


def _make(torch, kind, p, kw, stream):
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    if kind == "denoise":
        return EPTV(yt, p.xi, p.beta, stream=stream, **kw)
    return EPTV(yt, p.xi, p.beta, op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=4,
                cg_max_iter=20000, stream=stream, **kw)


def test_batch_equals_one_by_one():
    torch = cuda()
    stream = torch.cuda.Stream()
    probs = _problems()
    single = [_make(torch, k, p, kw, stream) for k, p, kw in probs]
    batched = [_make(torch, k, p, kw, stream) for k, p, kw in probs]
    for e in single:
        e.sweep(6, em_every=3)
    with Batch(batched) as b:
        b.sweep(6, em_every=3)
    torch.cuda.synchronize()
    # the deconvolution sites of the batch ran as graph replays, enqueued without host threads
    for (k, _, _), e in zip(probs, batched):
        if k != "denoise":
            assert e.graph_sweeps() == 6
    for e1, e2 in zip(single, batched):
        assert e1.status() == 0 and e2.status() == 0
        m1, v1 = e1.posterior()
        m2, v2 = e2.posterior()
        torch.cuda.synchronize()
        assert torch.equal(m1, m2) and torch.equal(v1, v2)
    for e in single + batched:
        e.close()


def test_batch_denoise_matches_oracle():
    torch = cuda()
    stream = torch.cuda.Stream()
    probs = [p for p in _problems() if p[0] == "denoise"]
    ctxs = [_make(torch, k, p, kw, stream) for k, p, kw in probs]
    with Batch(ctxs) as b:
        b.sweep(10, em_every=5)
    torch.cuda.synchronize()
    for (k, p, kw), e in zip(probs, ctxs):
        h, w = p.shape
        o = EPOracle("denoise", p.y, p.xi, p.beta, h, w, periodic=bool(kw.get("periodic", 1)))
        o.run(10, em_every=5)
        mu, var = (t.cpu().numpy() for t in e.posterior())
        assert_parity(mu, var, *o.posterior(), p.y)
        e.close()
