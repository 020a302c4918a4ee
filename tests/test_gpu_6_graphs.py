"""Sweeps replayed from captured CUDA graphs (contexts and batches without a
likelihood solver, on a non-default stream) give exactly what the same sweeps
give when launched one by one."""
import numpy as np
import pytest

from paper_2110_01585_gb300 import EPTV, Batch
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import cuda

pytestmark = pytest.mark.gpu


def _eq(a, b):
    ma, va = a.posterior()
    mb, vb = b.posterior()
    import torch
    torch.cuda.synchronize()
    return bool(torch.equal(ma, mb) and torch.equal(va, vb))


@pytest.mark.parametrize("n,em", [(10, 0), (12, 3), (9, 2)])
def test_context_graph_equals_plain_launches(n, em):
    torch = cuda()
    stream = torch.cuda.Stream()
    p = syn.denoise_problem(96, 130, sigma=0.1, beta=2.0, seed=31)
    y = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(y, p.xi, p.beta, stream=stream) as g, EPTV(y, p.xi, p.beta, stream=stream) as plain:
        g.sweep(n, em_every=em)                                  # graph replay
        plain.sweep(n, k_order=[[1, 2, 3, 4]] * n, em_every=em)  # explicit order: plain launches
        assert _eq(g, plain)
        # again from the other buffer parity, after an odd number of sweeps
        g.sweep(1)
        plain.sweep(1, k_order=[[1, 2, 3, 4]])
        g.sweep(n, em_every=em)
        plain.sweep(n, k_order=[[1, 2, 3, 4]] * n, em_every=em)
        assert _eq(g, plain)
        assert g.status() == 0 and plain.status() == 0
        period = 2 if em == 0 else (em if em % 2 == 0 else 2 * em)
        assert g.graph_sweeps() == 2 * (n // period) * period
        assert plain.graph_sweeps() == 0


def test_batch_graph_equals_one_by_one():
    torch = cuda()
    stream = torch.cuda.Stream()
    probs = [syn.denoise_problem(64, 96, sigma=0.1, beta=1.0, seed=41),
             syn.denoise_problem(37, 71, sigma=0.05, beta=1.0, seed=42),
             syn.denoise_problem(128, 128, sigma=0.2, beta=1.0, seed=43)]
    kw = [{}, {"periodic": 0}, {}]

    def make():
        return [EPTV(torch.as_tensor(p.y.astype(np.float32), device="cuda"), p.xi, p.beta,
                     stream=stream, **k) for p, k in zip(probs, kw)]

    batched, single = make(), make()
    with Batch(batched) as b:
        b.sweep(8, em_every=2)     # graph replay (period 2, four replays)
        b.sweep(3, em_every=0)     # plain launches (too short for a replay)
    for e in single:
        e.sweep(8, k_order=[[1, 2, 3, 4]] * 8, em_every=2)
        e.sweep(3, k_order=[[1, 2, 3, 4]] * 3)
    for e1, e2 in zip(batched, single):
        assert _eq(e1, e2)
        assert e1.status() == 0
        assert e1.graph_sweeps() == 8 and e2.graph_sweeps() == 0
    for e in batched + single:
        e.close()


@pytest.mark.parametrize("h,w,kernel,em", [(64, 64, 9, 3), (48, 80, 5, 0)])
def test_deconv_update_graph_equals_host_driven_loop(h, w, kernel, em):
    """The deconvolution likelihood site as one graph per update (refinement
    passes and CG iterations as conditional WHILE nodes on device counters)
    against the host-driven loop that runs when tracing is on: the same kernels
    in the same order on the same data, so the whole state (sites, solutions,
    beta, a_u) agrees bit for bit, over both prior-site buffers and with EM."""
    from paper_2110_01585_gb300 import OP_CONV_PERIODIC
    torch = cuda()
    stream = torch.cuda.Stream()
    p = syn.deconv_problem(h, w, kernel=syn.uniform_kernel(kernel), bsnr_db=35.0, beta0=2.0, seed=h + w,
                           grf_length=8.0)
    y = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    kw = dict(op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=6, stream=stream)
    with EPTV(y, p.xi, p.beta, **kw) as g, EPTV(y, p.xi, p.beta, **kw) as host:
        host.trace(True)  # tracing brackets every launch: the host-driven loop
        for n in (3, 4):
            g.sweep(n, em_every=em)
            host.sweep(n, em_every=em)
        assert g.status() == 0 and host.status() == 0
        assert g.state_export() == host.state_export()
        assert g.graph_sweeps() == 7 and host.graph_sweeps() == 0
        assert g.stats()["cg_iters"] > 0
        rep = g.solver_report()
        assert rep["relres_mean"] <= 1e-9 and rep["relres_probe_max"] <= 1e-6
