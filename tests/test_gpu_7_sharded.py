"""Row blocks of a sharded denoising image on the GPU (ep_tv_init_block and the
halo calls), against the whole image in one context.  The blocks of all ranks
run here one after another on one GPU, with the exchange of
paper_2110_01585_gb300.sharded done in-process (the multi-process protocol is
covered by tests/test_sharded_cpu.py with gloo ranks).  Every site update of a
block is the same arithmetic on the same inputs as in the whole image, so the
blocks' own rows equal it bit for bit."""
import numpy as np
import pytest

from paper_2110_01585_gb300 import EPTV, sharded
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import cuda

pytestmark = pytest.mark.gpu


def _run_blocks(p, world, periodic, sweeps, em_every=0):
    torch = cuda()
    blocks = [sharded.GpuBlock(p.y, p.xi, p.beta, r, world, periodic=periodic) for r in range(world)]
    betas = []
    for t in range(sweeps):
        for b in blocks:
            b.sweep()
        outs = [torch.stack([b.halo_out(0), b.halo_out(1)]) for b in blocks]
        for r, b in enumerate(blocks):
            up, down = sharded.neighbours(r, world, periodic)
            if up is not None:
                b.halo_in(0, outs[up][1])
            if down is not None:
                b.halo_in(1, outs[down][0])
        if em_every and (t + 1) % em_every == 0:
            beta = p.n_pixels / sum(b.abar() for b in blocks)
            for b in blocks:
                b.set_beta(beta)
            betas.append(beta)
    mu = torch.cat([b.posterior()[0] for b in blocks]).cpu().numpy()
    var = torch.cat([b.posterior()[1] for b in blocks]).cpu().numpy()
    for b in blocks:
        b.close()
    return mu, var, betas


@pytest.mark.parametrize("h,w,world,periodic", [(96, 130, 2, True), (71, 64, 3, False),
                                                (128, 200, 4, True)])
def test_blocks_equal_the_whole_image(h, w, world, periodic):
    torch = cuda()
    p = syn.denoise_problem(h, w, sigma=0.1, beta=15.0, seed=h + w)
    mu, var, _ = _run_blocks(p, world, periodic, 7)
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(yt, p.xi, p.beta, periodic=int(periodic)) as ep:
        ep.sweep(7)
        mu_r, var_r = (t.cpu().numpy() for t in ep.posterior())
    np.testing.assert_array_equal(mu, mu_r)
    np.testing.assert_array_equal(var, var_r)


def test_blocks_with_em_follow_the_whole_image():
    """EM every two sweeps from the blocks' summed a_u (their own edges): the
    beta trajectory of the whole image, up to the order of the FP64 sums."""
    torch = cuda()
    p = syn.denoise_problem(96, 128, sigma=0.1, beta=1.0, seed=5)
    mu, var, betas = _run_blocks(p, 2, True, 8, em_every=2)
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    ref = []
    with EPTV(yt, p.xi, p.beta) as ep:
        for _ in range(4):
            ep.sweep(2)
            ref.append(ep.em_beta()[0])
        mu_r, var_r = (t.cpu().numpy() for t in ep.posterior())
    np.testing.assert_allclose(betas, ref, rtol=1e-6)
    np.testing.assert_allclose(mu, mu_r, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(var, var_r, rtol=1e-5)
