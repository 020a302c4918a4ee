"""One denoising image split by rows over gloo ranks on the CPU: the halo and
EM protocol of paper_2110_01585_gb300.sharded, each rank computing its band with
the oracle (the per-block GPU computation is checked against the whole-image
GPU run in tests/test_gpu_7_sharded.py).  The bands' own rows must equal the
whole-image oracle to rounding: every site update is an elementwise function of
the same inputs, but NumPy evaluates exp and log of an element in vector or
scalar code depending on its position in the array, which can change the last
bit (1e-13 relative, here); with EM the statistic is also summed over the ranks
in another order."""
import os
import socket

import numpy as np
import pytest

from paper_2110_01585_gb300 import sharded
from paper_2110_01585_gb300 import synthetic as syn


class OracleBand:
    """One rank's band computed by the oracle: its rows plus the halo rows, rows
    not wrapping, the EM statistic taken over its own rows' edges."""

    def __init__(self, y, xi, beta, rank, world, periodic):
        from oracle.ep import EPOracle
        h, w = y.shape
        self.row0, self.rows = sharded.block_rows(h, world, periodic)[rank]
        self.top, _ = sharded.halo_sizes(h, self.row0, self.rows, periodic)
        ext = sharded.extended_rows(h, self.row0, self.rows, periodic)
        self.w = w
        self.o = EPOracle("denoise", y[ext], xi, beta, len(ext), w, periodic=periodic,
                          periodic_rows=False, count_rows=(self.top, self.top + self.rows))

    def sweep(self):
        self.o.sweep()

    def _rows(self, r):
        return slice(r * self.w, (r + 2) * self.w)

    def halo_out(self, side):
        import torch
        r = self.top if side == 0 else self.top + self.rows - 2
        sl = self._rows(r)
        return torch.as_tensor(np.concatenate([self.o.tau[1:, sl].ravel(), self.o.nu[1:, sl].ravel()]))

    def halo_in(self, side, buf):
        r = 0 if side == 0 else self.top + self.rows
        sl = self._rows(r)
        v = buf.numpy().reshape(2, 4, 2 * self.w)
        self.o.tau[1:, sl] = v[0]
        self.o.nu[1:, sl] = v[1]

    def abar(self):
        return self.o.abar

    def set_beta(self, beta):
        self.o.lam = beta

    def own_posterior(self):
        mu, var = self.o.posterior()
        return mu[self.top:self.top + self.rows], var[self.top:self.top + self.rows]


def _problem():
    return syn.denoise_problem(24, 40, sigma=0.1, beta=12.0, seed=31)


def _rank(rank, world, port, periodic, sweeps, em_every, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        band = OracleBand(p.y, p.xi, p.beta, rank, world, periodic)
        proto = sharded.BlockProtocol(band, rank, world, periodic, p.n_pixels, sharded.TorchComm())
        betas = proto.sweep(sweeps, em_every=em_every)
        mu, var = band.own_posterior()
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), mu=mu, var=var, row0=band.row0,
                 betas=np.asarray(betas))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,periodic,em_every", [(2, True, 0), (3, False, 0), (2, True, 2),
                                                     (3, True, 3)])
def test_row_bands_equal_the_whole_image(tmp_path, world, periodic, em_every):
    import torch.multiprocessing as tmp
    from oracle.ep import EPOracle
    sweeps = 6
    tmp.spawn(_rank, args=(world, _free_port(), periodic, sweeps, em_every, str(tmp_path)),
              nprocs=world, join=True)
    p = _problem()
    h, w = p.y.shape
    o = EPOracle("denoise", p.y, p.xi, p.beta, h, w, periodic=periodic)
    betas = o.run(sweeps, em_every=em_every)
    mu, var = o.posterior()
    for r in range(world):
        d = np.load(tmp_path / f"r{r}.npz")
        r0 = int(d["row0"])
        rows = slice(r0, r0 + d["mu"].shape[0])
        if em_every:
            np.testing.assert_allclose(d["betas"], betas, rtol=1e-12)
        np.testing.assert_allclose(d["mu"], mu[rows], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(d["var"], var[rows], rtol=1e-13)


def test_block_rows_partition():
    assert sharded.block_rows(24, 2, True) == [(0, 12), (12, 12)]
    assert sharded.block_rows(24, 3, False) == [(0, 8), (8, 8), (16, 8)]
    assert sharded.block_rows(25, 3, False) == [(0, 8), (8, 8), (16, 9)]
    assert sharded.block_rows(20, 3, True) == [(0, 8), (8, 6), (14, 6)]
    with pytest.raises(ValueError):
        sharded.block_rows(25, 2, True)
    assert list(sharded.extended_rows(24, 0, 12, True)) == [22, 23] + list(range(14))
    assert list(sharded.extended_rows(24, 0, 8, False)) == list(range(10))
    assert sharded.neighbours(0, 3, True) == (2, 1) and sharded.neighbours(0, 3, False) == (None, 1)
