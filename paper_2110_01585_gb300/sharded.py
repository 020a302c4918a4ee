"""One denoising image split by rows over the ranks of a torch.distributed group.

A sweep of Algorithm 1 moves information across at most one row per vertical
update (V3 and V4), two rows per sweep.  So a rank that holds its own rows plus
the two rows above and below them (a halo) computes the sweep of its own rows
exactly as the whole image would.  After every sweep the ranks trade the two
boundary rows of their prior sites; the EM statistic (Sec. IV) is the sum of
every rank's own edges, and beta = N / sum on every rank.  Nothing else is
exchanged: the likelihood site of denoising is local (Eq. tilted_P_1, H = I).

The protocol (BlockProtocol) is independent of how a block computes its sweep:
GpuBlock runs it with the library's row-block context (ep_tv_init_block), and
any object with the same five methods can stand in for it.  Messages go through
an all-gather of each rank's two boundary-row buffers, which works with NCCL
and gloo and for any number of ranks.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Tuple

import numpy as np

from . import _lib

HALO = 2  # rows a sweep can reach across (two vertical updates)


def block_rows(height: int, world: int, periodic: bool) -> List[Tuple[int, int]]:
    """(row0, rows) of each rank: contiguous blocks as equal as the pairing
    allows, every block starting on an even row (the matchings V3 and V4 pair
    rows (2b, 2b + 1) and (2b + 1, 2b + 2)); on the torus every block has an even
    number of rows."""
    if world < 1 or height < 2 * world:
        raise ValueError("every block needs at least two rows")
    pairs = height // 2
    base, extra = divmod(pairs, world)
    out, r = [], 0
    for k in range(world):
        n = 2 * (base + (1 if k < extra else 0))
        out.append((r, n))
        r += n
    if r < height:  # free boundary with an odd height: the last block takes the odd row
        if periodic:
            raise ValueError("the torus needs an even height")
        r0, n = out[-1]
        out[-1] = (r0, n + height - r)
    return out


def halo_sizes(height: int, row0: int, rows: int, periodic: bool) -> Tuple[int, int]:
    """Halo rows above and below a block: HALO where the whole image has rows."""
    top = HALO if (periodic or row0 > 0) else 0
    bottom = HALO if (periodic or row0 + rows < height) else 0
    return top, bottom


def extended_rows(height: int, row0: int, rows: int, periodic: bool) -> np.ndarray:
    """Whole-image row index of every row a block holds, top halo first."""
    top, bottom = halo_sizes(height, row0, rows, periodic)
    return np.arange(row0 - top, row0 + rows + bottom) % height


def neighbours(rank: int, world: int, periodic: bool) -> Tuple[Optional[int], Optional[int]]:
    """Ranks holding the rows above and below this rank's block (None: none)."""
    up = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    down = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return up, down


class TorchComm:
    """The two collectives the protocol uses, on a torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def all_gather(self, t):
        out = [t.new_empty(t.shape) for _ in range(self.dist.get_world_size(self.group))]
        self.dist.all_gather(out, t.contiguous(), group=self.group)
        return out

    def all_reduce_sum(self, value: float, like) -> float:
        import torch
        t = torch.tensor([value], dtype=torch.float64, device=like.device)
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())


class BlockProtocol:
    """Sweeps of one rank's block, with the halo exchange after each sweep and the
    EM update of beta every em_every sweeps.

    block: sweep(), halo_out(side) -> tensor, halo_in(side, tensor), abar() -> float
    (the a_u of its own edges in the last sweep), set_beta(beta)."""

    def __init__(self, block, rank: int, world: int, periodic: bool, n_pixels: int, comm):
        self.block, self.rank, self.world = block, rank, world
        self.periodic, self.n_pixels, self.comm = periodic, n_pixels, comm
        self.up, self.down = neighbours(rank, world, periodic)

    def exchange(self):
        import torch
        mine = torch.stack([self.block.halo_out(0), self.block.halo_out(1)])
        every = self.comm.all_gather(mine)
        if self.up is not None:
            self.block.halo_in(0, every[self.up][1])    # the block above: its last rows
        if self.down is not None:
            self.block.halo_in(1, every[self.down][0])  # the block below: its first rows

    def sweep(self, n: int = 1, em_every: int = 0):
        betas = []
        for t in range(n):
            self.block.sweep()
            self.exchange()
            if em_every and (t + 1) % em_every == 0:
                total = self.comm.all_reduce_sum(self.block.abar(), self.block.halo_out(0))
                beta = self.n_pixels / total
                self.block.set_beta(beta)
                betas.append(beta)
        return betas


class GpuBlock:
    """A rank's block on its GPU: the library's row-block context."""

    def __init__(self, y_full: np.ndarray, xi: float, beta: float, rank: int, world: int,
                 periodic: bool = True, device=None, stream=None, **params):
        import torch
        height, width = y_full.shape
        self.row0, self.rows = block_rows(height, world, periodic)[rank]
        self.top, self.bottom = halo_sizes(height, self.row0, self.rows, periodic)
        ext = extended_rows(height, self.row0, self.rows, periodic)
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.y = torch.as_tensor(np.ascontiguousarray(y_full[ext], dtype=np.float32), device=self.device)
        self.height, self.width = len(ext), width
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._lib = _lib.load()
        op = _lib.Operator()
        op.op, op.height, op.width, op.m = _lib.OP_IDENTITY, self.height, width, self.height * width
        from . import default_params
        self.params = default_params(xi=float(xi), beta=float(beta), periodic=int(periodic), **params)
        blk = _lib.Block()
        blk.global_height, blk.row0, blk.rows = height, self.row0, self.rows
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self._lib.ep_tv_init_block(ctypes.byref(op), ctypes.c_void_p(self.y.data_ptr()),
                                                  ctypes.byref(self.params), ctypes.byref(blk),
                                                  ctypes.c_void_p(self.stream.cuda_stream),
                                                  ctypes.byref(ctx)), "ep_tv_init_block")
        self._ctx = ctx
        self._bufs = [torch.empty(16 * width, dtype=torch.float32, device=self.device) for _ in range(2)]

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.ep_tv_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self):
        _lib.check(self._lib.ep_tv_sweep(self._ctx, 1, None, 0), "ep_tv_sweep")

    def halo_out(self, side: int):
        buf = self._bufs[side]
        _lib.check(self._lib.ep_tv_block_halo_out(self._ctx, int(side), ctypes.c_void_p(buf.data_ptr())),
                   "ep_tv_block_halo_out")
        self.stream.synchronize()
        return buf.clone()

    def halo_in(self, side: int, buf):
        buf = buf.to(self.device).contiguous()
        _lib.check(self._lib.ep_tv_block_halo_in(self._ctx, int(side), ctypes.c_void_p(buf.data_ptr())),
                   "ep_tv_block_halo_in")
        self.stream.synchronize()

    def abar(self) -> float:
        a = ctypes.c_double()
        _lib.check(self._lib.ep_tv_em_beta(self._ctx, None, ctypes.byref(a)), "ep_tv_em_beta")
        return a.value

    def set_beta(self, beta: float):
        _lib.check(self._lib.ep_tv_set_beta(self._ctx, float(beta)), "ep_tv_set_beta")

    def posterior(self):
        """Posterior mean and variance of the block's own rows (CUDA tensors)."""
        import torch
        mean = torch.empty((self.height, self.width), dtype=torch.float32, device=self.device)
        var = torch.empty_like(mean)
        _lib.check(self._lib.ep_tv_posterior(self._ctx, ctypes.c_void_p(mean.data_ptr()),
                                             ctypes.c_void_p(var.data_ptr())), "ep_tv_posterior")
        sl = slice(self.top, self.top + self.rows)
        return mean[sl], var[sl]
