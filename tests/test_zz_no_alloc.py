"""The allocation-free prior-site pass (ep_tv_prior_sweep_noalloc) against the
regular ep_tv_sweep, through the C ABI.

The allocation-free entry point is for callers that cannot call cudaMalloc when
they run a sweep (code that must not allocate after start-up, or that runs
inside a runtime owning all device memory); its scratch lives in a fixed static
device array.  It runs the same kernel as ep_tv_sweep on the same inputs, so two
calls in a row (the second fed with the first's output) must give the prior
sites and the EM statistic a_u of two regular sweeps bit for bit."""
import ctypes

import numpy as np
import pytest

from paper_2110_01585_gb300 import EPTV, OP_CONV_PERIODIC, _lib, default_params
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import cuda

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _two_calls(ep, h, w, params, beta, y, order, site0_stored):
    """Runs ep.sweep(1) and the allocation-free pass alternately, twice, and
    checks the prior sites and a_u of each pair for bit identity."""
    torch = cuda()
    lib = _lib.load()
    n = h * w
    stream = torch.cuda.current_stream()
    beta_d = torch.tensor([beta], dtype=torch.float64, device="cuda")
    # prior sites as Algorithm 1 initialises them
    t_a = torch.full((4, n), 1e-8, dtype=torch.float32, device="cuda")
    n_a = torch.zeros((4, n), dtype=torch.float32, device="cuda")
    t_b = torch.empty_like(t_a)
    n_b = torch.empty_like(n_a)
    abar = torch.zeros(1, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    ko = None if order is None else (ctypes.c_int8 * 4)(*order)
    for call in range(2):
        tau_before, nu_before = ep.sites()
        tau0 = tau_before[0].reshape(-1).contiguous()
        nu0 = nu_before[0].reshape(-1).contiguous()
        ep.sweep(1, k_order=None if order is None else [order])
        tau_ref, nu_ref = ep.sites()
        _, abar_ref = ep.em_beta()
        ep.set_beta(beta)  # keep beta fixed for the next regular sweep
        src, dst = ((t_a, n_a), (t_b, n_b)) if call == 0 else ((t_b, n_b), (t_a, n_a))
        if site0_stored:
            y_arg, t0_arg, n0_arg = None, _ptr(tau0), _ptr(nu0)
        else:
            y_arg, t0_arg, n0_arg = _ptr(y), None, None
        code = lib.ep_tv_prior_sweep_noalloc(
            h, w, ctypes.byref(params), _ptr(beta_d), y_arg, t0_arg, n0_arg,
            _ptr(src[0]), _ptr(src[1]), _ptr(dst[0]), _ptr(dst[1]), ko,
            _ptr(abar), _ptr(flags), ctypes.c_void_p(stream.cuda_stream))
        assert code == 0, _lib.STATUS_NAMES.get(code, code)
        torch.cuda.synchronize()
        assert int(flags.item()) == 0
        # same kernel, same inputs: identical bits
        assert torch.equal(dst[0], tau_ref.reshape(5, n)[1:]), call
        assert torch.equal(dst[1], nu_ref.reshape(5, n)[1:]), call
        assert float(abar.item()) == abar_ref, (float(abar.item()), abar_ref)


@pytest.mark.parametrize("hw,periodic,order", [((96, 130), 1, None), ((37, 71), 0, None),
                                               ((64, 124), 1, (3, 1, 4, 2))])
def test_noalloc_prior_pass_matches_ep_tv_sweep(hw, periodic, order):
    """Denoising (site 0 formed from y inside the kernel), periodic and free
    boundary, default and a non-default order of the four updates."""
    torch = cuda()
    h, w = hw
    p = syn.denoise_problem(h, w, sigma=0.1, beta=15.0, seed=h + w)
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    params = default_params(xi=p.xi, beta=p.beta, periodic=periodic)
    with EPTV(yt, p.xi, p.beta, periodic=periodic) as ep:
        _two_calls(ep, h, w, params, p.beta, yt.reshape(-1), order, site0_stored=False)


def test_noalloc_prior_pass_with_stored_likelihood_site():
    """y = NULL: the likelihood site is passed in (tau0, nu0), as for a
    deconvolution context, whose site 0 changes every sweep."""
    torch = cuda()
    h = w = 32
    p = syn.deconv_problem(h, w, kernel=syn.uniform_kernel(5), bsnr_db=30.0, beta0=3.0, seed=41,
                           grf_length=8.0)
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    params = default_params(xi=p.xi, beta=p.beta)
    with EPTV(yt, p.xi, p.beta, op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=2) as ep:
        _two_calls(ep, h, w, params, p.beta, None, (2, 4, 1, 3), site0_stored=True)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """Argument checks run on the host; nothing is launched."""
    lib = _lib.load()
    params = default_params(xi=0.01, beta=1.0)
    dummy = ctypes.c_void_p(256)

    def call(h, w, prm):
        return lib.ep_tv_prior_sweep_noalloc(h, w, ctypes.byref(prm), dummy, dummy, None, None,
                                             dummy, dummy, ctypes.c_void_p(512),
                                             ctypes.c_void_p(768), None, dummy, None, None)

    # ceil(64 / 60) * ceil(((16 * 65537 + 1) // 2 + 1) / 16) = 2 * 32769 work units
    # (16 row pairs of a 60-column strip each) exceed the 65536 of the fixed array
    assert call(16 * 65537, 64, params) == 1
    # more than 2^31 pixels: rejected before any unit count could overflow
    assert call(1 << 30, 4, params) == 1
    assert call(1 << 30, 1 << 30, params) == 1
    bad = default_params(xi=0.01, beta=1.0, precision=7)
    assert call(64, 64, bad) == 1
