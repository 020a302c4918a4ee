"""The allocation-free prior-site pass (ep_tv_prior_sweep_noalloc) against the
regular ep_tv_sweep, through the C ABI.

The allocation-free entry point is for callers that cannot call cudaMalloc when
they run a sweep; its scratch lives in a fixed static device array.  Two calls
in a row (the second fed with the first's output) must give the sites and the
EM statistic a_u of two regular sweeps."""
import ctypes

import numpy as np
import pytest

from paper_2110_01585_gb300 import EPTV, _lib, default_params
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import cuda

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("hw,periodic", [((96, 130), 1), ((37, 71), 0)])
def test_noalloc_prior_pass_matches_ep_tv_sweep(hw, periodic):
    torch = cuda()
    h, w = hw
    p = syn.denoise_problem(h, w, sigma=0.1, beta=15.0, seed=h + w)
    lib = _lib.load()
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    n = h * w
    stream = torch.cuda.current_stream()
    params = default_params(xi=p.xi, beta=p.beta, periodic=periodic)
    beta_d = torch.tensor([p.beta], dtype=torch.float64, device="cuda")
    # prior sites as Algorithm 1 initialises them
    t_a = torch.full((4, n), 1e-8, dtype=torch.float32, device="cuda")
    n_a = torch.zeros((4, n), dtype=torch.float32, device="cuda")
    t_b = torch.empty_like(t_a)
    n_b = torch.empty_like(n_a)
    abar = torch.zeros(1, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    with EPTV(yt, p.xi, p.beta, periodic=periodic) as ep:
        for call in range(2):
            ep.sweep(1)
            tau_ref, nu_ref = ep.sites()
            _, abar_ref = ep.em_beta()
            ep.set_beta(p.beta)  # keep beta fixed for the next regular sweep
            src, dst = ((t_a, n_a), (t_b, n_b)) if call == 0 else ((t_b, n_b), (t_a, n_a))
            code = lib.ep_tv_prior_sweep_noalloc(
                h, w, ctypes.byref(params), _ptr(beta_d), _ptr(yt), None, None,
                _ptr(src[0]), _ptr(src[1]), _ptr(dst[0]), _ptr(dst[1]), None,
                _ptr(abar), _ptr(flags), ctypes.c_void_p(stream.cuda_stream))
            assert code == 0, _lib.STATUS_NAMES.get(code, code)
            torch.cuda.synchronize()
            assert int(flags.item()) == 0
            tau_got = dst[0].cpu().numpy().astype(np.float64)
            nu_got = dst[1].cpu().numpy().astype(np.float64)
            tau_exp = tau_ref.cpu().numpy().reshape(5, n)[1:].astype(np.float64)
            nu_exp = nu_ref.cpu().numpy().reshape(5, n)[1:].astype(np.float64)
            # same kernel on the same inputs: the site tolerance of the parity tests
            np.testing.assert_allclose(tau_got, tau_exp, rtol=2e-4, atol=1e-7)
            scale = np.abs(nu_exp) + np.abs(tau_exp)
            assert np.max(np.abs(nu_got - nu_exp) / scale) < 2e-4
            assert abs(float(abar.item()) / abar_ref - 1.0) < 2e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """Argument checks run on the host; nothing is launched."""
    lib = _lib.load()
    params = default_params(xi=0.01, beta=1.0)
    dummy = ctypes.c_void_p(256)
    # 65537 tiles of 16 x 64 pixels exceed the fixed scratch array
    code = lib.ep_tv_prior_sweep_noalloc(16 * 65537, 64, ctypes.byref(params), dummy, dummy, None,
                                         None, dummy, dummy, ctypes.c_void_p(512),
                                         ctypes.c_void_p(768), None, dummy, None, None)
    assert code == 1
