"""GPU parity of the denoising path (fused prior-site sweep) against the oracle."""
import numpy as np
import pytest

from oracle.ep import EPOracle
from paper_2110_01585_gb300 import EPTV, solve_host
from paper_2110_01585_gb300 import synthetic as syn

from ._parity import assert_parity, cuda

pytestmark = pytest.mark.gpu


def _gpu_run(y, xi, beta, sweeps, em_every=0, k_orders=None, **params):
    torch = cuda()
    yt = torch.as_tensor(np.asarray(y, np.float32), device="cuda")
    with EPTV(yt, xi, beta, **params) as ep:
        if k_orders is None:
            ep.sweep(sweeps, em_every=em_every)
        else:
            ep.sweep(sweeps, k_order=k_orders, em_every=em_every)
        mu, var = ep.posterior()
        assert ep.status() == 0
        torch.cuda.synchronize()
        return mu.cpu().numpy(), var.cpu().numpy(), ep


def _oracle_run(y, xi, beta, sweeps, em_every=0, k_orders=None, periodic=True):
    h, w = y.shape
    o = EPOracle("denoise", y, xi, beta, h, w, periodic=periodic)
    o.run(sweeps, em_every=em_every, k_orders=k_orders)
    return o.posterior() + (o,)


def test_config_denoise_64():
    """64x64, 8 rectangles, sigma 0.1, beta 20, damping 0.5, 50 sweeps."""
    p = syn.denoise_problem(64, 64, sigma=0.1, beta=20.0, seed=0)
    mu, var, _ = _gpu_run(p.y, p.xi, p.beta, 50)
    mu_r, var_r, _ = _oracle_run(p.y, p.xi, p.beta, 50)
    assert_parity(mu, var, mu_r, var_r, p.y)


@pytest.mark.parametrize("hw", [(86, 150), (16, 64), (18, 66), (130, 34)])
def test_multi_tile_and_ragged(hw):
    h, w = hw
    p = syn.denoise_problem(h, w, sigma=0.08, beta=15.0, seed=h + w)
    mu, var, _ = _gpu_run(p.y, p.xi, p.beta, 20)
    mu_r, var_r, _ = _oracle_run(p.y, p.xi, p.beta, 20)
    assert_parity(mu, var, mu_r, var_r, p.y)


@pytest.mark.parametrize("hw", [(37, 71), (1, 2), (5, 1), (17, 130)])
def test_free_boundary_odd_sizes(hw):
    h, w = hw
    rng = np.random.default_rng(h * 1000 + w)
    y = rng.random((h, w))
    mu, var, _ = _gpu_run(y, 0.01, 10.0, 15, periodic=0)
    mu_r, var_r, _ = _oracle_run(y, 0.01, 10.0, 15, periodic=False)
    assert_parity(mu, var, mu_r, var_r, y)


@pytest.mark.parametrize("hw", [(2, 2), (2, 4), (4, 2), (6, 8)])
def test_tiny_periodic_images(hw):
    h, w = hw
    rng = np.random.default_rng(7 * h + w)
    y = rng.random((h, w))
    mu, var, _ = _gpu_run(y, 0.02, 6.0, 12)
    mu_r, var_r, _ = _oracle_run(y, 0.02, 6.0, 12)
    assert_parity(mu, var, mu_r, var_r, y)


def test_random_k_order_per_sweep():
    p = syn.denoise_problem(48, 70, sigma=0.1, beta=12.0, seed=4)
    rng = np.random.default_rng(5)
    orders = [list(rng.permutation([1, 2, 3, 4])) for _ in range(10)]
    mu, var, _ = _gpu_run(p.y, p.xi, p.beta, 10, k_orders=orders)
    mu_r, var_r, _ = _oracle_run(p.y, p.xi, p.beta, 10, k_orders=orders)
    assert_parity(mu, var, mu_r, var_r, p.y)


def test_em_every_5_sweeps_matches_beta_trajectory():
    p = syn.denoise_problem(64, 96, sigma=0.1, beta=1.0, seed=8)
    torch = cuda()
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    o = EPOracle("denoise", p.y, p.xi, 1.0, 64, 96)
    with EPTV(yt, p.xi, 1.0) as ep:
        for t in range(6):
            ep.sweep(5)
            beta, abar = ep.em_beta()
            o.run(5)
            abar_r = o.abar
            beta_r = o.em_update()
            assert abs(abar / abar_r - 1) < 2e-5, (t, abar, abar_r)
            assert abs(beta / beta_r - 1) < 2e-5, (t, beta, beta_r)
        mu, var = ep.posterior()
        mu, var = mu.cpu().numpy(), var.cpu().numpy()
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, p.y)


def test_device_side_em_equals_explicit_em():
    p = syn.denoise_problem(32, 64, sigma=0.1, beta=1.0, seed=9)
    torch = cuda()
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(yt, p.xi, 1.0) as a, EPTV(yt, p.xi, 1.0) as b:
        a.sweep(20, em_every=5)
        for _ in range(4):
            b.sweep(5)
            b.em_beta(sync=False)
        ma, va = a.posterior()
        mb, vb = b.posterior()
        assert torch.equal(ma, mb) and torch.equal(va, vb)


def test_sites_after_one_sweep():
    """Site-level parity of all ten planes after one sweep."""
    p = syn.denoise_problem(40, 70, sigma=0.1, beta=20.0, seed=10)
    torch = cuda()
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    o = EPOracle("denoise", p.y, p.xi, p.beta, 40, 70)
    with EPTV(yt, p.xi, p.beta) as ep:
        for _ in range(3):
            ep.sweep(1)
            o.sweep()
            tau, nu = (t.cpu().numpy().reshape(5, -1).astype(np.float64) for t in ep.sites())
            np.testing.assert_allclose(tau, o.tau, rtol=2e-4, atol=1e-7)
            # a capped site (precision 1/var_cap) keeps nu = tau E + (E - m) / c, which
            # is not small: compare nu on the scale of |nu| + |tau| (|y| + 1)
            scale = np.abs(o.nu) + np.abs(o.tau) * (np.abs(p.y.reshape(-1)) + 1.0)
            assert np.max(np.abs(nu - o.nu) / scale) < 2e-4


def test_beta_zero_closed_form():
    p = syn.denoise_problem(32, 32, seed=11)
    mu, var, _ = _gpu_run(p.y, p.xi, 0.0, 10)
    np.testing.assert_allclose(var, 1.0 / (1.0 / p.xi + 4e-8), rtol=1e-6)
    np.testing.assert_allclose(mu, p.y, rtol=1e-5, atol=1e-6)


def test_solve_host_matches_device_api():
    p = syn.denoise_problem(64, 64, sigma=0.1, beta=1.0, seed=12)
    mu_h, var_h, beta_h = solve_host(p.y, p.xi, 1.0, 20, em_every=5)
    o = EPOracle("denoise", p.y, p.xi, 1.0, 64, 64)
    o.run(20, em_every=5)
    mu_r, var_r = o.posterior()
    assert_parity(mu_h, var_h, mu_r, var_r, p.y)
    assert abs(beta_h / o.lam - 1) < 2e-5


def test_checkpoint_resume_is_bit_identical():
    p = syn.denoise_problem(48, 64, sigma=0.1, beta=1.0, seed=13)
    torch = cuda()
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(yt, p.xi, 1.0) as a, EPTV(yt, p.xi, 1.0) as b:
        a.sweep(12, em_every=4)
        blob = a.state_export()
        a.sweep(8, em_every=4)
        b.state_import(blob)
        b.sweep(8, em_every=4)
        ma, va = a.posterior()
        mb, vb = b.posterior()
        assert torch.equal(ma, mb) and torch.equal(va, vb)


def test_full_size_sampled_sites_4096():
    """4096^2 (the size the bench times): one sweep from a mid-run state; sampled
    pixels recomputed by the oracle on a local patch (each pixel's new sites depend
    only on a +-2 pixel neighbourhood)."""
    torch = cuda()
    h = w = 4096
    p = syn.denoise_problem(h, w, sigma=0.1, beta=20.0, seed=14, n_rect=40)
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(yt, p.xi, p.beta) as ep:
        ep.sweep(3)
        tau0, nu0 = (t.cpu().numpy() for t in ep.sites())
        ep.sweep(1)
        tau1, nu1 = (t.cpu().numpy() for t in ep.sites())
    rng = np.random.default_rng(15)
    samples = [(int(r), int(c)) for r, c in rng.integers(0, 4096, size=(40, 2))]
    samples += [(0, 0), (4095, 4095), (0, 4095), (4095, 0), (15, 63), (16, 64)]
    for r, c in samples:
        # 12 x 12 patch with even origin, wrapping around the torus
        r0, c0 = (r - 6) & ~1, (c - 6) & ~1
        rows = [(r0 + i) % h for i in range(12)]
        cols = [(c0 + j) % w for j in range(12)]
        o = EPOracle("denoise", p.y[np.ix_(rows, cols)], p.xi, p.beta, 12, 12, periodic=False)
        o.tau = tau0[:, rows][:, :, cols].reshape(5, -1).astype(np.float64)
        o.nu = nu0[:, rows][:, :, cols].reshape(5, -1).astype(np.float64)
        o.sweep()
        idx = (r - r0) * 12 + (c - c0)
        np.testing.assert_allclose(tau1[:, r, c], o.tau[:, idx], rtol=2e-4, atol=1e-7)
        np.testing.assert_allclose(nu1[:, r, c], o.nu[:, idx], rtol=2e-4,
                                   atol=2e-4 * np.abs(o.tau[:, idx]).max())


@pytest.mark.parametrize("prior,theta,sweeps", [("mog2", (0.3, 0.1, 1e-4), 30),
                                                ("bg", (0.8, 0.1), 10)])
@pytest.mark.parametrize("h,w,periodic", [(64, 64, 1), (37, 50, 0)])
def test_mixture_priors_match_oracle(prior, theta, sweeps, h, w, periodic):
    """MoG2-TV and BG-TV denoising (Sec. II-B, Eq. MoG2_TV_prior, Eq. BG_TV) against
    the oracle, on the torus and on an odd free-boundary grid.  These priors are
    not log-concave: edges across intensity steps ask for negative site variances,
    which the cap of Sec. III-C replaces on both sides (the counts of capped site
    updates agree up to updates that sit on the cap's threshold in FP32).  With
    BG-TV's point mass, once the cap fires the site precisions of tied pixels
    grow from sweep to sweep in the oracle too (EP counting the exact-equality
    constraint around the graph's loops), so that case is compared after 10
    sweeps, while the state is still well scaled."""
    from paper_2110_01585_gb300 import PRIOR_BG, PRIOR_MOG2
    torch = cuda()
    p = syn.denoise_problem(h, w, sigma=0.1, beta=0.0, seed=h * w + len(prior))
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    kw = dict(prior=PRIOR_MOG2 if prior == "mog2" else PRIOR_BG, omega=theta[0], s1_sq=theta[1])
    if prior == "mog2":
        kw["s2_sq"] = theta[2]
    with EPTV(yt, p.xi, 0.0, periodic=periodic, **kw) as ep:
        ep.sweep(sweeps)
        mu, var = (t.cpu().numpy() for t in ep.posterior())
        capped = ep.stats()["n_capped"]
        assert ep.status() == 0
    o = EPOracle("denoise", p.y, p.xi, 0.0, h, w, periodic=bool(periodic), prior=prior, theta=theta)
    o.run(sweeps)
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, p.y)
    assert o.n_capped > 0
    assert abs(capped - o.n_capped) <= max(4, 0.01 * o.n_capped), (capped, o.n_capped)


@pytest.mark.parametrize("option", [1, 2, 3])
def test_em_options_match_beta_trajectory(option):
    """The three approximations of a_0 (Sec. IV): Option 1 (Eq. ax, E|x_i - x_j|
    under Q(x)), Option 2 (Eq. au, E|u_n| under the matched Gaussian Q(u_n)) and
    Option 3 (Eq. 3rd_alternative_a0, the tilted P_k(u_n)), each driving the EM
    update every sweep from beta0 = 1 (the fast EP-EM of Sec. V), against the
    oracle's beta trajectory and final posterior."""
    p = syn.denoise_problem(64, 96, sigma=0.1, beta=1.0, seed=8)
    torch = cuda()
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    o = EPOracle("denoise", p.y, p.xi, 1.0, 64, 96)
    with EPTV(yt, p.xi, 1.0, em_option=option) as ep:
        for t in range(12):
            ep.sweep(1)
            beta, a = ep.em_beta()
            o.sweep()
            a_r = o.em_statistic(option)
            beta_r = o.em_update(option)
            assert abs(a / a_r - 1) < 2e-5, (t, a, a_r)
            assert abs(beta / beta_r - 1) < 2e-5, (t, beta, beta_r)
        mu, var = (x.cpu().numpy() for x in ep.posterior())
        # the same through the device-side EM of ep_tv_sweep
        with EPTV(yt, p.xi, 1.0, em_option=option) as ep2:
            ep2.sweep(12, em_every=1)
            beta2, _ = ep2.em_beta()
            assert abs(beta2 / beta_r - 1) < 2e-5
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, p.y)


def test_full_ep_em_matches_oracle():
    """Algorithm 2 with the EP of Algorithm 1 run to convergence inside every EM
    iteration (sweeps until the largest change of a posterior mean is below
    1e-5 of the largest mean), from beta0 = 1: beta after each iteration and the
    length of each inner run against the oracle."""
    p = syn.denoise_problem(48, 64, sigma=0.1, beta=1.0, seed=12)
    torch = cuda()
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(yt, p.xi, 1.0) as ep:
        betas, sweeps = ep.ep_em(5, max_sweeps=300, tol=1e-5)
        mu, var = (x.cpu().numpy() for x in ep.posterior())
    o = EPOracle("denoise", p.y, p.xi, 1.0, 48, 64)
    betas_r, sweeps_r = o.ep_em(5, max_sweeps=300, tol=1e-5)
    assert all(s < 300 for s in sweeps_r)
    # the stop decision is taken in FP32 on the GPU: a run may end one sweep apart
    assert all(abs(a - b) <= 1 for a, b in zip(sweeps, sweeps_r)), (sweeps, sweeps_r)
    np.testing.assert_allclose(betas, betas_r, rtol=2e-4)
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, p.y, rtol_mean=3e-4, rtol_var=3e-3)


@pytest.mark.parametrize("sigma", [0.05, 0.1, 0.2])
def test_lambda_study_option3_nearest_mse_optimum(sigma):
    """Sec. IV (Fig. 3): of the three approximations of a_0, Option 3
    (Eq. 3rd_alternative_a0) gives the EM estimate of beta nearest (in log) the
    MSE-optimal value and the lowest MSE of the three, here on seeded synthetic
    64 x 64 denoising problems at three noise levels."""
    from paper_2110_01585_gb300.lambda_study import study
    p = syn.denoise_problem(64, 64, sigma=sigma, beta=1.0, seed=7)
    grid = np.exp(np.linspace(np.log(1.0), np.log(400.0), 25))
    beta_opt, mse_opt, _, opts = study(p, grid)
    dist = {k: abs(np.log(opts[k][0] / beta_opt)) for k in opts}
    assert dist[3] <= dist[1] and dist[3] <= dist[2], (beta_opt, opts)
    assert opts[3][1] <= opts[1][1] and opts[3][1] <= opts[2][1], opts
    # every EP-EM estimate is worse than the grid optimum
    assert all(v[1] >= mse_opt * (1 - 1e-6) for v in opts.values())


def test_diagonal_noise_denoising_matches_oracle():
    """Denoising with one noise variance per pixel (a diagonal noise covariance,
    Sec. III-C): variances spread over a factor of 20, EM every 5 sweeps."""
    torch = cuda()
    h, w = 64, 80
    p = syn.denoise_problem(h, w, sigma=0.1, beta=5.0, seed=44)
    xi = 0.004 * np.exp(np.random.default_rng(45).uniform(0.0, 3.0, h * w))
    y = p.x + np.sqrt(xi.reshape(h, w)) * np.random.default_rng(46).standard_normal((h, w))
    xi32 = xi.astype(np.float32)
    yt = torch.as_tensor(y.astype(np.float32), device="cuda")
    with EPTV(yt, 0.0, p.beta, xi_plane=torch.as_tensor(xi32, device="cuda")) as ep:
        ep.sweep(20, em_every=5)
        mu, var = (t.cpu().numpy() for t in ep.posterior())
        beta, _ = ep.em_beta()
        assert ep.status() == 0
    o = EPOracle("denoise", y.astype(np.float32).astype(np.float64), xi32.astype(np.float64), p.beta,
                 h, w)
    o.run(20, em_every=5)
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, y)
    assert abs(beta / o.em_update() - 1) < 1e-4
