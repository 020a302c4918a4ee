"""GPU parity of the deconvolution path (prior sweep + CG/RBMC likelihood site)."""
import numpy as np
import pytest

from oracle import operators
from oracle.ep import EPOracle
from paper_2110_01585_gb300 import EPTV, OP_CONV_PERIODIC
from paper_2110_01585_gb300 import synthetic as syn

from ._cases import DECONV_CASES, oracle_run, probes, y32
from ._parity import assert_parity, cuda

pytestmark = pytest.mark.gpu


def _probes(S, n, seed):
    return syn.rbmc_probes(S, n, n, seed=seed)


def _gpu(p, sweeps, S, pr, em_every=0, cg_rtol=1e-9, **kw):
    torch = cuda()
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    ep = EPTV(yt, p.xi, p.beta, op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=S,
              cg_rtol=cg_rtol, **kw)
    ep.set_probes(torch.as_tensor(pr[0], dtype=torch.float32, device="cuda"),
                  torch.as_tensor(pr[1], dtype=torch.float32, device="cuda"))
    ep.sweep(sweeps, em_every=em_every)
    mu, var = ep.posterior()
    st = ep.status()
    out = mu.cpu().numpy(), var.cpu().numpy(), ep
    assert st == 0, st
    return out


@pytest.mark.parametrize("name", sorted(DECONV_CASES))
def test_deconv_parity(name):
    """Uniform 9x9 with EM, uniform 5x5 on a ragged 48x80 grid with EM, a
    non-separable 5x3 kernel, a 15x15 Gaussian (the first solve after one prior
    pass with capped prior sites needs thousands of iterations), and Algorithm 1
    as listed (likelihood site first: the first solve sees a flat cavity of
    precision 4e-8, the worst-conditioned system of the run)."""
    make, (S, seed), sweeps, em_every, order, opts = DECONV_CASES[name]
    p = make()
    pr = probes(p, S, seed)
    mu, var, ep = _gpu(p, sweeps, S, pr, em_every=em_every, **opts)
    mu_r, var_r = oracle_run(p, y32(p), pr, sweeps, em_every, order)
    assert_parity(mu, var, mu_r, var_r, p.y)
    ep.close()


@pytest.mark.parametrize("h,w", [(24, 400), (320, 24)])
def test_deconv_parity_512_point_transforms(h, w):
    """Padded sizes whose preconditioner rows (24 x 400, padded to 32 x 512) or
    columns (320 x 24, padded to 512 x 32) go through the register-resident
    512-point transforms; the oracle does every solve by FP64 CG on the FFT
    operator."""
    p = syn.deconv_problem(h, w, kernel=syn.uniform_kernel(5), bsnr_db=30.0, beta0=2.0, seed=31,
                           grf_length=8.0)
    S = 4
    pr = probes(p, S, 32)
    mu, var, ep = _gpu(p, 3, S, pr)
    o = EPOracle("deconv", y32(p), p.xi, p.beta, h, w, kernel=p.kernel, site0="rbmc_cg", probes=pr)
    o.run(3)
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, p.y)
    ep.close()


@pytest.mark.parametrize("h,w", [(24, 520), (520, 24)])
def test_deconv_parity_1024_point_transforms(h, w):
    """Padded sizes whose preconditioner rows (24 x 520, padded to 32 x 1024) or
    columns (520 x 24, padded to 1024 x 32) go through the register-resident
    1024-point transforms (one decimation-in-frequency step into two 512-point
    ones); the oracle does every solve by FP64 CG on the FFT operator."""
    p = syn.deconv_problem(h, w, kernel=syn.uniform_kernel(5), bsnr_db=30.0, beta0=2.0, seed=31,
                           grf_length=8.0)
    S = 4
    pr = probes(p, S, 32)
    mu, var, ep = _gpu(p, 3, S, pr)
    o = EPOracle("deconv", y32(p), p.xi, p.beta, h, w, kernel=p.kernel, site0="rbmc_cg", probes=pr)
    o.run(3)
    mu_r, var_r = o.posterior()
    assert_parity(mu, var, mu_r, var_r, p.y)
    ep.close()


def test_unit_kernel_equals_denoising_path():
    """H = I through the CG/RBMC route: diagonal precision, exact RB estimate."""
    torch = cuda()
    p = syn.denoise_problem(32, 64, sigma=0.1, beta=10.0, seed=11)
    p.kernel = np.ones((1, 1))
    pr = _probes(2, 32 * 64, 12)
    mu, var, ep = _gpu(p, 8, 2, pr)
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(yt, p.xi, p.beta) as d:
        d.sweep(8)
        mu_d, var_d = (t.cpu().numpy() for t in d.posterior())
    np.testing.assert_allclose(mu, mu_d, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(var, var_d, rtol=1e-5)
    ep.close()


def test_checkpoint_resume_deconv():
    torch = cuda()
    p = syn.deconv_problem(32, 32, kernel=syn.uniform_kernel(5), bsnr_db=30.0, seed=13,
                           grf_length=8.0)
    pr = _probes(4, 1024, 14)
    _, _, a = _gpu(p, 4, 4, pr, em_every=2)
    _, _, b = _gpu(p, 0, 4, pr, em_every=2)
    blob = a.state_export()
    a.sweep(4, em_every=2)
    b.state_import(blob)
    b.sweep(4, em_every=2)
    ma, va = a.posterior()
    mb, vb = b.posterior()
    assert torch.equal(ma, mb) and torch.equal(va, vb)
    a.close()
    b.close()


def test_library_probes_have_standard_normal_statistics():
    """The library's own SplitMix64/Box-Muller probes (no caller probes): run and
    check that the variance estimate is close to the exact-solve oracle."""
    torch = cuda()
    p = syn.deconv_problem(32, 32, kernel=syn.uniform_kernel(5), bsnr_db=30.0, seed=15,
                           grf_length=8.0)
    yt = torch.as_tensor(p.y.astype(np.float32), device="cuda")
    with EPTV(yt, p.xi, p.beta, op=OP_CONV_PERIODIC, kernel=p.kernel, rbmc_samples=64) as ep:
        ep.sweep(3)
        mu, var = (t.cpu().numpy() for t in ep.posterior())
    o = EPOracle("deconv", p.y, p.xi, p.beta, 32, 32, kernel=p.kernel, site0="exact")
    o.run(3)
    mu_r, var_r = o.posterior()
    # Monte Carlo error of the variance with 64 probes: a few percent at most
    assert np.median(np.abs(var / var_r - 1)) < 0.05
    assert np.max(np.abs(mu - mu_r)) < 0.05 * (p.y.max() - p.y.min())


def test_full_size_512_residual_and_site0_samples():
    """512^2, 9x9 uniform blur, BSNR 40 dB: after a sweep, the mean solve satisfies
    Q E = b everywhere (checked in FP64 with the oracle's operator), and the new
    likelihood site at sampled pixels follows the RB estimate and Eq. update_q0_x."""
    torch = cuda()
    h = w = 512
    S = 32
    p = syn.deconv_problem(h, w, kernel=syn.uniform_kernel(9), bsnr_db=40.0, beta0=1.0, seed=0)
    pr = _probes(S, h * w, 21)
    _, _, ep = _gpu(p, 2, S, pr, em_every=0)
    tau0, nu0 = (t.cpu().numpy().astype(np.float64) for t in ep.sites())
    ep.sweep(1)
    tau1, nu1 = (t.cpu().numpy().astype(np.float64) for t in ep.sites())
    blob = np.frombuffer(ep.state_export(), dtype=np.uint8)
    n = h * w
    off = 4 * 8 + 4 * 8 + 2 * 4 * 5 * n
    X = np.frombuffer(blob[off:].tobytes(), dtype=np.float64).reshape(1 + S, h, w)
    ep.close()
    d = tau1[1:].sum(axis=0)          # cavity precision of site 0 (prior sites of this sweep)
    ncav = nu1[1:].sum(axis=0)
    k = p.kernel
    def Q(v):
        return operators.conv_periodic_t(operators.conv_periodic(v, k), k) / p.xi + d * v
    b = operators.conv_periodic_t(p.y, k) / p.xi + ncav
    r = b - Q(X[0])
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b)
    # probe systems
    g0 = float(np.sum(k * k)) / p.xi
    Ws = []
    for s in range(S):
        w_s = (operators.conv_periodic_t(pr[0][s].reshape(h, w), k) / np.sqrt(p.xi)
               + np.sqrt(d) * pr[1][s].reshape(h, w))
        rs = w_s - Q(X[s + 1])
        # probe solves stop at a relative residual of 1e-6 (mean solve: cg_rtol)
        assert np.linalg.norm(rs) <= 2e-6 * np.linalg.norm(w_s), s
        Ws.append(w_s)
    # site 0 at sampled pixels
    rng = np.random.default_rng(22)
    for rr, cc in rng.integers(0, 512, size=(50, 2)):
        qii = g0 + d[rr, cc]
        acc = 0.0
        for s in range(S):
            acc += (Ws[s][rr, cc] - qii * X[s + 1, rr, cc]) ** 2
        var = 1 / qii + acc / S / qii ** 2
        E = X[0, rr, cc]
        t_new = max(1 / var - d[rr, cc], 1e-8)
        n_new = t_new * E + d[rr, cc] * E - ncav[rr, cc]
        t_exp = 0.5 * t_new + 0.5 * tau0[0, rr, cc]
        n_exp = 0.5 * n_new + 0.5 * nu0[0, rr, cc]
        assert abs(tau1[0, rr, cc] / t_exp - 1) < 1e-4
        assert abs(nu1[0, rr, cc] - n_exp) <= 1e-4 * abs(t_exp) * (abs(E) + 0.1)


def test_config2_512_against_oracle_samples():
    """The deconvolution configuration at its stated size: 512 x 512, 9 x 9
    uniform periodic blur, BSNR 40 dB, 32 RBMC probes, beta0 = 1, six sweeps with
    the EM update after the fifth.  The FP64 oracle (every solve by CG to 1e-11)
    takes about 20 minutes for this on 8 cores, so its result is stored by
    tests/golden/make_deconv512.py (which calls only the oracle and the input
    generators) at 8192 sampled pixels, with the image-wide sums of the mean and
    the variance and the EM output."""
    import os

    from .golden import make_deconv512 as g

    ref = np.load(os.path.join(os.path.dirname(g.__file__), "deconv512_oracle.npz"))
    p, y32_, eps1, eps2 = g.inputs()
    # the same inputs as the stored run
    np.testing.assert_allclose(g.checksums(y32_, eps1, eps2), ref["checksums"], rtol=1e-12)
    torch = cuda()
    _, _, ep = _gpu(p, 0, g.S, (eps1, eps2))
    em = int(ref["em_every"])
    assert int(ref["sweeps"]) == em + 1
    ep.sweep(em, em_every=em)
    # ep_tv_em_beta recomputes N / a_u from the same (fifth) sweep: the beta the
    # in-sweep EM step just set, and the a_u it used
    beta, abar = ep.em_beta()
    ep.sweep(1)
    mu_t, var_t = ep.posterior()
    mu, var = (t.cpu().numpy().reshape(-1).astype(np.float64) for t in (mu_t, var_t))
    assert ep.status() == 0
    ep.close()
    assert abs(abar / float(ref["abar"]) - 1.0) < 1e-5, (abar, float(ref["abar"]))
    assert abs(beta / float(ref["beta"]) - 1.0) < 1e-5, (beta, float(ref["beta"]))
    idx = ref["idx"]
    assert_parity(mu[idx], var[idx], ref["mean"], ref["var"], p.y)
    assert abs(mu.sum() / float(ref["mean_sum"]) - 1.0) < 1e-5
    assert abs(var.sum() / float(ref["var_sum"]) - 1.0) < 1e-4


def test_deconv_mog2_prior_parity_and_no_em():
    """The MoG2-TV prior with the deconvolution likelihood site (Sec. II-B with
    Eq. tilted_P_1) against the oracle with the same probes, on an instance where
    thousands of site updates hit the variance cap; EM is refused for the mixture
    priors (Sec. IV defines it for l1-TV only)."""
    from paper_2110_01585_gb300 import PRIOR_MOG2, EPTVError

    from ._cases import MOG2_DECONV, mog2_deconv_problem, mog2_oracle_run
    c = MOG2_DECONV
    p = mog2_deconv_problem()
    pr = probes(p, c["S"], c["probe_seed"])
    theta = c["theta"]
    mu, var, ep = _gpu(p, c["sweeps"], c["S"], pr, prior=PRIOR_MOG2, omega=theta[0],
                       s1_sq=theta[1], s2_sq=theta[2])
    capped = ep.stats()["n_capped"]
    with pytest.raises(EPTVError):
        ep.sweep(1, em_every=1)
    with pytest.raises(EPTVError):
        ep.em_beta()
    ep.close()
    mu_r, var_r, capped_r = mog2_oracle_run(p, y32(p), pr)
    assert_parity(mu, var, mu_r, var_r, p.y)
    assert abs(capped - capped_r) <= max(4, 0.01 * capped_r), (capped, capped_r)
