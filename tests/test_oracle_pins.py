"""Pins that tie the FP64 oracle to the paper and to mathematics, not to itself.

Each test checks the oracle against something it does not compute itself:
high-precision quadrature, textbook closed forms, an exact special case of the
method, brute-force enumeration, FFT closed forms or a symmetry of the model.
"""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy.stats import norm

from oracle import operators
from oracle.ep import EPOracle
from oracle.partition import edges
from oracle.tilted import laplace_tilted
from paper_2110_01585_gb300 import synthetic as syn


# ---------------------------------------------------------------- tilted moments
def _quad_tilted(mu, s2, lam, dps=30):
    """Mean, variance and E|u| of N(u; mu, s2) exp(-lam|u|) by mpmath quadrature
    of the raw integrand on a grid refined around the kink and the modes."""
    mp.mp.dps = dps
    mu, s2, lam = mp.mpf(mu), mp.mpf(s2), mp.mpf(lam)
    s = mp.sqrt(s2)

    def f(u):
        return mp.exp(-(u - mu) ** 2 / (2 * s2) - lam * abs(u))

    pts = set()
    for md in (max(mp.mpf(0), mu - lam * s2), min(mp.mpf(0), mu + lam * s2), mp.mpf(0)):
        for k in range(-30, 31):
            pts.add(md + k * s / 2)
    a_plus, a_minus = lam * s - mu / s, lam * s + mu / s
    for a, sign in ((a_plus, 1), (a_minus, -1)):
        if a > 1:
            for k in range(0, 61):
                pts.add(sign * k * s / a / 2)
    pts = sorted(pts)
    grid = [pts[0] - 20 * s] + pts + [pts[-1] + 20 * s]
    z = mp.quad(f, grid)
    m1 = mp.quad(lambda u: u * f(u), grid) / z
    var = mp.quad(lambda u: (u - m1) ** 2 * f(u), grid) / z
    eabs = mp.quad(lambda u: abs(u) * f(u), grid) / z
    return float(m1), float(var), float(eabs)


QUAD_CASES = [(m, l) for m in (-50.0, -7.0, -0.3, 0.0, 3.0, 12.0, 50.0)
              for l in (1e-4, 0.3, 4.0, 50.0)]


@pytest.mark.parametrize("mu_over_s,lam_s", QUAD_CASES)
def test_tilted_moments_match_quadrature(mu_over_s, lam_s):
    """P1: the closed forms (erfcx and continued fraction) agree with quadrature to 1e-10."""
    s2 = 0.04
    s = math.sqrt(s2)
    mu, lam = mu_over_s * s, lam_s / s
    ref = _quad_tilted(mu, s2, lam)
    got = [float(v[0]) for v in laplace_tilted(np.array([mu]), np.array([s2]), lam)]
    assert abs(got[0] - ref[0]) <= 1e-10 * max(abs(ref[0]), 1e-3 * s)
    assert abs(got[1] - ref[1]) <= 1e-10 * ref[1]
    assert abs(got[2] - ref[2]) <= 1e-10 * ref[2]


def test_tilted_lambda_zero_is_gaussian_and_folded_normal():
    """lam = 0: the tilted law is N(mu, s2); E|u| is the folded-normal mean."""
    rng = np.random.default_rng(3)
    mu = rng.normal(size=200) * 3
    s2 = rng.uniform(0.01, 4, size=200)
    m, v, ea = laplace_tilted(mu, s2, 0.0)
    s = np.sqrt(s2)
    folded = s * math.sqrt(2 / math.pi) * np.exp(-mu ** 2 / (2 * s2)) + mu * (1 - 2 * norm.cdf(-mu / s))
    np.testing.assert_allclose(m, mu, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(v, s2, rtol=1e-12)
    np.testing.assert_allclose(ea, folded, rtol=1e-12)


def test_tilted_log_concavity_and_symmetry():
    """P6: for a log-concave factor the tilted variance never exceeds s2; the
    moments are odd/even in mu because exp(-lam|u|) is even."""
    rng = np.random.default_rng(4)
    mu = rng.normal(size=2000) * 5
    s2 = np.exp(rng.uniform(-8, 3, size=2000))
    for lam in (0.01, 1.0, 30.0, 400.0):
        m, v, ea = laplace_tilted(mu, s2, lam)
        assert np.all(v <= s2 * (1 + 1e-13))
        assert np.all(v > 0) and np.all(ea > 0)
        m2, v2, ea2 = laplace_tilted(-mu, s2, lam)
        np.testing.assert_allclose(m2, -m, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(v2, v, rtol=1e-12)
        np.testing.assert_allclose(ea2, ea, rtol=1e-12)


# ---------------------------------------------------------------- partition
@pytest.mark.parametrize("hw", [(2, 2), (4, 6), (6, 4), (8, 8)])
def test_partition_is_four_matchings_covering_the_torus(hw):
    h, w = hw
    n = h * w
    # brute-force list of the 2N torus edges (a multigraph when a side is 2)
    torus = []
    for r in range(h):
        for c in range(w):
            torus.append(tuple(sorted((r * w + c, r * w + (c + 1) % w))))
            torus.append(tuple(sorted((r * w + c, ((r + 1) % h) * w + c))))
    got = []
    for k in (1, 2, 3, 4):
        f, s = edges(h, w, k)
        assert f.size == n // 2
        # a matching: no pixel twice; every pixel exactly once
        assert sorted(np.concatenate([f, s]).tolist()) == list(range(n))
        got += [tuple(sorted(p)) for p in zip(f.tolist(), s.tolist())]
    assert sorted(got) == sorted(torus)


def test_partition_free_boundary_drops_wrap_edges():
    h, w = 5, 7
    total = 0
    for k in (1, 2, 3, 4):
        f, s = edges(h, w, k, periodic=False)
        for a, b in zip(f.tolist(), s.tolist()):
            ra, ca = divmod(a, w)
            rb, cb = divmod(b, w)
            assert abs(ra - rb) + abs(ca - cb) == 1
        total += f.size
    assert total == h * (w - 1) + (h - 1) * w


# ---------------------------------------------------------------- operators
def test_convolution_matches_fft_and_adjoint():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(12, 10))
    k = rng.random((5, 3))
    np.testing.assert_allclose(operators.conv_periodic(x, k), syn.circular_blur(x, k), atol=1e-13)
    z = rng.normal(size=(12, 10))
    lhs = np.sum(z * operators.conv_periodic(x, k))
    rhs = np.sum(x * operators.conv_periodic_t(z, k))
    assert abs(lhs - rhs) < 1e-12


# ---------------------------------------------------------------- exact 1x2 case
def _exact_pair_moments(y, xi, lam, empty_tau):
    """Moments of p(x1, x2) ~ N(y1; x1, xi) N(y2; x2, xi) exp(-lam|x1 - x2|)
    exp(-empty_tau (x1^2 + x2^2) / 2) by 2-D Gauss-Legendre quadrature on the
    two half-planes x1 > x2 and x1 < x2 (coordinates u = x1 - x2, v = x1 + x2)."""
    sd = math.sqrt(xi)
    nodes, weights = np.polynomial.legendre.leggauss(600)
    v_lo, v_hi = y[0] + y[1] - 16 * sd, y[0] + y[1] + 16 * sd
    u_span = abs(y[0] - y[1]) + 16 * sd
    acc = np.zeros(7)
    for u_lo, u_hi in ((-u_span, 0.0), (0.0, u_span)):
        u = 0.5 * (u_hi - u_lo) * nodes + 0.5 * (u_hi + u_lo)
        wu = 0.5 * (u_hi - u_lo) * weights
        v = 0.5 * (v_hi - v_lo) * nodes + 0.5 * (v_hi + v_lo)
        wv = 0.5 * (v_hi - v_lo) * weights
        U, V = np.meshgrid(u, v, indexing="ij")
        W = np.outer(wu, wv)
        x1, x2 = (V + U) / 2, (V - U) / 2
        logp = (-(y[0] - x1) ** 2 / (2 * xi) - (y[1] - x2) ** 2 / (2 * xi)
                - lam * np.abs(x1 - x2) - empty_tau * (x1 ** 2 + x2 ** 2) / 2)
        p = np.exp(logp) * W
        acc += [p.sum(), (p * x1).sum(), (p * x2).sum(), (p * x1 ** 2).sum(),
                (p * x2 ** 2).sum(), (p * np.abs(x1 - x2)).sum(), (p * (x1 - x2) ** 2).sum()]
    z = acc[0]
    m1, m2 = acc[1] / z, acc[2] / z
    return m1, m2, acc[3] / z - m1 ** 2, acc[4] / z - m2 ** 2, acc[5] / z, acc[6] / z


@pytest.mark.parametrize("y,xi,lam", [((0.3, 0.7), 0.01, 20.0), ((0.9, -0.2), 0.04, 3.0),
                                      ((0.5, 0.52), 0.01, 80.0)])
def test_one_by_two_image_is_exact(y, xi, lam):
    """P2: with a single edge the tilted distribution is the exact posterior and
    the projection is exact, so the EP fixed point has the exact marginals."""
    o = EPOracle("denoise", np.array([y]), xi, lam, 1, 2, periodic=False)
    o.run(80)
    mu, var = o.posterior()
    # sites 2, 3, 4 have no edge here and keep precision 1/var_cap each
    m1, m2, v1, v2, eabs, _ = _exact_pair_moments(y, xi, lam, 3.0 / o.var_cap)
    np.testing.assert_allclose(mu.ravel(), [m1, m2], rtol=1e-8)
    np.testing.assert_allclose(var.ravel(), [v1, v2], rtol=1e-8)
    # EM (Algorithm 2, Option 3): a_u = E|x1 - x2| under the exact posterior
    lam_new = o.em_update()
    assert abs(lam_new - 2.0 / eabs) <= 1e-8 * lam_new


# ---------------------------------------------------------------- mixture priors
def _mixture_quad(mu, s2, omega, v1, v2):
    """Mean and variance of N(u; mu, s2) [omega N(u; 0, v1) + (1 - omega) N(u; 0, v2)]
    by mpmath quadrature of the raw integrand (v2 = 0: the second component is
    delta(u), whose mass (1 - omega) N(0; mu, s2) sits at u = 0).  Each Gaussian
    component's integrals run over u = c + r t, t in (-inf, inf), with c and r
    the centre and width of the product of its two Gaussians: only the placement
    of the quadrature nodes depends on them, the integrand is the raw product.
    The variance is integrated as a central moment, so it does not cancel.  All
    integrands are divided by one common constant (the largest component
    density at its node t = 0): mpmath's tolerance is absolute, and these
    densities can be as small as 1e-55."""
    sd = mp.sqrt(s2)
    comps = [(omega, v1)] + ([(1 - omega, v2)] if v2 > 0 else [])
    grid = [-mp.inf, -12, -6, -3, -1, 0, 1, 3, 6, 12, mp.inf]

    def raw(k, t):
        wk, vk = comps[k]
        c = mp.mpf(mu) * vk / (vk + s2)
        r = mp.sqrt(mp.mpf(vk) * s2 / (vk + s2))
        u = c + r * t
        return u, wk * mp.npdf(u, 0, mp.sqrt(vk)) * mp.npdf(u, mu, sd) * r

    scale = max(raw(k, 0)[1] for k in range(len(comps)))

    def integral(k, g):
        def integrand(t):
            u, fu = raw(k, t)
            return g(u) * fu / scale
        return mp.quad(integrand, grid)

    point = 0 if v2 > 0 else (1 - omega) * mp.npdf(0, mu, sd) / scale
    z = sum(integral(k, lambda u: 1) for k in range(len(comps))) + point
    m = sum(integral(k, lambda u: u) for k in range(len(comps))) / z
    v = (sum(integral(k, lambda u: (u - m) ** 2) for k in range(len(comps))) + point * m ** 2) / z
    return float(m), float(v)


@pytest.mark.parametrize("theta", [(0.3, 0.5, 0.001), (0.8, 4.0, 0.1), (0.05, 0.2, 0.0),
                                   (0.6, 1.0, 0.0)])
def test_mixture_tilted_moments_match_quadrature(theta):
    """The tilted moments of the MoG2-TV (Eq. MoG2_TV_prior) and BG-TV (Eq. BG_TV,
    v2 = 0) edge factors against quadrature, from edges inside the small-gradient
    component to edges far in the tail, to 1e-10 relative (the mean relative to
    the larger of its size and the tilted standard deviation)."""
    from oracle.tilted import gaussian_mixture_tilted
    mp.mp.dps = 30
    for mu in (-3.0, -0.2, 0.0, 1.0, 7.0):
        for s2 in (1e-4, 0.01, 30.0):
            mq, vq = _mixture_quad(mu, s2, *theta)
            mo, vo = gaussian_mixture_tilted(mu, s2, *theta)
            assert abs(mo - mq) <= 1e-10 * max(abs(mq), math.sqrt(vq)), (mu, s2, mo, mq)
            assert abs(vo - vq) <= 1e-10 * vq, (mu, s2, vo, vq)


def test_mixture_prior_with_one_gaussian_component_has_exact_means():
    """With omega = 1 the MoG2-TV factor is the Gaussian N(x_i - x_j; 0, v1), the
    posterior is Gaussian, and the EP fixed point has its exact means (the
    variances of a diagonal approximation on a loopy graph are not exact)."""
    h, w = 4, 6
    rng = np.random.default_rng(1)
    y = rng.random((h, w))
    xi, v1 = 0.05, 0.02
    o = EPOracle("denoise", y, xi, 0.0, h, w, prior="mog2", theta=(1.0, v1, 1.0))
    o.run(300)
    mu, var = o.posterior()
    n = h * w
    prec = np.eye(n) / xi
    for k in (1, 2, 3, 4):
        for a, b in zip(*edges(h, w, k, True)):
            d = np.zeros(n)
            d[a], d[b] = 1.0, -1.0
            prec += np.outer(d, d) / v1
    exact = np.linalg.solve(prec, y.reshape(-1) / xi)
    np.testing.assert_allclose(mu.reshape(-1), exact, rtol=0, atol=1e-12)
    assert np.all(var.reshape(-1) < np.diag(np.linalg.inv(prec)))


def _exact_pair_mixture(y, xi, omega, v1, v2, empty_tau):
    """Exact marginal means and variances of p(x1, x2) ~ N(y1; x1, xi) N(y2; x2, xi)
    exp(-empty_tau (x1^2 + x2^2) / 2) phi(x1 - x2) for phi = omega N(.; 0, v1) +
    (1 - omega) N(.; 0, v2), or (1 - omega) delta(.) when v2 = 0.  Each component
    gives a Gaussian posterior in closed form (for the delta: the line x1 = x2),
    weighted by its evidence."""
    y = np.asarray(y, float)
    b = y / xi
    lap = np.array([[1.0, -1.0], [-1.0, 1.0]])
    comps = []
    for wk, vk in ((omega, v1), (1.0 - omega, v2)):
        if vk > 0:
            a = np.diag([1 / xi + empty_tau] * 2) + lap / vk
            m = np.linalg.solve(a, b)
            logz = (math.log(wk) - 0.5 * math.log(2 * math.pi * vk) - 0.5 * math.log(np.linalg.det(a))
                    + 0.5 * b @ m + math.log(2 * math.pi))
            comps.append((logz, m, np.diag(np.linalg.inv(a))))
        else:
            a = 2 / xi + 2 * empty_tau
            bs = b.sum()
            logz = math.log(wk) - 0.5 * math.log(a) + 0.5 * bs * bs / a + 0.5 * math.log(2 * math.pi)
            comps.append((logz, np.full(2, bs / a), np.full(2, 1 / a)))
    lz = np.array([c[0] for c in comps])
    wts = np.exp(lz - lz.max())
    wts /= wts.sum()
    mean = sum(wts[k] * comps[k][1] for k in range(2))
    var = sum(wts[k] * (comps[k][2] + comps[k][1] ** 2) for k in range(2)) - mean ** 2
    return mean, var


@pytest.mark.parametrize("prior,theta", [("mog2", (0.3, 1.0, 1e-3)), ("mog2", (0.7, 0.5, 0.02)),
                                         ("bg", (0.4, 0.5)), ("bg", (0.8, 2.0))])
@pytest.mark.parametrize("y,xi", [((0.3, 0.7), 0.01), ((0.9, -0.2), 0.04), ((0.5, 0.52), 0.01)])
def test_one_by_two_image_mixture_priors(prior, theta, y, xi):
    """P2 for the MoG2-TV and BG-TV priors (Sec. II-B): with a single edge the
    tilted distribution is the exact posterior, so the EP means are exact.  Where
    the exact marginal variance is below the cavity (likelihood) variance the
    variances are exact too; where the posterior is so bimodal that it is above
    it, the new edge site has a negative variance and the cap of Sec. III-C sets
    its precision to 1/var_cap, leaving the posterior variance of the likelihood
    and the four capped sites."""
    o = EPOracle("denoise", np.array([y]), xi, 0.0, 1, 2, periodic=False, prior=prior, theta=theta)
    o.run(200)
    mu, var = (a.ravel() for a in o.posterior())
    v2 = theta[2] if prior == "mog2" else 0.0
    cap = 1.0 / o.var_cap
    mean, v = _exact_pair_mixture(y, xi, theta[0], theta[1], v2, 3.0 * cap)
    np.testing.assert_allclose(mu, mean, rtol=0, atol=1e-12)
    cavity_var = 1.0 / (1.0 / xi + 3.0 * cap)
    if np.all(v < cavity_var):
        assert np.all(o.tau[1] > 2 * cap)
        np.testing.assert_allclose(var, v, rtol=1e-10)
    else:
        np.testing.assert_array_equal(o.tau[1], cap)
        np.testing.assert_allclose(var, 1.0 / (1.0 / xi + 4.0 * cap), rtol=1e-12)


# ---------------------------------------------------------------- 2x2 loop
def _exact_2x2(y, xi, lam, empty_tau, n=1201, half=9.0):
    """Exact marginal means, variances and E sum|x_i - x_j| of the 2x2 free-boundary
    denoising posterior, p(x) ~ prod_i N(y_i; x_i, xi) exp(-empty_tau x_i^2 / 2)
    prod_edges exp(-lam |x_i - x_j|), whose four edges (V1: 0-1, 2-3; V3: 0-2, 1-3,
    pixels numbered row-major) form the cycle 0-1-3-2-0.  The 4-D integral is a
    trace around the cycle of n x n matrices on one shared trapezoid grid:
    Z = tr(F0 Phi F1 Phi F3 Phi F2 Phi), F_i = diag(node weights x site factors)."""
    sd = math.sqrt(xi)
    g = np.linspace(min(y) - half * sd, max(y) + half * sd, n)
    h = g[1] - g[0]
    w = np.full(n, h)
    w[0] = w[-1] = h / 2
    f = [np.exp(-(g - y[i]) ** 2 / (2 * xi) - empty_tau * g ** 2 / 2) * w for i in range(4)]
    diff = np.abs(g[:, None] - g[None, :])
    phi = np.exp(-lam * diff)
    aphi = diff * phi

    def ring(fs, edge=(phi, phi, phi, phi)):
        m = np.diag(fs[0]) @ edge[0] @ np.diag(fs[1]) @ edge[1] @ np.diag(fs[3]) @ edge[2]
        return float(np.trace(m @ np.diag(fs[2]) @ edge[3]))

    z = ring(f)
    mean, var = np.zeros(4), np.zeros(4)
    for i in range(4):
        f1, f2 = list(f), list(f)
        f1[i], f2[i] = f[i] * g, f[i] * g * g
        mean[i] = ring(f1) / z
        var[i] = ring(f2) / z - mean[i] ** 2
    eabs = sum(ring(f, tuple(aphi if e == k else phi for e in range(4))) for k in range(4)) / z
    return mean, var, eabs


@pytest.mark.parametrize("y,xi,lam", [((0.68, 0.05, 0.92, 0.41), 0.25, 2.0),
                                      ((0.13, 0.77, 0.52, 0.29), 0.04, 8.0),
                                      ((0.85, 0.62, 0.09, 0.48), 0.01, 20.0)])
def test_two_by_two_loop_against_exact_posterior(y, xi, lam):
    """P7: on a 2x2 image with the free boundary the four edges form a loop, so
    the V_k updates interact through the cavities and EP is no longer exact.
    Against the exact posterior (brute-force 4-D quadrature) the EP fixed point
    is close: means within 0.03 posterior standard deviations, variances within
    12%, and the EM statistic a_u of the tilted distributions within 8% of the
    exact E sum|x_i - x_j|.  A sign flip of the tilted mean, exchanged c_i / c_j
    in the projection or a 10% error in the tilted variance each break one of
    these bounds."""
    y = np.asarray(y)
    o = EPOracle("denoise", y.reshape(2, 2), xi, lam, 2, 2, periodic=False)
    o.run(300)
    mu, var = (a.reshape(-1) for a in o.posterior())
    # V2 and V4 have no edge on a free 2x2 grid: those sites stay at 1/var_cap
    mean, v, eabs = _exact_2x2(y, xi, lam, 2.0 / o.var_cap)
    assert np.max(np.abs(mu - mean) / np.sqrt(v)) <= 0.03
    assert np.max(np.abs(var / v - 1.0)) <= 0.12
    assert abs(o.abar / eabs - 1.0) <= 0.08


def test_folded_normal_mean_matches_quadrature():
    from oracle.tilted import folded_normal_mean
    mp.mp.dps = 30
    for m in (-4.0, -0.3, 0.0, 0.01, 2.5):
        for s2 in (1e-6, 0.04, 9.0):
            sd = mp.sqrt(s2)
            q = mp.quad(lambda u: abs(u) * mp.npdf(u, m, sd), [-mp.inf, min(0, m), max(0, m), mp.inf])
            assert abs(folded_normal_mean(m, s2) - float(q)) <= 1e-12 * max(float(q), 1e-300)


@pytest.mark.parametrize("y,xi,lam", [((0.3, 0.7), 0.01, 20.0), ((0.9, -0.2), 0.04, 3.0)])
def test_em_option2_on_one_by_two_image(y, xi, lam):
    """Eq. au (Option 2): on a 1 x 2 image the tilted law of u = x1 - x2 is the
    exact posterior of u, so Q(u) carries its exact mean and variance and a_u is
    the folded-normal mean of N(E u, Var u) from the exact posterior."""
    from oracle.tilted import folded_normal_mean
    o = EPOracle("denoise", np.array([y]), xi, lam, 1, 2, periodic=False)
    o.run(80)
    m1, m2, _, _, _, eu2 = _exact_pair_moments(y, xi, lam, 3.0 / o.var_cap)
    mu_u = m1 - m2
    assert abs(o.em_statistic(2) / folded_normal_mean(mu_u, eu2 - mu_u ** 2) - 1.0) <= 1e-8


def test_em_options_agree_at_lambda_zero():
    """With lam = 0 every prior site stays at the cap, Q(x) has mean y and
    variance 1 / (1/xi + 4/var_cap), and the tilted laws of the edges are the
    Gaussians of their cavities: Options 1, 2 and 3 (Eq. ax, Eq. au,
    Eq. 3rd_alternative_a0) all give sum over edges of E|N(y_i - y_j, c_i + c_j)|,
    with c the cavity variance 1 / (1/xi + 3/var_cap)."""
    from oracle.tilted import folded_normal_mean
    h, w = 6, 8
    y = np.random.default_rng(3).random((h, w))
    xi = 0.02
    o = EPOracle("denoise", y, xi, 0.0, h, w)
    o.run(3)
    yf = y.reshape(-1)
    c = 1.0 / (1.0 / xi + 3.0 / o.var_cap)
    post = 1.0 / (1.0 / xi + 4.0 / o.var_cap)
    ref_tilted = sum(float(np.sum(folded_normal_mean(yf[f] - yf[g], 2 * c))) for f, g in o.edge_lists)
    ref_q = sum(float(np.sum(folded_normal_mean(yf[f] - yf[g], 2 * post))) for f, g in o.edge_lists)
    assert abs(o.em_statistic(3) / ref_tilted - 1) <= 1e-10
    assert abs(o.em_statistic(2) / ref_tilted - 1) <= 1e-10
    assert abs(o.em_statistic(1) / ref_q - 1) <= 1e-10


# ---------------------------------------------------------------- Hadamard operator
def test_paley_ordered_walsh_functions_from_rademacher_products():
    """Sec. II-A (iii): row k of the Paley-ordered Walsh matrix is the product of
    the Rademacher functions r_i(t) = sign(sin(2^i pi t)) over the set bits i of k
    (bit 0 -> r_1), sampled at t = (x + 1/2) / n; the oracle builds it as the
    Sylvester row with the bits of k reversed."""
    for n in (2, 8, 32):
        bits = n.bit_length() - 1
        t = (np.arange(n) + 0.5) / n
        for k in range(n):
            ref = np.ones(n)
            for i in range(bits):
                if k >> i & 1:
                    ref *= np.sign(np.sin(2.0 ** (i + 1) * np.pi * t))
            row = operators.hadamard_matrix(1, n, [k])[0] * 1.0  # M = 1: unscaled
            np.testing.assert_array_equal(row, ref)


def test_hadamard_rows_orthogonal_and_kronecker():
    """All N patterns give sqrt(N) times an orthogonal matrix (H H^T = N/M I with
    M = N), and a 2-D pattern is the outer product of its 1-D row and column
    Walsh functions."""
    h, w = 4, 8
    n = h * w
    H = operators.hadamard_matrix(h, w, range(n)) * math.sqrt(n)
    np.testing.assert_array_equal(H @ H.T, n * np.eye(n))
    rows = operators.hadamard_matrix(1, h, range(h)) * math.sqrt(h)
    cols = operators.hadamard_matrix(1, w, range(w)) * math.sqrt(w)
    for kr in range(h):
        for kc in range(w):
            np.testing.assert_array_equal(H[kr * w + kc], np.outer(rows[kr], cols[kc]).ravel())


# ---------------------------------------------------------------- non-i.i.d. noise
def _noise_plane(n, seed):
    """Noise variances spread over a factor of 20 (seeded)."""
    return 0.005 * np.exp(np.random.default_rng(seed).uniform(0.0, 3.0, n))


def test_diagonal_noise_lambda_zero_closed_forms():
    """Sec. III-C: a diagonal noise covariance enters Eq. tilted_P_1 in place of
    xi I.  With lam = 0 the prior sites stay at the cap: the EP variances are those
    of the Gaussian posterior with precision H^T diag(1/xi) H + 4/var_cap (per
    pixel for denoising, the diagonal of the dense inverse for deconvolution),
    and the mean tends to the weighted least-squares solution (y for denoising,
    H^{-1} y for an invertible blur, whatever the weights)."""
    h, w = 6, 8
    n = h * w
    xi = _noise_plane(n, 1)
    y = np.random.default_rng(2).random((h, w))
    o = EPOracle("denoise", y, xi, 0.0, h, w)
    o.run(30)
    mu, var = (a.reshape(-1) for a in o.posterior())
    ridge = 4.0 / o.var_cap
    np.testing.assert_allclose(var, 1.0 / (1.0 / xi + ridge), rtol=1e-13)
    np.testing.assert_allclose(mu, y.reshape(-1), rtol=1e-9, atol=1e-12)
    k = np.array([[0.02, 0.05, 0.01], [0.04, 0.7, 0.08], [0.03, 0.06, 0.01]])
    o = EPOracle("deconv", y, xi, 0.0, h, w, kernel=k, site0="exact")
    o.run(40)
    mu, var = (a.reshape(-1) for a in o.posterior())
    H = operators.conv_matrix(h, w, k)
    cov = np.linalg.inv(H.T @ np.diag(1.0 / xi) @ H + ridge * np.eye(n))
    np.testing.assert_allclose(var, np.diag(cov), rtol=1e-10)
    np.testing.assert_allclose(mu, np.linalg.solve(H, y.reshape(-1)), rtol=0, atol=1e-6)


def test_diagonal_noise_woodbury_equals_dense_inverse():
    """Compressive sensing with a diagonal noise covariance: the Woodbury form
    (K = diag(xi) + H C H^T) equals the dense inverse of Eq. tilted_P_1."""
    rng = np.random.default_rng(6)
    n, m = 256, 77
    H = rng.standard_normal((m, n)) / math.sqrt(m)
    xi = _noise_plane(m, 7)
    c = rng.uniform(0.5, 2.0, n)
    mv = rng.standard_normal(n)
    o = EPOracle("cs", rng.standard_normal(m), xi, 1.0, 16, 16, A=H, site0="woodbury")
    E, V = o._woodbury(H, c, mv)
    Q = H.T @ np.diag(1.0 / xi) @ H + np.diag(1.0 / c)
    cov = np.linalg.inv(Q)
    np.testing.assert_allclose(V, np.diag(cov), rtol=1e-10)
    np.testing.assert_allclose(E, cov @ (H.T @ (o.y / xi) + mv / c), rtol=1e-9, atol=1e-10)


def test_constant_noise_plane_equals_scalar_noise():
    h, w = 8, 8
    p = syn.denoise_problem(h, w, sigma=0.1, beta=10.0, seed=3)
    a = EPOracle("denoise", p.y, p.xi, p.beta, h, w)
    b = EPOracle("denoise", p.y, np.full(h * w, p.xi), p.beta, h, w)
    a.run(5)
    b.run(5)
    for x, z in zip(a.posterior(), b.posterior()):
        np.testing.assert_allclose(x, z, rtol=1e-14)


# ---------------------------------------------------------------- lam -> 0
def test_lambda_zero_denoise_closed_form():
    """P3: with lam = 0 every prior site sits at the cap, mu = y and
    sigma^2 = 1 / (1/xi + 4/var_cap)."""
    p = syn.denoise_problem(16, 12, seed=2)
    o = EPOracle("denoise", p.y, p.xi, 0.0, 16, 12)
    o.run(30)
    mu, var = o.posterior()
    np.testing.assert_allclose(var, 1.0 / (1.0 / p.xi + 4e-8), rtol=1e-13)
    np.testing.assert_allclose(mu, p.y, rtol=1e-9, atol=1e-12)


def test_lambda_zero_deconv_matches_fft_posterior():
    """P3: with lam = 0 and a periodic blur the q0 update gives the exact
    marginal variances of N(x; ., (H^T H / xi + 4e-8 I)^{-1}), which are the same
    at every pixel: (1/N) sum_f 1 / (|h_f|^2 / xi + 4e-8); the mean tends to the
    least-squares deconvolution."""
    h, w = 8, 10
    k = np.array([[0.02, 0.05, 0.01], [0.04, 0.7, 0.08], [0.03, 0.06, 0.01]])
    rng = np.random.default_rng(11)
    x = rng.random((h, w))
    xi = 1e-3
    y = syn.circular_blur(x, k) + math.sqrt(xi) * rng.normal(size=(h, w))
    o = EPOracle("deconv", y, xi, 0.0, h, w, kernel=k, site0="exact")
    o.run(40)
    mu, var = o.posterior()
    pad = np.zeros((h, w))
    pad[:3, :3] = k
    hf = np.fft.fft2(np.roll(pad, (-1, -1), axis=(0, 1)))
    var_ref = np.mean(1.0 / (np.abs(hf) ** 2 / xi + 4e-8))
    np.testing.assert_allclose(var, var_ref, rtol=1e-10)
    mu_ls = np.real(np.fft.ifft2(np.conj(hf) * np.fft.fft2(y) / np.abs(hf) ** 2))
    np.testing.assert_allclose(mu, mu_ls, rtol=0, atol=1e-6)


# ---------------------------------------------------------------- likelihood site
def test_denoise_site0_is_a_fixed_point():
    """C6: for H = I the q0 update returns (1/xi, y/xi) whatever the cavity."""
    p = syn.denoise_problem(10, 8, seed=5)
    o = EPOracle("denoise", p.y, p.xi, 15.0, 10, 8)
    for _ in range(3):
        for k in (1, 2, 3, 4):
            o.prior_update(k)
        before = (o.tau[0].copy(), o.nu[0].copy())
        o.site0_update()
        np.testing.assert_allclose(o.tau[0], before[0], rtol=1e-13)
        np.testing.assert_allclose(o.nu[0], before[1], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(o.tau[0], 1.0 / p.xi, rtol=1e-13)
        np.testing.assert_allclose(o.nu[0], p.y.ravel() / p.xi, rtol=1e-11, atol=1e-11)


def test_woodbury_equals_dense_inverse():
    """P4: the Woodbury form of Cov_P0 for compressive sensing equals the dense inverse."""
    p = syn.cs_problem(16, 16, m=77, seed=3)
    a = EPOracle("cs", p.y, p.xi, 2.0, 16, 16, A=p.A, site0="exact")
    rng = np.random.default_rng(15)
    c = rng.uniform(0.01, 1.0, size=256)
    m = rng.normal(size=256)
    e_dense, v_dense = a.tilted_p0(c, m)
    a.site0 = "woodbury"
    e_wood, v_wood = a.tilted_p0(c, m)
    np.testing.assert_allclose(e_wood, e_dense, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(v_wood, v_dense, rtol=1e-9)
    # whole runs agree up to the conditioning of the dense N x N solve
    a = EPOracle("cs", p.y, p.xi, 2.0, 16, 16, A=p.A, site0="exact")
    b = EPOracle("cs", p.y, p.xi, 2.0, 16, 16, A=p.A, site0="woodbury")
    a.run(4)
    b.run(4)
    for u, v in zip(a.posterior(), b.posterior()):
        np.testing.assert_allclose(u, v, rtol=1e-4, atol=1e-5)


def test_rbmc_is_exact_for_a_diagonal_precision():
    """With H = I the precision is diagonal, the conditional mean of each pixel
    is zero and the Rao-Blackwellised estimator returns 1/Q_ii exactly; the
    deconvolution route with a 1x1 unit kernel then equals denoising."""
    p = syn.denoise_problem(8, 6, seed=6)
    pr = syn.rbmc_probes(3, 48, 48, seed=1)
    a = EPOracle("deconv", p.y, p.xi, 9.0, 8, 6, kernel=np.ones((1, 1)), site0="rbmc", probes=pr)
    b = EPOracle("denoise", p.y, p.xi, 9.0, 8, 6)
    a.run(6)
    b.run(6)
    for u, v in zip(a.posterior(), b.posterior()):
        np.testing.assert_allclose(u, v, rtol=1e-11)


def test_rbmc_is_unbiased():
    """The RB estimate averaged over many probes approaches diag(Q^{-1})."""
    h, w = 6, 6
    n = h * w
    rng = np.random.default_rng(8)
    k = rng.random((3, 3)) ** 3       # asymmetric, so H^T differs from H
    k /= k.sum()
    y = rng.random((h, w))
    S = 4000
    pr = syn.rbmc_probes(S, n, n, seed=9)
    o = EPOracle("deconv", y, 1e-2, 1.0, h, w, kernel=k, site0="rbmc", probes=pr)
    c = rng.uniform(0.02, 0.5, size=n)
    m = rng.normal(size=n)
    _, v_rb = o.tilted_p0(c, m)
    o.site0 = "exact"
    _, v_ex = o.tilted_p0(c, m)
    # the estimator's spread is at most the spread of 1/Q_ii + (.)^2 terms; use 6 sigma
    rel = np.abs(v_rb / v_ex - 1)
    assert rel.max() < 6.0 / math.sqrt(S) * 2.0
    assert np.all(v_rb >= 1.0 / np.diag(o._operator()[0].T @ o._operator()[0] / 1e-2 + np.diag(1 / c)))


# ---------------------------------------------------------------- symmetry
def _run(y, lam, order=None, kind="denoise", kernel=None, xi=0.01, sweeps=8):
    h, w = y.shape
    o = EPOracle(kind, y, xi, lam, h, w, kernel=kernel)
    for _ in range(sweeps):
        o.sweep(order)
    return o.posterior()


def test_flip_and_transpose_symmetry():
    """P5: flips map each V_k to itself; the transpose swaps V1<->V3 and V2<->V4."""
    rng = np.random.default_rng(12)
    y = rng.random((8, 6))
    base = _run(y, 12.0)
    for f in (lambda a: a[:, ::-1], lambda a: a[::-1, :]):
        got = _run(f(y).copy(), 12.0)
        for u, v in zip(got, base):
            np.testing.assert_allclose(u, f(v), rtol=1e-12)
    got = _run(y.T.copy(), 12.0, order=[3, 4, 1, 2])
    for u, v in zip(got, base):
        np.testing.assert_allclose(u, v.T, rtol=1e-12)


def test_flip_symmetry_deconv_with_mirrored_kernel():
    rng = np.random.default_rng(13)
    y = rng.random((6, 8))
    k = rng.random((3, 3))
    k /= k.sum()
    base = _run(y, 5.0, kind="deconv", kernel=k, xi=1e-3, sweeps=4)
    got = _run(y[:, ::-1].copy(), 5.0, kind="deconv", kernel=k[:, ::-1].copy(), xi=1e-3, sweeps=4)
    for u, v in zip(got, base):
        np.testing.assert_allclose(u, v[:, ::-1], rtol=1e-10)


# ---------------------------------------------------------------- invariants
def test_site_invariants_after_sweeps():
    """P6: every site precision stays >= 1/var_cap; cavities stay proper; a_u > 0."""
    p = syn.denoise_problem(16, 16, seed=14)
    o = EPOracle("denoise", p.y, p.xi, 25.0, 16, 16)
    for _ in range(10):
        abar = o.sweep()
        assert abar > 0
        assert np.all(o.tau[1:] >= 1e-8 * (1 - 1e-15))
        for s in range(5):
            c, _ = o.cavity(s)
            assert np.all(c > 0)


def test_cg_mode_equals_dense_mode():
    """The CG/FFT route for large images gives the dense-solve result."""
    rng = np.random.default_rng(16)
    k = rng.random((3, 5))
    k /= k.sum()
    p = syn.deconv_problem(12, 10, kernel=k, bsnr_db=30.0, seed=17, grf_length=4.0)
    pr = syn.rbmc_probes(3, 120, 120, seed=18)
    a = EPOracle("deconv", p.y, p.xi, 3.0, 12, 10, kernel=k, site0="rbmc", probes=pr)
    b = EPOracle("deconv", p.y, p.xi, 3.0, 12, 10, kernel=k, site0="rbmc_cg", probes=pr)
    a.run(3)
    b.run(3)
    for u, v in zip(a.posterior(), b.posterior()):
        np.testing.assert_allclose(u, v, rtol=1e-8)
