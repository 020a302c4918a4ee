"""Damped parallel EP with the l1-TV prior, and its EM update (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

State (Sec. III-A): five Gaussian sites per pixel, q_{x,0} for the likelihood
and q_{x,k}, k = 1..4, one per matching V_k.  All covariances are diagonal, so
a site is a pair of per-pixel natural parameters: precision tau = 1/Sigma and
precision-times-mean nu = mu / Sigma.  Arrays ``tau`` and ``nu`` have shape
(5, N), row s holding site s.

The global approximation (Eq. Q_x_final) is tau_x = sum_s tau_s,
nu_x = sum_s nu_s, mu_x = nu_x / tau_x, Sigma_x = 1 / tau_x.  The cavity of
site s (Sec. III-B) is the product of the other four sites, i.e. the sums over
s' != s; the oracle recomputes it from the sites every time it needs it.

One sweep (Algorithm 1) updates q_{x,0} and the four q_{x,k}; all edges of one
V_k are updated together ("in parallel").  The readings of the points the
paper leaves open are:

* order: ``"prior_first"`` (default) runs the four V_k updates and then the
  q_{x,0} update, so that the initial q_{x,0} of Algorithm 1 is used;
  ``"q0_first"`` follows the listing literally.  For denoising the two agree
  because the q_{x,0} update returns the site unchanged.
* k order: 1, 2, 3, 4 unless an explicit order is passed per sweep.
* variance cap (Sec. III-C): a new site precision below 1/var_cap (negative or
  larger-than-cap variance) is set to 1/var_cap before the mean is formed.
* damping: natural parameters are mixed, new = a * updated + (1 - a) * old,
  with a the weight on the updated value; applied to every site.
* EM (Sec. IV, Algorithm 2, Option 3, Eq. 3rd_alternative_a0): the statistic
  a_u is the sum over the four V_k of E_{P_k}|u_n| over all edges, taken at the
  tilted distributions of the last sweep, and lam = N / a_u with N the number
  of pixels.  Options 1 (Eq. ax: E|x_i - x_j| under the diagonal Q(x) after the
  sweep) and 2 (Eq. au: E|u_n| under the Gaussian Q(u_n) whose moments were
  matched to P_k(u_n) during the sweep) replace a_u by those sums.
* initialisation (Algorithm 1): mu_{x,0} = y, Sigma_{x,0} = xi I, the other
  sites have zero mean and variance var_cap.  For compressive sensing y has
  length M < N; the oracle uses mu_{x,0} = H^T y.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np
import scipy.linalg

from . import operators
from .partition import edges
from .tilted import folded_normal_mean, gaussian_mixture_tilted, laplace_tilted


def _fft_qmul(hth, inv_c, xi, h, w, v):
    """Q v = H^T H v / xi + diag(1/c) v with the periodic blur applied through the
    FFT (H^T H is circulant with eigenvalues |h_f|^2 = hth)."""
    v2 = np.asarray(v).reshape(h, w)
    return np.real(np.fft.ifft2(hth * np.fft.fft2(v2))).reshape(-1) / xi + inv_c * v2.reshape(-1)


def _fft_cg_solve(job):
    """Q x = b by conjugate gradients to a relative residual of 1e-11 (a module
    function so that a process pool can run it)."""
    from scipy.sparse.linalg import LinearOperator, cg
    hth, inv_c, xi, h, w, b = job
    Q = LinearOperator((h * w, h * w), matvec=lambda v: _fft_qmul(hth, inv_c, xi, h, w, v),
                       dtype=np.float64)
    x, info = cg(Q, b, rtol=1e-11, atol=0.0, maxiter=20000)
    if info != 0:
        raise RuntimeError("oracle CG did not converge")
    return x


class EPOracle:
    """Algorithm 1 / Algorithm 2 in FP64.

    Parameters
    ----------
    kind : "denoise", "deconv" or "cs"
    y : observation, (H, W) for denoise/deconv, (M,) for cs
    xi : noise variance (Eq. likelihood): a scalar (i.i.d. noise), or one variance
        per measurement (length M) for a diagonal noise covariance, which the
        likelihood site takes in place of xi I (Sec. III-C, last sentence of the
        discussion of Eq. tilted_P_1).  The initial site 0 (Algorithm 1) then has
        variance xi_p per pixel when M = N, and the mean of xi for compressive
        sensing.
    lam : TV parameter lambda (Eq. L1_TV)
    height, width : image size
    kernel : blur kernel for "deconv"
    A : M x N sensing matrix for "cs"
    site0 : how the tilted moments of P_0 (Eq. tilted_P_1) are formed.
        "exact": dense inverse of Cov_P0^{-1} (small N only).
        "woodbury": Woodbury identity (cs; H^T H low rank).
        "rbmc": mean by a dense solve, variance by the Rao-Blackwellised
        Monte Carlo estimator with the given fixed probes (deconv).
        "rbmc_cg": the same estimator with every solve done by conjugate
        gradients to a relative residual of 1e-11 and H applied through the FFT
        (periodic convolution is diagonal in the Fourier basis); for images too
        large for dense factorisation (deconv).
    probes : (eps1 (S, M), eps2 (S, N)) standard normals for "rbmc".
    prior : the edge factor phi of Sec. II-B: "l1" (Eq. L1_TV, parameter lam),
        "mog2" (Eq. MoG2_TV_prior, theta = (omega, s1^2, s2^2)) or "bg"
        (Eq. BG_TV, theta = (omega, s^2)).  The EM update (Sec. IV) is defined
        for "l1" only.
    theta : the mixture parameters for "mog2" / "bg".
    periodic_rows : whether the rows wrap (default: periodic); a band of rows cut
        from a torus has wrapping columns and non-wrapping rows.
    count_rows : (lo, hi) or None; the EM statistics take only the edges whose
        first pixel's row is in [lo, hi) (one band's share of a whole image).
    pool : optional executor (e.g. a spawn-context process pool) on which
        "rbmc_cg" runs the 1 + S independent solves of one site-0 update; each
        solve is the same computation as without it, so results do not change.
    """

    def __init__(self, kind: str, y: np.ndarray, xi: float, lam: float,
                 height: int, width: int, kernel: Optional[np.ndarray] = None,
                 A: Optional[np.ndarray] = None, damping: float = 0.5,
                 var_cap: float = 1e8, periodic: bool = True,
                 order: str = "prior_first", site0: str = "exact",
                 probes=None, pool=None, prior: str = "l1", theta=None,
                 periodic_rows=None, count_rows=None):
        if kind not in ("denoise", "deconv", "cs"):
            raise ValueError(kind)
        if prior not in ("l1", "mog2", "bg"):
            raise ValueError(prior)
        self.prior = prior
        if prior == "mog2":
            omega, v1, v2 = (float(t) for t in theta)
            self.mixture = (omega, v1, v2)
        elif prior == "bg":
            omega, v1 = (float(t) for t in theta)
            self.mixture = (omega, v1, 0.0)
        self.kind = kind
        self.height, self.width = int(height), int(width)
        self.n = self.height * self.width
        self.y = np.asarray(y, dtype=np.float64).reshape(-1)
        xi_arr = np.asarray(xi, dtype=np.float64).reshape(-1)
        self.xi_vec = xi_arr if xi_arr.size > 1 else None  # per measurement, or None
        self.xi = float(xi_arr.mean())
        self.lam = float(lam)
        self.kernel = None if kernel is None else np.asarray(kernel, np.float64)
        self.A = None if A is None else np.asarray(A, np.float64)
        self.damping = float(damping)
        self.var_cap = float(var_cap)
        self.periodic = bool(periodic)
        self.order = order
        self.site0 = site0
        self.probes = probes
        self.pool = pool
        self.periodic_rows = self.periodic if periodic_rows is None else bool(periodic_rows)
        self.edge_lists = [edges(self.height, self.width, k, self.periodic, self.periodic_rows)
                           for k in (1, 2, 3, 4)]
        self.count_rows = count_rows
        self.abar = 0.0          # sum of E|u| over the edges of the last sweep
        self.abar_q = 0.0        # the same under the matched Gaussians Q(u_n) (Option 2)
        self._abar_q_sweep = 0.0
        self.n_sweeps = 0
        self.n_capped = 0        # site updates whose precision the cap replaced
        self.init()

    # ------------------------------------------------------------------ state
    def init(self):
        """Initialisation of Algorithm 1 in natural parameters."""
        n = self.n
        self.tau = np.zeros((5, n))
        self.nu = np.zeros((5, n))
        if self.kind == "cs":
            mu0 = self.A.T @ self.y
        else:
            mu0 = self.y.copy()
        xi0 = self.xi if (self.xi_vec is None or self.kind == "cs") else self.xi_vec
        self.tau[0] = 1.0 / xi0
        self.nu[0] = mu0 / xi0
        self.tau[1:] = 1.0 / self.var_cap
        self.nu[1:] = 0.0

    def cavity(self, s: int):
        """Cavity of site s (product of the other sites): (c, m) = variance, mean."""
        others = [t for t in range(5) if t != s]
        tau_c = self.tau[others].sum(axis=0)
        nu_c = self.nu[others].sum(axis=0)
        return 1.0 / tau_c, nu_c / tau_c

    def posterior(self):
        """Eq. Q_x_final: mean and marginal variance of Q(x)."""
        tau_x = self.tau.sum(axis=0)
        nu_x = self.nu.sum(axis=0)
        sigma = 1.0 / tau_x
        mu = sigma * nu_x
        return mu.reshape(self.height, self.width), sigma.reshape(self.height, self.width)

    # ---------------------------------------------------------- site updates
    def _new_site(self, E, Var, c, m):
        """Eq. update_qk_x / Eq. update_q0_x with the variance cap, natural form."""
        tau_new = 1.0 / Var - 1.0 / c
        capped = tau_new < 1.0 / self.var_cap
        self.n_capped += int(np.count_nonzero(capped))
        tau_new = np.where(capped, 1.0 / self.var_cap, tau_new)
        sigma_site = 1.0 / tau_new
        # mu_site = Sigma_site [(Sigma_site^-1 + Sigma_cav^-1) E - Sigma_cav^-1 m]
        mu_site = sigma_site * ((tau_new + 1.0 / c) * E - m / c)
        return tau_new, mu_site * tau_new

    def _damp(self, s: int, idx, tau_new, nu_new):
        a = self.damping
        self.tau[s, idx] = a * tau_new + (1.0 - a) * self.tau[s, idx]
        self.nu[s, idx] = a * nu_new + (1.0 - a) * self.nu[s, idx]

    def prior_update(self, k: int) -> float:
        """Update q_{x,k} and Q(u_k) for all edges of V_k at once; return sum E|u|."""
        first, second = self.edge_lists[k - 1]
        if first.size == 0:
            return 0.0
        c, m = self.cavity(k)
        ci, cj = c[first], c[second]
        mi, mj = m[first], m[second]
        # Eq. marginal_tilted_un
        mu_u = mi - mj
        s2 = ci + cj
        if self.prior == "l1":
            m_bar, S_bar, eabs = laplace_tilted(mu_u, s2, self.lam)
        else:
            m_bar, S_bar = gaussian_mixture_tilted(mu_u, s2, *self.mixture)
            eabs = np.zeros_like(m_bar)  # no EM for the mixture priors (Sec. IV)
        # projection of the edge moments onto (x_i, x_j) (Sec. III-C)
        Ei = mi + (m_bar - mu_u) / s2 * ci
        Ej = mj - (m_bar - mu_u) / s2 * cj
        Vi = ci + (S_bar - s2) / s2 ** 2 * ci ** 2
        Vj = cj + (S_bar - s2) / s2 ** 2 * cj ** 2
        tau_i, nu_i = self._new_site(Ei, Vi, ci, mi)
        tau_j, nu_j = self._new_site(Ej, Vj, cj, mj)
        self._damp(k, first, tau_i, nu_i)
        self._damp(k, second, tau_j, nu_j)
        counted = self._counted(first)
        if self.prior == "l1":
            self._abar_q_sweep += float(np.sum(folded_normal_mean(m_bar, S_bar)[counted]))
        return float(np.sum(eabs[counted]))

    def _counted(self, first):
        """Edges whose first pixel's row is in count_rows (all edges by default)."""
        if self.count_rows is None:
            return slice(None)
        rows = first // self.width
        return (rows >= self.count_rows[0]) & (rows < self.count_rows[1])

    def tilted_p0(self, c: np.ndarray, m: np.ndarray):
        """Mean and marginal variances of P_0 (Eq. tilted_P_1) for cavity (c, m)."""
        xi = self.xi if self.xi_vec is None else self.xi_vec  # per measurement
        if self.kind == "denoise":
            var = 1.0 / (1.0 / xi + 1.0 / c)
            return var * (self.y / xi + m / c), var
        if self.site0 == "rbmc_cg":
            if self.xi_vec is not None:
                raise ValueError("the FFT-based solves assume i.i.d. noise")
            return self._rbmc_cg(c, m)
        H, _ = self._operator()
        if self.site0 == "woodbury":
            return self._woodbury(H, c, m)
        Q = H.T @ (H / np.reshape(xi, (-1, 1))) + np.diag(1.0 / c)
        b = H.T @ (self.y / xi) + m / c
        cho = scipy.linalg.cho_factor(Q, lower=True)
        E = scipy.linalg.cho_solve(cho, b)
        if self.site0 == "exact":
            cov = scipy.linalg.cho_solve(cho, np.eye(self.n))
            return E, np.diag(cov).copy()
        if self.site0 == "rbmc":
            return E, self._rbmc_var(H, Q, cho, c)
        raise ValueError(self.site0)

    def _operator(self):
        """Dense H and H^T y (built once; the convolution from its definition)."""
        if getattr(self, "_H", None) is None:
            if self.kind == "deconv":
                self._H = operators.conv_matrix(self.height, self.width, self.kernel)
                self._Hty = operators.conv_periodic_t(
                    self.y.reshape(self.height, self.width), self.kernel).reshape(-1)
            else:
                self._H = self.A
                self._Hty = self.A.T @ self.y
        return self._H, self._Hty

    def _rbmc_var(self, H, Q, cho, c):
        """Rao-Blackwellised Monte Carlo estimate of diag(Q^{-1}).

        Samples z_s ~ N(0, Q^{-1}) are drawn by perturbation: z_s solves
        Q z_s = H^T (eps1_s / sqrt(xi)) + eps2_s / sqrt(c), whose right-hand side has
        covariance H^T diag(1/xi) H + diag(1/c) = Q.  For each pixel, x_i given the
        other pixels is Gaussian with variance 1/Q_ii and mean
        -(1/Q_ii) sum_{j != i} Q_ij z_j, so
        Var_i = 1/Q_ii + (1/S) sum_s ((sum_{j != i} Q_ij z_{s,j}) / Q_ii)^2.
        """
        eps1, eps2 = self.probes
        S = eps1.shape[0]
        qdiag = np.diag(Q).copy()
        acc = np.zeros(self.n)
        for s in range(S):
            xi = self.xi if self.xi_vec is None else self.xi_vec
            w = H.T @ (eps1[s] / np.sqrt(xi)) + eps2[s] / np.sqrt(c)
            z = scipy.linalg.cho_solve(cho, w)
            off = Q @ z - qdiag * z
            acc += (off / qdiag) ** 2
        return 1.0 / qdiag + acc / S

    def _rbmc_cg(self, c, m):
        """Site-0 moments with CG solves; same estimator as :meth:`_rbmc_var`."""
        h, w = self.height, self.width
        kh, kw = self.kernel.shape
        pad = np.zeros((h, w))
        pad[:kh, :kw] = self.kernel
        hf = np.fft.fft2(np.roll(pad, (-(kh // 2), -(kw // 2)), axis=(0, 1)))
        hth = np.abs(hf) ** 2
        inv_c = 1.0 / c

        def ht(v):
            return np.real(np.fft.ifft2(np.conj(hf) * np.fft.fft2(v.reshape(h, w)))).reshape(-1)

        eps1, eps2 = self.probes
        S = eps1.shape[0]
        rhs = [ht(self.y) / self.xi + m / c]
        rhs += [ht(eps1[s]) / math.sqrt(self.xi) + eps2[s] / np.sqrt(c) for s in range(S)]
        jobs = [(hth, inv_c, self.xi, h, w, b) for b in rhs]
        sols = list(self.pool.map(_fft_cg_solve, jobs)) if self.pool else [_fft_cg_solve(j) for j in jobs]
        E = sols[0]
        qdiag = np.sum(self.kernel ** 2) / self.xi + inv_c
        acc = np.zeros(self.n)
        for s in range(S):
            z = sols[1 + s]
            off = _fft_qmul(hth, inv_c, self.xi, h, w, z) - qdiag * z
            acc += (off / qdiag) ** 2
        return E, 1.0 / qdiag + acc / S

    def _woodbury(self, H, c, m):
        """Cov_P0 = C - C H^T (xi I + H C H^T)^{-1} H C with C = diag(c)."""
        xi = self.xi if self.xi_vec is None else self.xi_vec
        K = np.diag(np.broadcast_to(xi, (H.shape[0],)).astype(np.float64)) + (H * c[None, :]) @ H.T
        cho = scipy.linalg.cho_factor(K, lower=True)
        KinvH = scipy.linalg.cho_solve(cho, H)
        var = c - c * c * np.einsum("mi,mi->i", H, KinvH)
        E = m + c * (H.T @ scipy.linalg.cho_solve(cho, self.y - H @ m))
        return E, var

    def site0_update(self):
        """Update q_{x,0} (Eq. tilted_P_1 then Eq. update_q0_x)."""
        c, m = self.cavity(0)
        E, Var = self.tilted_p0(c, m)
        tau_new, nu_new = self._new_site(E, Var, c, m)
        self._damp(0, slice(None), tau_new, nu_new)

    # ------------------------------------------------------------ algorithms
    def sweep(self, k_order: Optional[Sequence[int]] = None) -> float:
        """One iteration of Algorithm 1; returns a_u of this sweep."""
        order = list(k_order) if k_order is not None else [1, 2, 3, 4]
        if sorted(order) != [1, 2, 3, 4]:
            raise ValueError("k_order must be a permutation of 1..4")
        abar = 0.0
        self._abar_q_sweep = 0.0
        if self.order == "q0_first":
            self.site0_update()
        for k in order:
            abar += self.prior_update(k)
        if self.order == "prior_first":
            self.site0_update()
        self.abar = abar
        self.abar_q = self._abar_q_sweep
        self.n_sweeps += 1
        return abar

    def em_statistic(self, option: int = 3) -> float:
        """The approximation of a_0 (Eq. a_0) used by the M-step (Sec. IV):
        option 1 = a_x (Eq. ax), 2 = a_u (Eq. au), 3 = abar_u (Eq. 3rd_alternative_a0)."""
        if option == 3:
            return self.abar
        if option == 2:
            return self.abar_q
        if option == 1:
            mu, var = (a.reshape(-1) for a in self.posterior())
            total = 0.0
            for first, second in self.edge_lists:
                f = folded_normal_mean(mu[first] - mu[second], var[first] + var[second])
                total += float(np.sum(f[self._counted(first)]))
            return total
        raise ValueError(option)

    def em_update(self, option: int = 3) -> float:
        """M-step of Algorithm 2: lam = N / a with a from em_statistic(option)."""
        if self.prior != "l1":
            raise ValueError("EM is defined for the l1-TV prior only (Sec. IV)")
        self.lam = self.n / self.em_statistic(option)
        return self.lam

    def run(self, n_sweeps: int, em_every: int = 0, k_orders=None, em_option: int = 3):
        """n_sweeps sweeps; with em_every > 0, lam is updated after every
        em_every-th sweep.  Returns the list of lam values after each update."""
        lams = []
        for t in range(n_sweeps):
            self.sweep(None if k_orders is None else k_orders[t])
            if em_every and (t + 1) % em_every == 0:
                lams.append(self.em_update(em_option))
        return lams

    def ep_em(self, n_em: int, max_sweeps: int, tol: float, em_option: int = 3):
        """Algorithm 2 with Algorithm 1 run to convergence inside every EM
        iteration (the StopRule is read as: the largest change of a posterior
        mean in one sweep is at most tol times the largest |posterior mean|, or
        max_sweeps sweeps), then the M-step.  Returns the lam after each
        iteration and the sweeps of each inner run."""
        lams, sweeps = [], []
        for _ in range(n_em):
            prev, _ = self.posterior()
            for s in range(max_sweeps):
                self.sweep()
                cur, _ = self.posterior()
                done = float(np.max(np.abs(cur - prev))) <= tol * float(np.max(np.abs(cur)))
                prev = cur
                if done:
                    break
            sweeps.append(s + 1)
            lams.append(self.em_update(em_option))
        return lams, sweeps
