"""Pins of the FP64 oracle against things other than itself: published known-answer
vectors, closed forms written independently (Student-t predictive, numerical
quadrature, Beta-binomial), distribution tests against scipy, exact transition
probabilities computed with independent samplers, and invariants.

A plausible slip in the oracle -- a dropped term in a marginal likelihood, a wrong
Bartlett degree of freedom, a transposed precision factor, a wrong Gumbel sign, an
off-by-one in the Hastings ratios -- fails at least one of these."""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- random streams

def test_philox_known_answer_vectors(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_uniform_conversion_endpoints(oracle_mod):
    assert O.u01(0, 0) == 2.0 ** -53
    assert O.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert 0.0 < O.u01(0, 0) < O.u01(1 << 6, 0) < O.u01(0xFFFFFFFF, 0xFFFFFFFF) < 1.0
    assert O.u01_f32(0) == np.float32(2.0 ** -24)
    assert O.u01_f32(0xFFFFFFFF) == np.float32(1.0 - 2.0 ** -24)
    # the reduced-precision uniform uses the leading bits of the same word
    a = 0x9ABCDEF1
    assert abs(O.u01(a, 0x12345678) - O.u01_f32(a)) < 2.0 ** -22


def test_normal_stream_is_standard_normal(oracle_mod):
    z = np.array([O.normal_variate(11, 3, 0, c0, 4, 1000, q) for c0 in range(200) for q in range(100)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # Box-Muller pairs (even q, odd q) are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 0.03


@pytest.mark.parametrize("shape", [0.3, 1.0, 2.5, 17.0, 900.0])
def test_gamma_variates_match_gamma_distribution(oracle_mod, shape):
    g = np.exp([O.log_gamma_variate(5, 1, 0, c0, 2, 0, shape) for c0 in range(6000)])
    assert stats.kstest(g, stats.gamma(shape).cdf).pvalue > 1e-3
    assert abs(g.mean() - shape) < 5 * math.sqrt(shape / g.size)


# ------------------------------------------------------------ marginal likelihoods

def _niw(d, seed=0, **kw):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d))
    psi0 = A @ A.T + d * np.eye(d)
    m0 = rng.standard_normal(d)
    o = O.Oracle(O.NIW, d, 8, 2.0, kappa0=0.7, m0=m0, nu0=d + 1.5, psi0=psi0, **kw)
    return o, m0, psi0


def test_niw_marginal_obeys_student_t_chain_rule(oracle_mod):
    """log f(C + x) - log f(C) must equal the posterior-predictive Student-t density
    (Murphy, 'Conjugate Bayesian analysis of the Gaussian distribution', 2007, Eq. 258)."""
    d = 3
    o, m0, psi0 = _niw(d)
    X = np.random.default_rng(1).standard_normal((12, d)) * 2 + 1
    for m in range(0, 11):
        C, x = X[:m], X[m]
        lhs = o.log_marginal_points(X[: m + 1]) - (o.log_marginal_points(C) if m else 0.0)
        kn, nun = 0.7 + m, d + 1.5 + m
        xbar = C.mean(0) if m else np.zeros(d)
        S = (C - xbar).T @ (C - xbar) if m else np.zeros((d, d))
        mn = (0.7 * m0 + m * xbar) / kn
        psin = psi0 + S + (0.7 * m / kn) * np.outer(xbar - m0, xbar - m0)
        df = nun - d + 1
        rhs = stats.multivariate_t(loc=mn, shape=psin * (kn + 1) / (kn * df), df=df).logpdf(x)
        assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(rhs)), (m, lhs, rhs)


def test_niw_marginal_d1_matches_quadrature(oracle_mod):
    """d=1: NIW = N(mu; m0, s2/kappa0) InvGamma(s2; nu0/2, psi0/2); integrate the
    likelihood numerically over (mu, log s2)."""
    x = np.array([0.3, -1.2, 2.1, 0.8])
    k0, m0, nu0, psi0 = 1.3, 0.4, 3.0, 2.0
    o = O.Oracle(O.NIW, 1, 4, 1.0, kappa0=k0, m0=[m0], nu0=nu0, psi0=[[psi0]])
    L = o.log_marginal_points(x.reshape(-1, 1))

    # composite Simpson rule on a fine grid (the integrand is smooth and negligible
    # outside the box)
    mu = np.linspace(-60.0, 60.0, 4001)
    ls2 = np.linspace(-10.0, 14.0, 1601)
    M, LS = np.meshgrid(mu, ls2, indexing="ij")
    S2 = np.exp(LS)
    lp = stats.invgamma(nu0 / 2, scale=psi0 / 2).logpdf(S2) + stats.norm(m0, np.sqrt(S2 / k0)).logpdf(M)
    for xi in x:
        lp = lp + stats.norm(M, np.sqrt(S2)).logpdf(xi)
    f = np.exp(lp - L) * S2  # Jacobian of s2 = exp(ls2); scaled by exp(-L)
    val = integrate.simpson(integrate.simpson(f, x=ls2, axis=1), x=mu)
    assert abs(val - 1.0) < 1e-6, val


def test_dirichlet_multinomial_marginal_matches_integrals(oracle_mod):
    # d=2: Beta-binomial sequence probability, integrated numerically over theta
    o2 = O.Oracle(O.DIRICHLET, 2, 4, 1.0, beta=[0.7, 1.9])
    a, b = 7.0, 4.0
    val, _ = integrate.quad(lambda t: t ** a * (1 - t) ** b * stats.beta(0.7, 1.9).pdf(t), 0, 1, epsabs=1e-14, epsrel=1e-12)
    assert abs(o2.dirmult_log_marginal([a, b]) - math.log(val)) < 1e-8
    # d=3: integrate over the simplex
    beta = np.array([1.5, 0.8, 2.2])
    o3 = O.Oracle(O.DIRICHLET, 3, 4, 1.0, beta=beta)
    c = np.array([3.0, 1.0, 2.0])
    dist = stats.dirichlet(beta)

    def f(t2, t1):
        t3 = 1 - t1 - t2
        if t3 <= 0:
            return 0.0
        return t1 ** c[0] * t2 ** c[1] * t3 ** c[2] * dist.pdf([t1, t2, t3])

    val, _ = integrate.dblquad(f, 0, 1, 0, lambda t1: 1 - t1, epsabs=1e-13, epsrel=1e-10)
    assert abs(o3.dirmult_log_marginal(c) - math.log(val)) < 1e-6


# --------------------------------------------------------------- posterior draws

def test_niw_draw_moments(oracle_mod):
    """Lambda ~ Wishart(nu_n, Psi_n^-1): E[Lambda] = nu_n Psi_n^-1,
    Var(Lambda_ij) = nu_n (S_ij^2 + S_ii S_jj), S = Psi_n^-1; E[mu] = m_n,
    Cov(mu) = Psi_n / ((nu_n - d - 1) kappa_n)."""
    d = 3
    o, _, _ = _niw(d)
    rng = np.random.default_rng(4)
    A = rng.standard_normal((d, d))
    psin = A @ A.T + np.eye(d)
    mn = rng.standard_normal(d)
    kn, nun = 5.0, 9.5
    R = 6000
    Ls, mus = np.empty((R, d, d)), np.empty((R, d))
    for r in range(R):
        W, mu, ld = o.niw_draw(99, r, 7, kn, mn, nun, psin)
        assert np.allclose(np.tril(W, -1), 0.0) and np.all(np.diag(W) > 0)
        assert abs(ld - np.log(np.diag(W)).sum()) < 1e-12
        Ls[r] = W @ W.T
        mus[r] = mu
    S = np.linalg.inv(psin)
    se = np.sqrt(nun * (S ** 2 + np.outer(np.diag(S), np.diag(S))) / R)
    assert np.all(np.abs(Ls.mean(0) - nun * S) < 5 * se)
    cov_mu = psin / ((nun - d - 1) * kn)
    assert np.all(np.abs(mus.mean(0) - mn) < 5 * np.sqrt(np.diag(cov_mu) / R))
    emp = np.cov(mus.T)
    assert np.all(np.abs(emp - cov_mu) < 0.12 * np.sqrt(np.outer(np.diag(cov_mu), np.diag(cov_mu))))


def test_dirichlet_draw_moments(oracle_mod):
    beta = np.array([0.5, 1.0, 3.0, 0.2])
    o = O.Oracle(O.DIRICHLET, 4, 4, 1.0, beta=beta)
    counts = np.array([2.0, 0.0, 7.0, 1.0])
    R = 6000
    th = np.exp([o.dirichlet_draw(3, r, 1, counts) for r in range(R)])
    a = beta + counts
    m = a / a.sum()
    assert np.allclose(th.sum(1), 1.0, atol=1e-12)
    var = m * (1 - m) / (a.sum() + 1)
    assert np.all(np.abs(th.mean(0) - m) < 5 * np.sqrt(var / R))


# ---------------------------------------------------------- restricted Gibbs step

def _gauss_logpdf(x, mu, W):
    Sigma = np.linalg.inv(W @ W.T)
    return stats.multivariate_normal(mu, Sigma).logpdf(x)


def test_label_step_is_exact_categorical_draw(oracle_mod):
    """Steps (e), (f): Gumbel-max frequencies against the normalised
    pi_k N(x; mu_k, Sigma_k) (chi-square per point)."""
    rng = np.random.default_rng(5)
    d, K, N = 2, 3, 4
    X = np.array([[0.0, 0.0], [1.0, 0.5], [-0.5, 1.0], [0.2, -0.8]])
    o = O.Oracle(O.NIW, d, 8, 3.0, nu0=3.0)
    o.set_data(X)
    o.set_state(K, np.array([0, 1, 2, 0], np.int32), np.array([0, 1, 0, 1], np.uint8))
    o.draw_params(17)
    p = o.params()
    R = 20000
    Z = np.empty((R, N), np.int32)
    ZB = np.empty((R, N), np.uint8)
    for t in range(R):
        Z[t], ZB[t] = o.label_probe(17, t)
    for i in range(N):
        lp = np.array([p["logw"][3 * k] + _gauss_logpdf(X[i], p["mu"][3 * k], p["W"][3 * k]) for k in range(K)])
        pr = np.exp(lp - lp.max())
        pr /= pr.sum()
        cnt = np.bincount(Z[:, i], minlength=K)
        assert stats.chisquare(cnt, pr * R).pvalue > 1e-4
        for k in range(K):  # sub-cluster label given the cluster label
            sel = Z[:, i] == k
            if sel.sum() < 200:
                continue
            lq = np.array([p["logw"][3 * k + 1 + h] + _gauss_logpdf(X[i], p["mu"][3 * k + 1 + h], p["W"][3 * k + 1 + h]) for h in range(2)])
            q = np.exp(lq - lq.max())
            q /= q.sum()
            c = np.bincount(ZB[sel, i], minlength=2)
            assert stats.chisquare(c, q * sel.sum()).pvalue > 1e-4


def _compact(z):
    used = sorted(set(z))
    m = {k: i for i, k in enumerate(used)}
    return tuple(m[k] for k in z)


def test_restricted_step_transition_kernel(oracle_mod):
    """One sweep of steps (a)-(f) from a fixed state, against the exact transition
    probabilities P(z', zbar' | z, zbar) integrated by Monte Carlo with independent
    samplers (numpy Dirichlet, scipy inverse-Wishart) over the conditional posterior
    of (pi, pibar, theta, thetabar)."""
    d, K = 1, 2
    X = np.array([[-1.0], [0.2], [1.5]])
    N = X.shape[0]
    z0 = np.array([0, 0, 1], np.int32)
    zb0 = np.array([0, 1, 0], np.uint8)
    alpha, k0, m0, nu0, psi0 = 1.5, 0.8, 0.0, 2.5, 1.2
    o = O.Oracle(O.NIW, d, 8, alpha, kappa0=k0, m0=[m0], nu0=nu0, psi0=[[psi0]], burn_out=10 ** 6)
    o.set_data(X)
    R = 30000
    counts = {}
    for r in range(R):
        o.set_state(K, z0, zb0)
        o.sweep(1, 1000 + r, mask=O.MASK_PARAMS | O.MASK_LABELS)
        z, zb = o.labels()
        key = (tuple(int(v) for v in z), tuple(int(v) for v in zb))
        counts[key] = counts.get(key, 0) + 1

    # exact kernel by Monte Carlo over the conditional posterior (independent code)
    rng = np.random.default_rng(123)
    M = 200000

    def post_draw(idx):
        n = len(idx)
        xs = X[idx, 0]
        kn, nun = k0 + n, nu0 + n
        xbar = xs.mean() if n else 0.0
        mn = (k0 * m0 + n * xbar) / kn
        psin = psi0 + ((xs - xbar) ** 2).sum() + (k0 * n / kn) * (xbar - m0) ** 2
        s2 = stats.invgamma(nun / 2, scale=psin / 2).rvs(size=M, random_state=rng)
        mu = mn + rng.standard_normal(M) * np.sqrt(s2 / kn)
        return mu, s2

    Nk = [int((z0 == k).sum()) for k in range(K)]
    pi = rng.dirichlet(Nk + [alpha], size=M)[:, :K]
    theta = [post_draw(np.nonzero(z0 == k)[0]) for k in range(K)]
    sub = {}
    pib = []
    for k in range(K):
        nl = int(((z0 == k) & (zb0 == 0)).sum())
        nr = int(((z0 == k) & (zb0 == 1)).sum())
        pib.append(rng.dirichlet([nl + alpha / 2, nr + alpha / 2], size=M))
        for h in range(2):
            sub[(k, h)] = post_draw(np.nonzero((z0 == k) & (zb0 == h))[0])
    # per point: P(z_i = k) and P(zbar_i = h | z_i = k), per Monte Carlo draw
    pz = np.empty((M, N, K))
    pzb = np.empty((M, N, K, 2))
    for i in range(N):
        lw = np.stack([np.log(pi[:, k]) + stats.norm(theta[k][0], np.sqrt(theta[k][1])).logpdf(X[i, 0]) for k in range(K)], 1)
        lw -= lw.max(1, keepdims=True)
        w = np.exp(lw)
        pz[:, i] = w / w.sum(1, keepdims=True)
        for k in range(K):
            lv = np.stack([np.log(pib[k][:, h]) + stats.norm(sub[(k, h)][0], np.sqrt(sub[(k, h)][1])).logpdf(X[i, 0]) for h in range(2)], 1)
            lv -= lv.max(1, keepdims=True)
            v = np.exp(lv)
            pzb[:, i, k] = v / v.sum(1, keepdims=True)
    exact = {}
    import itertools
    for zz in itertools.product(range(K), repeat=N):
        for bb in itertools.product(range(2), repeat=N):
            pr = np.ones(M)
            for i in range(N):
                pr = pr * pz[:, i, zz[i]] * pzb[:, i, zz[i], bb[i]]
            key = (_compact(zz), bb)
            exact[key] = exact.get(key, 0.0) + pr.mean()
    keys = sorted(exact)
    obs = np.array([counts.get(k, 0) for k in keys], float)
    exp_ = np.array([exact[k] for k in keys]) * R
    assert abs(sum(exact.values()) - 1.0) < 1e-9
    assert sum(counts.get(k, 0) for k in keys) == R
    keep = exp_ > 5
    chi = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum() + (obs[~keep].sum() - exp_[~keep].sum()) ** 2 / max(exp_[~keep].sum(), 1e-9)
    df = keep.sum()
    assert stats.chi2.sf(chi, df) > 1e-4, (chi, df)


# ----------------------------------------------------------------- split / merge

def _student_t_log_marginal(X, k0, m0, nu0, psi0):
    """f_x(C) of d=1 points by the chain rule of Student-t predictives (independent
    of the oracle's closed form)."""
    L = 0.0
    for m in range(len(X)):
        C = X[:m]
        kn, nun = k0 + m, nu0 + m
        xbar = C.mean() if m else 0.0
        S = ((C - xbar) ** 2).sum() if m else 0.0
        mn = (k0 * m0 + m * xbar) / kn
        psin = psi0 + S + (k0 * m / kn) * (xbar - m0) ** 2
        df = nun
        L += stats.t(df, loc=mn, scale=math.sqrt(psin * (kn + 1) / (kn * df))).logpdf(X[m])
    return L


def test_split_acceptance_rate_matches_hastings_ratio(oracle_mod):
    """Eq. sample_splits: P(accept) = min(1, H_split) with
    H = alpha Gamma(N_l) f(C_l) Gamma(N_r) f(C_r) / (Gamma(N) f(C))."""
    X = np.array([-0.6, -0.3, 0.1, 0.5, 0.9, 1.2])
    alpha, k0, m0, nu0, psi0 = 0.8, 0.5, 0.0, 2.0, 1.0
    zb = np.array([0, 0, 0, 1, 1, 1], np.uint8)
    Lf = lambda v: _student_t_log_marginal(v, k0, m0, nu0, psi0)
    lH = math.log(alpha) + math.lgamma(3) + Lf(X[:3]) + math.lgamma(3) + Lf(X[3:]) - math.lgamma(6) - Lf(X)
    H = min(1.0, math.exp(lH))
    assert 0.05 < H < 0.95, H  # a borderline case, so the rate is informative
    o = O.Oracle(O.NIW, 1, 8, alpha, kappa0=k0, m0=[m0], nu0=nu0, psi0=[[psi0]], burn_out=0)
    o.set_data(X.reshape(-1, 1))
    R = 6000
    acc = 0
    for r in range(R):
        o.set_state(1, np.zeros(6, np.int32), zb)
        o.sweep(1, 5000 + r, mask=O.MASK_SPLITMERGE)
        acc += o.K == 2
    assert abs(acc / R - H) < 5 * math.sqrt(H * (1 - H) / R), (acc / R, H)


def test_merge_acceptance_rate_matches_hastings_ratio(oracle_mod):
    """Eq. sample_merges, including the Gamma(alpha)/Gamma(alpha+N) and
    Gamma(alpha/2 + N_k) terms."""
    X = np.array([-0.2, 0.0, 0.3, 0.5, 0.6, 0.8, 1.0])
    alpha, k0, m0, nu0, psi0 = 1.3, 0.5, 0.0, 2.0, 2.0
    z = np.array([0, 0, 0, 1, 1, 1, 1], np.int32)
    Lf = lambda v: _student_t_log_marginal(v, k0, m0, nu0, psi0)
    n1, n2 = 3, 4
    lg = math.lgamma
    lH = (lg(n1 + n2) - math.log(alpha) - lg(n1) - lg(n2) + Lf(X) - Lf(X[:3]) - Lf(X[3:])
          + lg(alpha) - lg(alpha + n1 + n2) + lg(alpha / 2 + n1) + lg(alpha / 2 + n2) - 2 * lg(alpha / 2))
    H = min(1.0, math.exp(lH))
    assert 0.05 < H < 0.95, H
    # burn_out large: no split is proposed, so the only move is the merge
    o = O.Oracle(O.NIW, 1, 8, alpha, kappa0=k0, m0=[m0], nu0=nu0, psi0=[[psi0]], burn_out=10 ** 6)
    o.set_data(X.reshape(-1, 1))
    R = 6000
    acc = 0
    for r in range(R):
        o.set_state(2, z, np.zeros(7, np.uint8))
        o.sweep(1, 9000 + r, mask=O.MASK_SPLITMERGE)
        if o.K == 1:
            acc += 1
            _, zb = o.labels()
            assert list(zb) == [0, 0, 0, 1, 1, 1, 1]  # the old clusters become sub-clusters l, r
    assert abs(acc / R - H) < 5 * math.sqrt(H * (1 - H) / R), (acc / R, H)


# ------------------------------------------------- multinomial / Dirichlet branch

def _multinomial_logpmf(x, logtheta):
    """log Multinomial(x; sum x, theta) by scipy (includes the multinomial coefficient,
    which is the same for every cluster and cancels in every normalised probability)."""
    th = np.exp(np.asarray(logtheta, float))
    th = th / th.sum()
    return stats.multinomial(int(np.sum(x)), th).logpmf(np.asarray(x, int))


def test_label_step_is_exact_categorical_draw_dirichlet(oracle_mod):
    """Steps (e), (f) with the Dirichlet prior: Gumbel-max frequencies against the
    normalised pi_k Mult(x_i; theta_k) computed with scipy's multinomial pmf from the
    drawn parameters, per point, and the sub-label frequencies given each cluster label
    against pibar_kh Mult(x_i; theta_kh).  A slip in the multinomial score (theta in
    place of log theta, a wrong slot, a dropped weight) fails one of the chi-squares."""
    X = np.array([[2.0, 0.0, 1.0], [0.0, 2.0, 1.0], [1.0, 1.0, 1.0], [0.0, 0.0, 3.0]])
    N, d, K = X.shape[0], 3, 3
    o = O.Oracle(O.DIRICHLET, d, 8, 2.0, beta=np.array([1.0, 0.7, 1.3]))
    o.set_data(X)
    o.set_state(K, np.array([0, 1, 2, 0], np.int32), np.array([0, 1, 0, 1], np.uint8))
    o.draw_params(23)
    p = o.params()
    R = 20000
    Z = np.empty((R, N), np.int32)
    ZB = np.empty((R, N), np.uint8)
    for t in range(R):
        Z[t], ZB[t] = o.label_probe(23, t)
    informative = 0
    for i in range(N):
        lp = np.array([p["logw"][3 * k] + _multinomial_logpmf(X[i], p["logtheta"][3 * k]) for k in range(K)])
        pr = np.exp(lp - lp.max())
        pr /= pr.sum()
        informative += (pr > 0.05).sum() >= 2
        cnt = np.bincount(Z[:, i], minlength=K)
        assert stats.chisquare(cnt, pr * R).pvalue > 1e-4, (i, cnt, pr * R)
        for k in range(K):
            sel = Z[:, i] == k
            if sel.sum() < 200:
                continue
            lq = np.array([p["logw"][3 * k + 1 + h] + _multinomial_logpmf(X[i], p["logtheta"][3 * k + 1 + h])
                           for h in range(2)])
            q = np.exp(lq - lq.max())
            q /= q.sum()
            c = np.bincount(ZB[sel, i], minlength=2)
            assert stats.chisquare(c, q * sel.sum()).pvalue > 1e-4, (i, k, c, q * sel.sum())
    assert informative >= 2  # the draws are not all near-certain


def _beta_binomial_log_marginal(C, b1, b2):
    """f_x(C) of two-category count vectors without the multinomial coefficients: the
    Beta integral of prod_i theta^{a_i} (1 - theta)^{b_i} against Beta(b1, b2)."""
    from scipy.special import betaln

    C = np.asarray(C, float).reshape(-1, 2)
    return betaln(b1 + C[:, 0].sum(), b2 + C[:, 1].sum()) - betaln(b1, b2)


# Twelve two-category count vectors in three clusters of four, with sub-labels; chosen
# so that every split and merge of the three clusters is accepted with a probability
# near one half (each Hastings ratio is asserted to lie in (0.2, 0.8)).
_PLUMB_X = np.array([[2, 1], [0, 3], [1, 2], [0, 3], [0, 3], [0, 3], [1, 2], [2, 1], [0, 3], [1, 2], [2, 1], [0, 3]],
                    float)
_PLUMB_Z = np.repeat(np.arange(3), 4).astype(np.int32)
_PLUMB_ZB = np.array([1, 0, 1, 0, 0, 0, 1, 1, 1, 0, 1, 1], np.uint8)
_PLUMB_ALPHA, _PLUMB_B = 3.2, (2.16, 0.83)


def _plumb_ratios(X, z, zb, alpha, b1, b2, K):
    lg = math.lgamma
    Lf = lambda sel: _beta_binomial_log_marginal(X[sel], b1, b2)
    ps = []
    for k in range(K):  # Eq. sample_splits
        s = z == k
        l, r = s & (zb == 0), s & (zb == 1)
        nl, nr, n = l.sum(), r.sum(), s.sum()
        lH = math.log(alpha) + lg(nl) + Lf(l) + lg(nr) + Lf(r) - lg(n) - Lf(s)
        ps.append(min(1.0, math.exp(lH)))
    pm = {}
    for k1 in range(K):  # Eq. sample_merges
        for k2 in range(k1 + 1, K):
            s1, s2 = z == k1, z == k2
            n1, n2 = s1.sum(), s2.sum()
            lH = (lg(n1 + n2) - math.log(alpha) - lg(n1) - lg(n2) + Lf(s1 | s2) - Lf(s1) - Lf(s2) + lg(alpha)
                  - lg(alpha + n1 + n2) + lg(alpha / 2 + n1) + lg(alpha / 2 + n2) - 2 * lg(alpha / 2))
            pm[(k1, k2)] = min(1.0, math.exp(lH))
    return ps, pm


def test_split_acceptance_rate_matches_hastings_ratio_dirichlet(oracle_mod):
    """Eq. sample_splits with the Dirichlet prior: P(accept) = min(1, H_split), H from
    Beta-binomial marginals (scipy betaln, independent of the oracle's lgamma sums)."""
    X, zb = _PLUMB_X[:4], _PLUMB_ZB[:4]
    b1, b2 = _PLUMB_B
    ps, _ = _plumb_ratios(X, np.zeros(4, np.int32), zb, _PLUMB_ALPHA, b1, b2, 1)
    H = ps[0]
    assert 0.2 < H < 0.8, H
    o = O.Oracle(O.DIRICHLET, 2, 8, _PLUMB_ALPHA, beta=[b1, b2], burn_out=0)
    o.set_data(X)
    R = 6000
    acc = 0
    for r in range(R):
        o.set_state(1, np.zeros(4, np.int32), zb)
        o.sweep(1, 7000 + r, mask=O.MASK_SPLITMERGE)
        acc += o.K == 2
    assert abs(acc / R - H) < 5 * math.sqrt(H * (1 - H) / R), (acc / R, H)


def test_merge_acceptance_rate_matches_hastings_ratio_dirichlet(oracle_mod):
    """Eq. sample_merges with the Dirichlet prior (Beta-binomial marginals)."""
    X, z = _PLUMB_X[:8], _PLUMB_Z[:8]
    b1, b2 = _PLUMB_B
    _, pm = _plumb_ratios(X, z, _PLUMB_ZB[:8], _PLUMB_ALPHA, b1, b2, 2)
    H = pm[(0, 1)]
    assert 0.2 < H < 0.8, H
    o = O.Oracle(O.DIRICHLET, 2, 8, _PLUMB_ALPHA, beta=[b1, b2], burn_out=10 ** 6)
    o.set_data(X)
    R = 6000
    acc = 0
    for r in range(R):
        o.set_state(2, z, np.zeros(8, np.uint8))
        o.sweep(1, 11000 + r, mask=O.MASK_SPLITMERGE)
        if o.K == 1:
            acc += 1
            _, zbo = o.labels()
            assert list(zbo) == [0] * 4 + [1] * 4  # the old clusters become sub-clusters l, r
    assert abs(acc / R - H) < 5 * math.sqrt(H * (1 - H) / R), (acc / R, H)


def _plumb_outcomes(ps, pm, K, K_max, z, zb):
    """Exact distribution of one split/merge step from a fixed state, enumerated from the
    rules as the sampler states them: splits in increasing k, each accepted with
    probability ps[k] on its own uniform, but one that would exceed K_max is rejected
    and counted (that cluster stays untouched); the right half of an accepted split gets
    the next id; merges over pairs k1 < k2 in lexicographic order among clusters no split
    touched, each cluster in at most one merge, k1 keeps its id and its partner's points
    join it as sub-cluster r (k1's own points become l); absorbed ids are removed and the
    survivors renumbered in order.  Ages: 0 for clusters created or changed this sweep,
    else the old age + 1.  Returns {(K', z', ages', zbar' outside split clusters,
    (splits, merges, rejected)): probability}."""
    out = {}
    for sp in itertools.product([0, 1], repeat=K):
        p_sp = np.prod([ps[k] if sp[k] else 1 - ps[k] for k in range(K)])
        S, split_to, touched, rejected = K, [-1] * K, set(), 0
        for k in range(K):
            if sp[k]:
                if S >= K_max:
                    rejected += 1
                    continue
                split_to[k] = S
                touched |= {k}
                S += 1
        # merges: enumerate the accept/reject results of the pairs actually proposed
        def walk(k1, merged_into, head, prob):
            if k1 >= K:
                yield merged_into, head, prob
                return
            if k1 in touched or k1 in merged_into or k1 in head:
                yield from walk(k1 + 1, merged_into, head, prob)
                return
            cands = [k2 for k2 in range(k1 + 1, K) if k2 not in touched and k2 not in merged_into and k2 not in head]
            rej = 1.0
            for k2 in cands:
                yield from walk(k1 + 1, {**merged_into, k2: k1}, head | {k1}, prob * rej * pm[(k1, k2)])
                rej *= 1 - pm[(k1, k2)]
            yield from walk(k1 + 1, merged_into, head, prob * rej)

        for merged_into, head, prob in walk(0, {}, frozenset(), p_sp):
            zn, zbn = z.copy(), zb.astype(int).copy()
            for i in range(len(z)):
                k = z[i]
                if split_to[k] >= 0:
                    if zb[i] == 1:
                        zn[i] = split_to[k]
                    zbn[i] = -1  # redrawn: not part of the key
                elif k in merged_into:
                    zn[i], zbn[i] = merged_into[k], 1
                elif k in head:
                    zbn[i] = 0
            age = [1] * S
            for k in range(K):
                if split_to[k] >= 0:
                    age[k] = age[split_to[k]] = 0
                if k in head:
                    age[k] = 0
            alive = [k for k in range(S) if k not in merged_into]
            newid = {k: j for j, k in enumerate(alive)}
            key = (len(alive), tuple(newid[k] for k in zn), tuple(age[k] for k in alive), tuple(zbn),
                   (sum(v >= 0 for v in split_to), len(merged_into), rejected))
            out[key] = out.get(key, 0.0) + prob
    return out


def test_split_merge_plumbing_exact_distribution(oracle_mod):
    """One split/merge step (Eqs. sample_splits, sample_merges; one merge per cluster,
    Sec. 4.3) from a fixed three-cluster state with K_max = 4, so that at most one split
    fits and a second accepted split is rejected and counted: the joint distribution of
    (K, relabelled z, ages, the deterministic sub-labels, counters) over 20,000 runs
    against the exact distribution enumerated independently from the acceptance
    probabilities.  This pins the id assignment, the compaction, the sub-labels of
    merged clusters, the ages (split eligibility) and the K_max rule."""
    X, z, zb = _PLUMB_X, _PLUMB_Z, _PLUMB_ZB
    b1, b2 = _PLUMB_B
    K, K_max = 3, 4
    ps, pm = _plumb_ratios(X, z, zb, _PLUMB_ALPHA, b1, b2, K)
    assert all(0.2 < v < 0.8 for v in ps + list(pm.values())), (ps, pm)
    exact = _plumb_outcomes(ps, pm, K, K_max, z, zb)
    assert abs(sum(exact.values()) - 1.0) < 1e-12
    o = O.Oracle(O.DIRICHLET, 2, K_max, _PLUMB_ALPHA, beta=[b1, b2], burn_out=0)
    o.set_data(X)
    R = 20000
    counts = {}
    coin = []
    for r in range(R):
        o.set_state(K, z, zb)
        o.sweep(1, 30000 + r, mask=O.MASK_SPLITMERGE)
        zo, zbo = o.labels()
        c = o.counters()
        ages = tuple(int(v) for v in o.ages())
        # sub-labels of the clusters a split created are redrawn; compare the rest
        key_z = tuple(int(v) for v in zo)
        counts_key = None
        for key in exact:
            if key[0] == o.K and key[1] == key_z and key[2] == ages and key[4] == (c["splits"], c["merges"],
                                                                                 c["split_rejected_kmax"]):
                if all(e < 0 or e == int(g) for e, g in zip(key[3], zbo)):
                    counts_key = key
                    coin.extend(int(g) for e, g in zip(key[3], zbo) if e < 0)
                    break
        assert counts_key is not None, (o.K, key_z, ages, list(zbo), c)
        counts[counts_key] = counts.get(counts_key, 0) + 1
    keys = sorted(exact, key=lambda k: -exact[k])
    obs = np.array([counts.get(k, 0) for k in keys], float)
    exp_ = np.array([exact[k] for k in keys]) * R
    keep = exp_ > 5
    chi = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum()
    rest_o, rest_e = obs[~keep].sum(), exp_[~keep].sum()
    if rest_e > 0:
        chi += (rest_o - rest_e) ** 2 / rest_e
    df = int(keep.sum()) - 1 + (rest_e > 0)
    assert stats.chi2.sf(chi, df) > 1e-4, (chi, df)
    # the redrawn sub-labels of a split cluster are fair coins
    coin = np.array(coin)
    assert coin.size > 1000 and abs(coin.mean() - 0.5) < 5 * 0.5 / math.sqrt(coin.size)


# -------------------------------------------------------------------- invariants

@pytest.mark.parametrize("kind", [O.NIW, O.DIRICHLET])
def test_chain_invariants(oracle_mod, kind):
    import synth

    if kind == O.NIW:
        X, _ = synth.gaussian_mixture(1500, 3, 4, 10.0, seed=7, dtype=np.float64)
        o = O.Oracle(O.NIW, 3, 12, 5.0, nu0=6.0, burn_out=2)
    else:
        X, _ = synth.multinomial_mixture(1500, 10, 4, 30, seed=8)
        X = X.astype(np.float64)
        o = O.Oracle(O.DIRICHLET, 10, 12, 5.0, burn_out=2)
    o.set_data(X)
    N = X.shape[0]
    seen_split = False
    for t in range(40):
        o.sweep(1, 77)
        seen_split |= o.counters()["splits"] > 0
        K = o.K
        z, zb = o.labels()
        n, sx, sxx = o.stats()
        assert 1 <= K <= 12 and z.min() >= 0 and z.max() < K and zb.max() <= 1
        assert n[0::3].sum() == N and np.all(n[0::3] > 0)
        assert np.all(n[0::3] == n[1::3] + n[2::3])
        assert np.allclose(sx[0::3], sx[1::3] + sx[2::3])
        for k in range(K):
            for h in range(2):
                sel = (z == k) & (zb == h)
                assert n[3 * k + 1 + h] == sel.sum()
                assert np.allclose(sx[3 * k + 1 + h], X[sel].sum(0))
                if sxx is not None:
                    assert np.allclose(sxx[3 * k + 1 + h], X[sel].T @ X[sel])
    assert seen_split and o.K >= 2


# --------------------------------------------------------- exact brute force (N<=6)

def _partitions(n):
    if n == 0:
        yield []
        return
    for p in _partitions(n - 1):
        for i in range(len(p)):
            yield p[:i] + [p[i] + [n - 1]] + p[i + 1:]
        yield p + [[n - 1]]


def _brute_force_chi2(N=5, sweeps=100000, alpha=1.0):
    X = np.array([-2.1, -1.7, 0.3, 1.9, 2.4, 0.9][:N]).reshape(-1, 1)
    o = O.Oracle(O.NIW, 1, 8, alpha, kappa0=0.5, nu0=2.0, psi0=np.eye(1), burn_out=0)
    o.set_data(X)
    logp = {}
    for p in _partitions(N):
        z = [0] * N
        for k, b in enumerate(p):
            for i in b:
                z[i] = k
        lp = len(p) * math.log(alpha) + sum(math.lgamma(len(b)) + o.log_marginal_points(X[b]) for b in p)
        logp[_compact(z)] = lp
    mx = max(logp.values())
    Z = sum(math.exp(v - mx) for v in logp.values())
    post = {k: math.exp(v - mx) / Z for k, v in logp.items()}
    cnt = dict.fromkeys(post, 0)
    for t in range(sweeps):
        o.sweep(1, 7)
        cnt[_compact(o.labels()[0])] += 1
    chi = sum((cnt[k] - post[k] * sweeps) ** 2 / (post[k] * sweeps) for k in post)
    return chi, len(post) - 1, post, cnt


def test_brute_force_bell_numbers():
    assert [sum(1 for _ in _partitions(n)) for n in range(1, 7)] == [1, 2, 5, 15, 52, 203]


@pytest.mark.xfail(strict=True, reason=(
    "The chain as the paper states it (sub-cluster split proposals with Eq. sample_splits, "
    "random-split reverse terms in Eq. sample_merges) is not exactly invariant for the DP "
    "partition posterior: at N=5, d=1 it over-weights K=1 (chi^2 ~ 5e4 on 51 d.o.f.). Each "
    "step is pinned separately above (transition kernel of steps (a)-(f), acceptance rates of "
    "both Hastings ratios), so the gap is in the proposal pair, not in the oracle."))
def test_brute_force_partition_posterior(oracle_mod):
    chi, df, post, cnt = _brute_force_chi2(N=5, sweeps=60000)
    assert stats.chi2.sf(chi, df) > 1e-3, chi
