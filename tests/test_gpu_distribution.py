"""The reduced-precision chains sample the same posterior as the FP64 chain.

Per-step budgets (score error, label disagreement) bound what one step can change;
this test checks the whole chain in distribution.  Ten independent chains per arm
(different Philox seeds per arm, so the two samples are independent) run from K = 1
on the same synthetic data:
  - Gaussian, d = 32, N = 100,000 points from 10 clusters (the generator of the
    d = 32 workload): TF32 tensor-core chains against FP64-plain chains;
  - multinomial, d = 200, N = 50,000 count vectors of 100 draws from 10 topics (the
    generator of the multinomial workload): BF16 tensor-core chains against FP64.
For each chain: the mean of its cluster-count trajectory (K after every 10th sweep),
the final K, the final log joint log p(X, z) = log CRP(z; alpha) + sum_k log f(C_k)
(the collapsed joint of Sec. 2.2-2.3: alpha^K Gamma(alpha) / Gamma(alpha + N)
prod_k Gamma(N_k), times each cluster's marginal likelihood under the prior, which the
oracle's pinned closed forms evaluate from FP64 statistics of the original data under
the chain's final labels), and the NMI of the final labels to the generating labels.  Each quantity is compared between the arms by
a two-sided Mann-Whitney U test; the test fails when p < 0.001 for any of them (eight
tests in all: a false alarm rate below 1% for the file)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O

pytestmark = pytest.mark.gpu
P = None
ALPHA_TEST = 1e-3
SEEDS = 10


@pytest.fixture(scope="module", autouse=True)
def gpu():
    global P
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2204_08988_gb300 as mod

    P = mod


def nmi(a, b):
    """Normalised mutual information (arithmetic-mean normalisation) of two labelings."""
    a = np.unique(a, return_inverse=True)[1]
    b = np.unique(b, return_inverse=True)[1]
    n = len(a)
    C = np.zeros((a.max() + 1, b.max() + 1))
    np.add.at(C, (a, b), 1.0)
    pa, pb, pab = C.sum(1) / n, C.sum(0) / n, C / n
    nz = pab > 0
    mi = (pab[nz] * np.log(pab[nz] / np.outer(pa, pb)[nz])).sum()
    ha = -(pa[pa > 0] * np.log(pa[pa > 0])).sum()
    hb = -(pb[pb > 0] * np.log(pb[pb > 0])).sum()
    return 1.0 if ha + hb == 0 else 2.0 * mi / (ha + hb)


def log_joint(o, alpha, X, z, gaussian):
    """log CRP(z; alpha) + sum_k log f(C_k) of the labels z on the original data X (the
    statistics recounted in FP64 from X, so that both arms are scored on the same data:
    the TF32 path stores its points rounded to TF32, and its own statistics describe
    those rounded points)."""
    N = len(z)
    X64 = X.astype(np.float64)
    K = int(z.max()) + 1
    lj = K * math.log(alpha) + math.lgamma(alpha) - math.lgamma(alpha + N)
    for k in range(K):
        Xk = X64[z == k]
        lj += math.lgamma(len(Xk))
        if gaussian:
            lj += o.niw_log_marginal(len(Xk), Xk.sum(0), Xk.T @ Xk)
        else:
            lj += o.dirmult_log_marginal(Xk.sum(0))
    return lj


def run_chain(kind, X, y, prec, seed, alpha, sweeps, prior, o):
    N, d = X.shape
    g = P.DPMM(kind, d, 64, alpha, prec=prec, burn_out=5, **prior)
    g.set_data(X)
    traj = []
    for t in range(sweeps // 10):
        g.sweep(10, seed)
        traj.append(g.K)
    K = g.K
    z, _ = g.labels()
    g.close()
    assert z.max() + 1 == K
    return dict(traj_mean=float(np.mean(traj)), K=K, log_joint=log_joint(o, alpha, X, z, kind == 0), nmi=nmi(z, y))


def compare(kind, X, y, prec_fast, alpha, sweeps, prior):
    o = O.Oracle(O.NIW if kind == 0 else O.DIRICHLET, X.shape[1], 8, alpha, **prior)
    fast = [run_chain(kind, X, y, prec_fast, 100 + s, alpha, sweeps, prior, o) for s in range(SEEDS)]
    ref = [run_chain(kind, X, y, P.PREC_FP64_PLAIN, 200 + s, alpha, sweeps, prior, o) for s in range(SEEDS)]
    report = {}
    for q in ("traj_mean", "K", "log_joint", "nmi"):
        a = np.array([r[q] for r in fast], float)
        b = np.array([r[q] for r in ref], float)
        p = 1.0 if np.all(a == a[0]) and np.all(b == a[0]) else stats.mannwhitneyu(a, b, alternative="two-sided").pvalue
        report[q] = (a.mean(), a.std(), b.mean(), b.std(), p)
    print("\n%s: quantity: fast mean (sd) | fp64 mean (sd) | Mann-Whitney p" % ("gauss_d32" if kind == 0 else "multinomial"))
    for q, (am, asd, bm, bsd, p) in report.items():
        print("  %-9s %.6g (%.3g) | %.6g (%.3g) | p = %.3g" % (q, am, asd, bm, bsd, p))
    return report


def test_tf32_chain_matches_fp64_chain_in_distribution():
    import synth

    d = 32
    X, y = synth.gaussian_mixture(100_000, d, 10, 5.0, seed=2002)
    prior = dict(kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))
    rep = compare(0, X, y, P.PREC_TF32, 10.0, 100, prior)
    for q, v in rep.items():
        assert v[4] > ALPHA_TEST, (q, v)
    assert rep["nmi"][0] > 0.9 and rep["nmi"][2] > 0.9  # both arms find the mixture


def test_bf16_multinomial_chain_matches_fp64_chain_in_distribution():
    import synth

    d = 200
    X, y = synth.multinomial_mixture(50_000, d, 10, 100, seed=2003)
    prior = dict(beta=np.ones(d))
    rep = compare(1, X, y, P.PREC_BF16, 10.0, 100, prior)
    for q, v in rep.items():
        assert v[4] > ALPHA_TEST, (q, v)
    assert rep["nmi"][0] > 0.9 and rep["nmi"][2] > 0.9
