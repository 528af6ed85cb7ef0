"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5.1 DPGMM and
Sec. 5.2 DPMNMM synthetic suites).  This module holds data generation only: no step
of the sampler.  Both the CUDA path's tests/benchmark and the oracle's tests draw
their inputs from here, with numpy's PCG64 stream (seed = 1000 + workload index
unless given).

Workloads (sizes as the benchmark uses them):
  gauss_d2   : d=2, N=10,000, 10 isotropic clusters, means U[-10,10]^2, sigma 1,
               equal weights (labels i mod 10, shuffled); FP64.
  gauss_d32  : d=32, N=1e6, 20 clusters, weights Dir(1), means N(0, 25 I),
               covariances Wishart(I, d+2); FP32.
  multinomial: d=200, N=1e6 count vectors of 100 draws, 50 topics with
               probabilities Dir(0.1 * 1), weights Dir(1); int32.
  gauss_d128 : d=128, N=1e7, 64 clusters, weights Dir(1), means N(0, 16 I),
               covariances Wishart(I, d+2); FP32.
  batched    : 512 independent mixtures, N log-uniform on [1e3, 1e6] (about 7.4e7
               points in all), d drawn from {2, 8, 32, 64}, true K uniform on {2..30},
               generated as gauss_d32; FP32 (batch_problems).
  newsgroups : d=20,000 word counts of N=11,314 documents from 20 topics, lengths
               log-uniform on [30, 600] words (newsgroups_like), compressed rows.
"""
from __future__ import annotations

import numpy as np


def _wishart_identity(rng, d, df):
    """A draw from Wishart(I_d, df) for integer df: G G^T with G a d x df standard normal."""
    G = rng.standard_normal((d, df))
    return G @ G.T


def gaussian_mixture(N, d, K, mean_scale, seed, equal_weights=False, cov="wishart",
                     sigma=1.0, mean_low=None, mean_high=None, dtype=np.float32):
    """Points from a K-component Gaussian mixture.  Returns (X [N, d], labels [N]).

    cov="wishart": each covariance ~ Wishart(I, d+2); cov="iso": sigma^2 I.
    Means ~ N(0, mean_scale^2 I), or U[mean_low, mean_high]^d when both are given.
    """
    rng = np.random.default_rng(seed)
    if mean_low is not None:
        means = rng.uniform(mean_low, mean_high, size=(K, d))
    else:
        means = rng.standard_normal((K, d)) * mean_scale
    if equal_weights:
        labels = np.arange(N) % K
        rng.shuffle(labels)
    else:
        w = rng.dirichlet(np.ones(K))
        labels = rng.choice(K, size=N, p=w)
    X = np.empty((N, d), dtype=np.float64)
    for k in range(K):
        idx = np.nonzero(labels == k)[0]
        if idx.size == 0:
            continue
        if cov == "wishart":
            S = _wishart_identity(rng, d, d + 2)
            Lc = np.linalg.cholesky(S)
        else:
            Lc = np.eye(d) * sigma
        X[idx] = means[k] + rng.standard_normal((idx.size, d)) @ Lc.T
    return X.astype(dtype, copy=False), labels.astype(np.int32)


def multinomial_mixture(N, d, K, draws, seed, topic_conc=0.1):
    """Count vectors: each row has `draws` draws from one of K topics.

    Topics ~ Dir(topic_conc * 1_d), mixture weights ~ Dir(1).  Returns
    (X [N, d] int32, labels [N])."""
    rng = np.random.default_rng(seed)
    theta = rng.dirichlet(np.full(d, topic_conc), size=K)
    w = rng.dirichlet(np.ones(K))
    labels = rng.choice(K, size=N, p=w)
    X = np.empty((N, d), dtype=np.int32)
    for k in range(K):
        idx = np.nonzero(labels == k)[0]
        if idx.size:
            X[idx] = rng.multinomial(draws, theta[k], size=idx.size)
    return X, labels.astype(np.int32)


def newsgroups_like(N=11_314, d=20_000, K=20, seed=1006, topic_conc=0.05, len_lo=30, len_hi=600):
    """Count vectors shaped like the 20newsgroups bag-of-words data of Sec. 5.3 (N = 11,314
    documents, a 20,000-word vocabulary, 20 groups), synthetic: topics ~ Dir(topic_conc 1_d),
    mixture weights Dir(1), document lengths log-uniform on [len_lo, len_hi] words, each
    word drawn from the document's topic.  Returns compressed rows (indptr int64[N + 1],
    indices int32[nnz] increasing within a row, counts int32[nnz]) and the labels."""
    rng = np.random.default_rng(seed)
    theta = rng.dirichlet(np.full(d, topic_conc), size=K)
    w = rng.dirichlet(np.ones(K))
    labels = rng.choice(K, size=N, p=w).astype(np.int32)
    lengths = np.exp(rng.uniform(np.log(len_lo), np.log(len_hi), N)).astype(np.int64)
    rows = [None] * N
    for k in range(K):
        docs = np.nonzero(labels == k)[0]
        if docs.size == 0:
            continue
        words = rng.choice(d, size=int(lengths[docs].sum()), p=theta[k])
        cut = np.cumsum(lengths[docs])[:-1]
        for i, ws in zip(docs, np.split(words, cut)):
            rows[i] = np.unique(ws, return_counts=True)
    indptr = np.zeros(N + 1, np.int64)
    indptr[1:] = np.cumsum([r[0].size for r in rows])
    indices = np.concatenate([r[0] for r in rows]).astype(np.int32)
    counts = np.concatenate([r[1] for r in rows]).astype(np.int32)
    return indptr, indices, counts, labels


def csr_to_dense(indptr, indices, counts, d, dtype=np.int32):
    N = indptr.size - 1
    X = np.zeros((N, d), dtype=dtype)
    rows = np.repeat(np.arange(N), np.diff(indptr))
    X[rows, indices] = counts
    return X


def workload(name, N=None, seed=None):
    """The named workload's data (optionally at a smaller N) and its prior settings."""
    if name == "gauss_d2":
        N = 10_000 if N is None else N
        X, y = gaussian_mixture(N, 2, 10, None, 1000 + 1 if seed is None else seed, equal_weights=True,
                                cov="iso", sigma=1.0, mean_low=-10.0, mean_high=10.0, dtype=np.float64)
        prior = dict(kind=0, kappa0=1.0, m0=np.zeros(2), nu0=4.0, psi0=np.eye(2))
        return X, y, prior, dict(alpha=10.0)
    if name == "gauss_d32":
        N = 1_000_000 if N is None else N
        X, y = gaussian_mixture(N, 32, 20, 5.0, 1000 + 2 if seed is None else seed)
        prior = dict(kind=0, kappa0=1.0, m0=np.zeros(32), nu0=35.0, psi0=np.eye(32))
        return X, y, prior, dict(alpha=10.0)
    if name == "multinomial":
        N = 1_000_000 if N is None else N
        X, y = multinomial_mixture(N, 200, 50, 100, 1000 + 3 if seed is None else seed)
        prior = dict(kind=1, beta=np.ones(200))
        return X, y, prior, dict(alpha=10.0)
    if name == "gauss_d128":
        N = 10_000_000 if N is None else N
        X, y = gaussian_mixture(N, 128, 64, 4.0, 1000 + 4 if seed is None else seed)
        prior = dict(kind=0, kappa0=1.0, m0=np.zeros(128), nu0=131.0, psi0=np.eye(128))
        return X, y, prior, dict(alpha=100.0)
    raise KeyError(name)


def batch_problems(n_problems=512, seed=1005, N_min=1_000, N_max=1_000_000, dims=(2, 8, 32, 64)):
    """The batched workload, one problem at a time: (X, y, d) with N log-uniform on
    [N_min, N_max], d drawn from dims and the true K uniform on {2..30}; each problem is
    generated like gauss_d32 (weights Dir(1), means N(0, 25 I), covariances Wishart(I, d+2))
    with its own seed.  Prior per problem: NIW kappa0 = 1, m0 = 0, nu0 = d + 3, Psi0 = I;
    alpha = 10."""
    rng = np.random.default_rng(seed)
    Ns = np.exp(rng.uniform(np.log(N_min), np.log(N_max), n_problems)).astype(np.int64)
    ds = rng.choice(np.asarray(dims), n_problems)
    Ks = rng.integers(2, 31, n_problems)
    for p in range(n_problems):
        X, y = gaussian_mixture(int(Ns[p]), int(ds[p]), int(Ks[p]), 5.0, seed=seed * 1000 + p)
        yield X, y, int(ds[p])
