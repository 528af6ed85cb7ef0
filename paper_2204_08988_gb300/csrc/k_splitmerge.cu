// k_splitmerge.cu -- splits and merges (Sec. 4.1, Eqs. sample_splits and
// sample_merges; Sec. 4.3 "a cluster takes part in at most one merge").
//
//   marginal : log f_x(C; lambda) for every cluster, sub-cluster and cluster pair,
//              FP64, one CTA per item (NIW: Cholesky log-determinant of Psi_n;
//              Dirichlet-multinomial: lgamma sums).
//   decision : one thread walks the proposals in the fixed order (splits by
//              increasing k, then merge pairs in lexicographic order) with the
//              Philox uniforms (tag SPLIT, c0 = k; tag MERGE, c0 = k1, block k2,
//              indices after removing emptied clusters), and writes the relabel map.
//   relabel  : applies it to z, z-bar (sub-labels of split clusters re-drawn, tag
//              RESUB); gated: it returns at once when nothing changed.
#include <math.h>

#include <cmath>

#include "dpmm_internal.cuh"
#include "fp64_chol.cuh"

namespace dpmm {

struct SMArgs {
    const double* stats;
    StatLayout L;
    const double* shift_stats;  // K_max x d
    const double* m0s;          // d (storage coordinates)
    const double* psi0;         // d x d
    const double* beta;         // d
    double kappa0, nu0, logdet_psi0, alpha;
    double log_alpha, lg_alpha, lg_half_alpha;  // log a, lgamma(a), lgamma(a / 2), from the host
    double lmvg_nu0;                            // sum_j lgamma(nu0 / 2 - j / 2), from the host
    double half_d_log_kappa0;                   // d / 2 log kappa0, from the host
    double sum_beta, lg_sum_beta, sum_lg_beta;  // sum beta_j, its lgamma, sum lgamma(beta_j)
    int stage;                                  // statistics blocks staged in shared memory
    int kind, K_max;
    const int* dK;
};

__device__ inline double smv(const SMArgs& a, int k, int h, int j, int l) {
    int e = a.L.ent(j, l);
    if (h >= 0) return a.stats[(size_t)(2 * k + h) * a.L.E + e];
    return a.stats[(size_t)(2 * k) * a.L.E + e] + a.stats[(size_t)(2 * k + 1) * a.L.E + e];
}

__device__ inline double lmvgamma(double x, int d) {
    double s = 0.25 * d * (d - 1) * log(M_PI);
    for (int j = 1; j <= d; ++j) s += lgamma(x + 0.5 * (1 - j));
    return s;
}

// per-slot lgamma table after the log marginals: lg[2 s] = lgamma(n_s),
// lg[2 s + 1] = lgamma(alpha / 2 + n_s)
__host__ __device__ inline size_t lg_offset(int K_max) { return 3 * (size_t)K_max + (size_t)K_max * (K_max - 1) / 2 + 1; }
// then lgamma(n) and lgamma(alpha + n) of every merge pair's n = n_k1 + n_k2 (two per pair)
__host__ __device__ inline size_t lg_pair_offset(int K_max) { return lg_offset(K_max) + 6 * (size_t)K_max; }

__device__ inline void pair_of(int p, int K, int& k1, int& k2) {
    int r = 0, off = 0;
    while (off + (K - r - 1) <= p) {
        off += K - r - 1;
        ++r;
    }
    k1 = r;
    k2 = r + 1 + (p - off);
}

// One item (slot or merge pair) of marginal_kernel.  Dynamic shared memory: d (d | 1) + 10 d
// doubles (+ 2 E when the statistics are staged).
__device__ __forceinline__ void marginal_item(const SMArgs& a, double* Ltab, int* derr, int K, int e) {
    extern __shared__ double smem[];
    __shared__ double sh[32];
    __shared__ double s_n, s_n1, s_n2;
    const int d = a.L.d, tid = threadIdx.x, nt = blockDim.x;
    int k1, k2, h;
    if (e < 3 * K) {
        k1 = e / 3;
        k2 = -1;
        h = e % 3 - 1;
    } else {
        pair_of(e - 3 * K, K, k1, k2);
        h = -1;
    }
    double* out = Ltab + (e < 3 * K ? e : 3 * a.K_max + (e - 3 * K));
    if (tid == 32 || tid == 33) {  // the slot's or the pair's lgamma terms for the Hastings ratios
        if (e < 3 * K) {
            const double ns = smv(a, k1, h, d, d);
            Ltab[lg_offset(a.K_max) + 2 * e + (tid - 32)] = lgamma(tid == 32 ? ns : 0.5 * a.alpha + ns);
        } else {
            const double nm = smv(a, k1, -1, d, d) + smv(a, k2, -1, d, d);
            Ltab[lg_pair_offset(a.K_max) + 2 * (e - 3 * K) + (tid - 32)] = lgamma(tid == 32 ? nm : a.alpha + nm);
        }
    }
    if (a.kind == DPMM_PRIOR_DIRICHLET) {
        // the prior's terms (sum beta, lgamma(sum beta), sum lgamma(beta_j)) come from the host
        double sc = 0.0, acc = 0.0;
        for (int j = tid; j < d; j += nt) {
            double c = smv(a, k1, h, j, d) + (k2 >= 0 ? smv(a, k2, -1, j, d) : 0.0);
            sc += c;
            acc += lgamma(a.beta[j] + c);
        }
        double tot = 0.0;
        // sum counts and lgamma terms over the block (fixed order)
        for (int o = 16; o > 0; o >>= 1) {
            sc += __shfl_xor_sync(0xffffffffu, sc, o);
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
        }
        __shared__ double shc[32], sha[32];
        if ((tid & 31) == 0) {
            shc[tid >> 5] = sc;
            sha[tid >> 5] = acc;
        }
        __syncthreads();
        if (tid == 0) {
            double c = 0.0, l = 0.0;
            for (int w = 0; w < (nt + 31) / 32; ++w) {
                c += shc[w];
                l += sha[w];
            }
            tot = l - a.sum_lg_beta + a.lg_sum_beta - lgamma(a.sum_beta + c);
            *out = tot;
        }
        return;
    }
    const int ld = d | 1;      // odd row stride: column reads without bank conflicts
    double* A = smem;          // d x ld (lower triangle)
    double* xb = A + d * ld;   // merged mean
    double* x1 = xb + d;
    double* x2 = x1 + d;
    double* piv = x2 + d;      // pivots of the factorisation
    double* rs = piv + d;
    double* cols = rs + d;     // 4 d: the factorisation's scaled panel columns
    double* dxb = cols + 4 * d;  // merged mean - m0
    double* S1 = dxb + d;      // staged statistics of (k1, h) and of cluster k2 (E each)
    double* S2 = S1 + a.L.E;
    const bool staged = a.stage != 0;
    if (staged) {
        stage_slot(a.stats, a.L.E, k1, h, S1);
        if (k2 >= 0) stage_slot(a.stats, a.L.E, k2, -1, S2);
        __syncthreads();
    }
    // M[j][l] (j <= l) of the first and second statistics block
    auto M1 = [&](int j, int l) -> double { return staged ? S1[a.L.ent(j, l)] : smv(a, k1, h, j, l); };
    auto M2 = [&](int j, int l) -> double { return staged ? S2[a.L.ent(j, l)] : smv(a, k2, -1, j, l); };
    __shared__ double s_r1, s_r2, s_rn, s_w12;
    if (tid == 0) {  // reciprocals once: FP64 division is slow on GB300's narrow FP64 pipe
        const double n1 = M1(d, d), n2 = k2 >= 0 ? M2(d, d) : 0.0, n = n1 + n2;
        s_n1 = n1;
        s_n2 = n2;
        s_n = n;
        s_r1 = n1 > 0 ? 1.0 / n1 : 0.0;
        s_r2 = n2 > 0 ? 1.0 / n2 : 0.0;
        s_rn = n > 0 ? 1.0 / n : 0.0;
        s_w12 = n1 * n2 * s_rn;
    }
    __syncthreads();
    const double n1 = s_n1, n2 = s_n2, n = s_n, r1 = s_r1, r2 = s_r2, rn = s_rn, w12 = s_w12;
    for (int j = tid; j < d; j += nt) {
        double m1 = n1 > 0 ? a.shift_stats[(size_t)k1 * d + j] + M1(j, d) * r1 : 0.0;
        double m2 = (k2 >= 0 && n2 > 0) ? a.shift_stats[(size_t)k2 * d + j] + M2(j, d) * r2 : 0.0;
        x1[j] = m1;
        x2[j] = m2;
        xb[j] = n > 0 ? (n1 * m1 + n2 * m2) * rn : 0.0;
        dxb[j] = xb[j] - a.m0s[j];
    }
    __syncthreads();
    const double kn = a.kappa0 + n, nun = a.nu0 + n;
    const double f = n > 0 ? a.kappa0 * n / kn : 0.0;
    const int ntri = d * (d + 1) / 2;
    for (int e0 = tid; e0 < ntri; e0 += 4 * nt) {  // the Psi0 entries of four entries loaded first
        int jj[4], ll[4];
        double p0[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            tri_index(min(e0 + u * nt, ntri - 1), jj[u], ll[u]);  // l <= j: the factorisation reads nothing else
            p0[u] = a.psi0[jj[u] * d + ll[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (e0 + u * nt >= ntri) break;
            const int j = jj[u], l = ll[u];
            const int q = j * ld + l;
            double C = 0.0;
            if (n1 > 0) C += M1(l, j) - M1(l, d) * M1(j, d) * r1;
            if (k2 >= 0 && n2 > 0) {
                C += M2(l, j) - M2(l, d) * M2(j, d) * r2;
                if (n1 > 0) C += w12 * (x1[j] - x2[j]) * (x1[l] - x2[l]);
            }
            A[q] = p0[u] + C + f * dxb[j] * dxb[l];
        }
    }
    __syncthreads();
    chol_ldl(A, d, ld, piv, rs, cols, derr);
    // -(nun/2) log|Psi_n| and the multivariate-lgamma ratio (the prior's part from the
    // host), summed over j by all threads; lane 0 of warp 0 adds log kappa_n
    double part = 0.0;
    for (int j = tid; j < d; j += nt) part += -0.5 * nun * log(piv[j]) + lgamma(0.5 * nun - 0.5 * j);
    if (tid == 0) part -= 0.5 * d * log(kn);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) sh[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (nt + 31) / 32; ++w) s += sh[w];
        // 1.1447298858494002 = log(pi)
        *out = -0.5 * n * d * 1.1447298858494002 + s - a.lmvg_nu0 + 0.5 * a.nu0 * a.logdet_psi0 + a.half_d_log_kappa0;
    }
}

// Log marginal likelihoods of every slot (cluster and sub-clusters) and merge pair: the
// resident blocks take the items in turn, so that no block is launched for the slots and
// pairs beyond the current K.
__global__ void marginal_kernel(SMArgs a, double* Ltab, int* derr) {
    const int K = *a.dK;
    const int total = 3 * K + K * (K - 1) / 2;
    for (int e = blockIdx.x; e < total; e += gridDim.x) {
        marginal_item(a, Ltab, derr, K, e);
        __syncthreads();  // shared memory is reused by the next item
    }
}

// The Dirichlet-multinomial log marginals from the sub-cluster counts (Src: the FP32 compact
// table of compressed-row data, or the statistics table of dense data on the reduced-precision
// paths).  Only categories with a nonzero count contribute (for c = 0,
// lgamma(beta_j + c) - lgamma(beta_j) = 0).  The term for count c is read from a table of
// lgamma(beta + c) - lgamma(beta) made on the host when every beta_j is equal and c is below
// its length, and computed otherwise.  Same outputs as marginal_kernel (Ltab), one CTA per
// cluster, sub-cluster and pair.
template <typename Src>
__device__ __forceinline__ void marginal_counts_item(const SMArgs& a, const Src& cnt, const double* lgt, int nlgt,
                                                     const double* lgb, double* Ltab, int K, int e) {
    __shared__ double shc[32], sha[32];
    const int d = a.L.d, tid = threadIdx.x, nt = blockDim.x;
    int k1, k2, h;
    if (e < 3 * K) {
        k1 = e / 3;
        k2 = -1;
        h = e % 3 - 1;
    } else {
        pair_of(e - 3 * K, K, k1, k2);
        h = -1;
    }
    double* out = Ltab + (e < 3 * K ? e : 3 * a.K_max + (e - 3 * K));
    if (tid == 32 || tid == 33) {  // the slot's or the pair's lgamma terms for the Hastings ratios
        if (e < 3 * K) {
            const double ns = smv(a, k1, h, d, d);
            Ltab[lg_offset(a.K_max) + 2 * e + (tid - 32)] = lgamma(tid == 32 ? ns : 0.5 * a.alpha + ns);
        } else {
            const double nm = smv(a, k1, -1, d, d) + smv(a, k2, -1, d, d);
            Ltab[lg_pair_offset(a.K_max) + 2 * (e - 3 * K) + (tid - 32)] = lgamma(tid == 32 ? nm : a.alpha + nm);
        }
    }
    using V = decltype(cnt(0, 0));  // the source's own type: FP32 sums stay off the FP64 pipe
    const int s0 = 2 * k1 + (h < 0 ? 0 : h);
    double sc = 0.0, acc = 0.0;
    for (int j = tid; j < d; j += nt) {
        V c = cnt(s0, j);
        if (h < 0) c += cnt(2 * k1 + 1, j);
        if (k2 >= 0) c += cnt(2 * k2, j) + cnt(2 * k2 + 1, j);  // integer counts: exact
        if (c > V(0)) {
            sc += (double)c;
            acc += (lgt && c < (V)nlgt) ? lgt[(int)c] : lgamma(a.beta[j] + (double)c) - lgb[j];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    if ((tid & 31) == 0) {
        shc[tid >> 5] = sc;
        sha[tid >> 5] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        double c = 0.0, l = 0.0;
        for (int w = 0; w < (nt + 31) / 32; ++w) {  // fixed order
            c += shc[w];
            l += sha[w];
        }
        *out = l + a.lg_sum_beta - lgamma(a.sum_beta + c);
    }
}

template <typename Src>
__global__ void marginal_counts_kernel(SMArgs a, Src cnt, const double* lgt, int nlgt, const double* lgb, double* Ltab) {
    const int K = *a.dK;
    const int total = 3 * K + K * (K - 1) / 2;
    for (int e = blockIdx.x; e < total; e += gridDim.x) {
        marginal_counts_item<Src>(a, cnt, lgt, nlgt, lgb, Ltab, K, e);
        __syncthreads();  // shared memory is reused by the next item
    }
}

// Every split and merge ratio with its Philox uniform, in parallel: acc[k] for the
// split of cluster k, acc[K_max + p] for merge pair p; 1 = accepted if proposed.
// Indices in the Philox counters are those after removing emptied clusters.
constexpr int DEC_KMAX_SM = 1024;  // K_max <= 1000

// One warp per block: the warp first finds which clusters hold points and their indices
// after removing the empty ones (a prefix count in shared memory), then each lane takes a
// proposal.
__global__ void __launch_bounds__(32) hastings_kernel(SMArgs a, const double* Ltab, const uint32_t* diter, uint64_t seed,
                                                      int labels_ran, int* acc) {
    __shared__ int s_live[DEC_KMAX_SM], s_cid[DEC_KMAX_SM];
    const int K = *a.dK;
    const int d = a.L.d, lane = threadIdx.x;
    for (int q0 = 0, base = 0; q0 < K; q0 += 32) {
        const int q = q0 + lane;
        const int lv = q < K ? (labels_ran ? (smv(a, q, -1, d, d) > 0 ? 1 : 0) : 1) : 0;
        const unsigned m = __ballot_sync(0xffffffffu, lv);
        if (q < K) {
            s_live[q] = lv;
            s_cid[q] = base + __popc(m & ((1u << lane) - 1u));
        }
        base += __popc(m);
    }
    __syncwarp();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = K * (K - 1) / 2;
    if (e >= K + npairs) return;
    Key key{seed, diter[0], diter[1], diter[2]};
    auto live = [&](int k) { return s_live[k] != 0; };
    auto cid = [&](int k) { return s_cid[k]; };
    const double la = a.log_alpha, al = a.alpha;
    const double* lg = Ltab + lg_offset(a.K_max);
    if (e < K) {
        const int k = e;
        const double nl = smv(a, k, 0, d, d), nr = smv(a, k, 1, d, d);
        int ok = 0;
        if (live(k) && nl >= 1 && nr >= 1) {
            const double lH = la + lg[2 * (3 * k + 1)] + Ltab[3 * k + 1] + lg[2 * (3 * k + 2)] + Ltab[3 * k + 2] -
                              lg[2 * (3 * k)] - Ltab[3 * k];
            ok = log(d_uniform(key, (uint32_t)cid(k), TAG_SPLIT, 0)) < lH;
        }
        acc[k] = ok;
    } else {
        const int p = e - K;
        int k1, k2;
        pair_of(p, K, k1, k2);
        int ok = 0;
        if (live(k1) && live(k2)) {
            // lgamma(n_k1 + n_k2) and lgamma(alpha + n_k1 + n_k2), formed by the marginal kernel
            const double* lgp = Ltab + lg_pair_offset(a.K_max) + 2 * (size_t)p;
            const double lH = lgp[0] - la - lg[2 * (3 * k1)] - lg[2 * (3 * k2)] + Ltab[3 * a.K_max + p] -
                              Ltab[3 * k1] - Ltab[3 * k2] + a.lg_alpha - lgp[1] + lg[2 * (3 * k1) + 1] +
                              lg[2 * (3 * k2) + 1] - 2.0 * a.lg_half_alpha;
            ok = log(d_uniform(key, (uint32_t)cid(k1), TAG_MERGE, (uint32_t)cid(k2))) < lH;
        }
        acc[a.K_max + p] = ok;
    }
}

struct DecArgs {
    SMArgs s;
    const double* Ltab;
    const uint32_t* diter;
    uint64_t seed;
    int burn_out, labels_ran, sm_enabled, init_mode;
    const int* acc;    // hastings_kernel's accept flags
    int* age;          // K_max
    int* dK;
    int* relabel;      // 3 K_max: map_l, map_r, zmode
    int* counters;     // [0] splits [1] merges [2] rejected (K_max) [3] removed [4] changed
    double* shift_new; // K_max x d
    float* shift32;
    int* derr;
};

#define DEC_KMAX 1024

// Dynamic shared memory: the accept flags (one byte per proposal) when they fit in
// dyn_flags bytes, so that the sequential walk reads shared memory only.  The
// bookkeeping (live clusters, split targets, new ids, ages, relabel maps) is done by
// ballot prefix counts over chunks of 32 clusters in cluster order, which gives the ids
// a sequential walk gives; only the merge walk is sequential (on bit masks for K <= 64).
__global__ void decision_kernel(DecArgs a, int dyn_flags) {
    __shared__ int live[DEC_KMAX], split_to[DEC_KMAX], merged_into[DEC_KMAX], head[DEC_KMAX];
    __shared__ int newid[DEC_KMAX], newid_split[DEC_KMAX], src[DEC_KMAX], nage[DEC_KMAX], cid[DEC_KMAX];
    __shared__ unsigned long long rowm[64];
    __shared__ int s_Kc, s_nsplit, s_nrej, s_nmerge, s_nid;
    extern __shared__ unsigned char flg[];
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned below = (1u << lane) - 1u;
    const int K = *a.s.dK;
    const int d = a.s.L.d;
    const int nflags = K + K * (K - 1) / 2;
    const bool staged = a.sm_enabled && nflags <= dyn_flags;
    for (int k = tid; k < K; k += blockDim.x) {
        live[k] = a.labels_ran ? (smv(a.s, k, -1, d, d) > 0) : 1;
        nage[k] = a.age[k];
        split_to[k] = -1;
        merged_into[k] = -1;
        head[k] = 0;
    }
    if (staged) {
        for (int q = tid; q < nflags; q += blockDim.x) flg[q] = (unsigned char)(q < K ? a.acc[q] : a.acc[a.s.K_max + q - K]);
    }
    __syncthreads();
    auto acc_split = [&](int k) { return staged ? (int)flg[k] : a.acc[k]; };
    auto acc_merge = [&](int p) { return staged ? (int)flg[K + p] : a.acc[a.s.K_max + p]; };
    // splits: the accepted proposals of live clusters past burn-out, in cluster order, take
    // the ids Kc, Kc + 1, ... below K_max; the ones beyond K_max are rejected
    if (tid < 32) {
        int Kc = 0;
        for (int k0 = 0; k0 < K; k0 += 32) Kc += __popc(__ballot_sync(0xffffffffu, k0 + lane < K && live[k0 + lane]));
        int want = 0, ns = 0;
        if (a.sm_enabled) {
            const int room = a.s.K_max - Kc;
            for (int k0 = 0; k0 < K; k0 += 32) {
                const int k = k0 + lane;
                const bool w = k < K && live[k] && nage[k] >= a.burn_out && acc_split(k);
                const unsigned m = __ballot_sync(0xffffffffu, w);
                const int r = want + __popc(m & below);
                if (w && r < room) split_to[k] = Kc + r;
                want += __popc(m);
            }
            ns = min(want, max(room, 0));
        }
        if (lane == 0) {
            s_Kc = Kc;
            s_nsplit = ns;
            s_nrej = want - ns;
        }
    }
    __syncthreads();
    // merges: for k1 in order, the first eligible k2 > k1 whose proposal is accepted
    // (eligible: live, not split, not merged, not already a merge's head)
    if (tid < 32) {
        int nm = 0;
        if (a.sm_enabled) {
            if (K <= 64) {
                for (int k1 = lane; k1 < K; k1 += 32) {  // bit k2 of row k1: pair (k1, k2) accepted
                    unsigned long long row = 0;
                    const int p0 = k1 * (2 * K - k1 - 1) / 2 - k1 - 1;
                    for (int k2 = k1 + 1; k2 < K; ++k2)
                        if (acc_merge(p0 + k2)) row |= 1ull << k2;
                    rowm[k1] = row;
                }
                unsigned long long el = 0;
                for (int k0 = 0; k0 < K; k0 += 32) {
                    const int k = k0 + lane;
                    el |= (unsigned long long)__ballot_sync(0xffffffffu, k < K && live[k] && split_to[k] < 0) << k0;
                }
                __syncwarp();
                if (lane == 0) {
                    for (int k1 = 0; k1 < K; ++k1) {
                        if (!((el >> k1) & 1ull)) continue;
                        const unsigned long long cand = el & rowm[k1];
                        if (cand) {
                            const int k2 = __ffsll((long long)cand) - 1;
                            merged_into[k2] = k1;
                            head[k1] = 1;
                            el &= ~((1ull << k1) | (1ull << k2));
                            ++nm;
                        }
                    }
                }
            } else {  // 32 candidates at a time by the warp; same outcome as the plain double loop
                auto elig = [&](int k) { return live[k] && split_to[k] < 0 && merged_into[k] < 0 && !head[k]; };
                for (int k1 = 0; k1 < K; ++k1) {
                    if (!elig(k1)) continue;
                    int found = -1;
                    for (int b0 = k1 + 1; b0 < K && found < 0; b0 += 32) {
                        const int k2 = b0 + lane;
                        const bool ok = k2 < K && elig(k2) && acc_merge(k1 * (2 * K - k1 - 1) / 2 + (k2 - k1 - 1));
                        const unsigned m = __ballot_sync(0xffffffffu, ok);
                        if (m) found = b0 + __ffs(m) - 1;
                    }
                    if (found >= 0) {
                        if (lane == 0) {
                            merged_into[found] = k1;
                            head[k1] = 1;
                        }
                        ++nm;
                    }
                    __syncwarp();
                }
            }
        }
        if (lane == 0) s_nmerge = nm;
    }
    __syncthreads();
    // new ids: the clusters that stay (live, not merged away) keep their order, then the
    // second halves of the splits in cluster order; src[new id] = old cluster
    if (tid < 32) {
        int base = 0;
        for (int k0 = 0; k0 < K; k0 += 32) {
            const int k = k0 + lane;
            const bool sv = k < K && live[k] && merged_into[k] < 0;
            const unsigned m = __ballot_sync(0xffffffffu, sv);
            const int q = base + __popc(m & below);
            if (k < K) newid[k] = sv ? q : -1;
            if (sv) src[q] = k;
            base += __popc(m);
        }
        for (int k0 = 0; k0 < K; k0 += 32) {
            const int k = k0 + lane;
            const bool sp = k < K && split_to[k] >= 0;
            const unsigned m = __ballot_sync(0xffffffffu, sp);
            const int q = base + __popc(m & below);
            if (sp) {
                newid_split[k] = q;
                src[q] = k;
            }
            base += __popc(m);
        }
        if (lane == 0) {
            if (base == 0) {  // no cluster holds a point: the statistics disagree with the labels
                atomicExch(a.derr, (int)DPMM_ENUMERIC);
                newid[0] = 0;
                src[0] = 0;
                live[0] = 1;
                base = 1;
            }
            s_nid = base;
        }
    }
    __syncthreads();
    const int nid = s_nid;
    // ages: survivors one sweep older, clusters created by a split or merge start at 0
    for (int q = tid; q < nid; q += blockDim.x) {
        const int k = src[q];
        const bool fresh = split_to[k] >= 0 || head[k];  // both halves of a split, and a merge
        cid[q] = fresh ? 0 : nage[k] + (a.init_mode ? 0 : 1);
    }
    int* map_l = a.relabel;
    int* map_r = a.relabel + a.s.K_max;
    int* zmode = a.relabel + 2 * a.s.K_max;
    for (int k = tid; k < K; k += blockDim.x) {
        if (!live[k]) {
            map_l[k] = map_r[k] = -1;
            zmode[k] = 0;
        } else if (split_to[k] >= 0) {
            map_l[k] = newid[k];
            map_r[k] = newid_split[k];
            zmode[k] = 3;
        } else if (merged_into[k] >= 0) {
            map_l[k] = map_r[k] = newid[merged_into[k]];
            zmode[k] = 2;
        } else if (head[k]) {
            map_l[k] = map_r[k] = newid[k];
            zmode[k] = 1;
        } else {
            map_l[k] = map_r[k] = newid[k];
            zmode[k] = 0;
        }
    }
    if (tid == 0) {
        const int nsplit = s_nsplit, nmerge = s_nmerge;
        a.counters[0] = nsplit;
        a.counters[1] = nmerge;
        a.counters[2] = s_nrej;
        a.counters[3] = K - s_Kc;
        a.counters[4] = (nid != K || nsplit || nmerge) ? 1 : 0;
    }
    __syncthreads();
    const int Kn = nid;
    // the statistics shifts follow their clusters (Gaussian only: the multinomial
    // statistics are not shifted, and d x K can be 20,000 x 100 there)
    if (a.s.kind == DPMM_PRIOR_NIW)
    for (int q = tid; q < Kn * d; q += blockDim.x) {
        int k = q / d, j = q % d;
        double v = a.s.shift_stats[(size_t)src[k] * d + j];
        a.shift_new[(size_t)k * d + j] = v;
        a.shift32[(size_t)k * d + j] = (float)v;
    }
    for (int k = tid; k < Kn; k += blockDim.x) a.age[k] = cid[k];
    __syncthreads();
    if (tid == 0) *a.dK = Kn;
}

__global__ void relabel_kernel(int64_t N, const int* relabel, int Kmax, const int* gate, const uint32_t* diter,
                               uint64_t seed, int32_t* z, uint8_t* zbar, int* derr) {
    if (*gate == 0) return;
    const Key key{seed, diter[0], diter[1], diter[2]};
    // grid-stride: the launch is one wave, so that the usual gated-off launch is cheap
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int k = z[i];
        const int h = zbar[i];
        if ((unsigned)k >= (unsigned)Kmax) {  // never for consistent state: keep memory safe, report
            atomicExch(derr, (int)DPMM_ENUMERIC);
            k = 0;
        }
        const int mode = relabel[2 * Kmax + k];
        int nz = h ? relabel[Kmax + k] : relabel[k];
        if (nz < 0) {  // a point in a cluster counted as empty
            atomicExch(derr, (int)DPMM_ENUMERIC);
            nz = 0;
        }
        z[i] = nz;
        if (mode == 1) zbar[i] = 0;
        else if (mode == 2) zbar[i] = 1;
        else if (mode == 3) zbar[i] = d_uniform(key, (uint32_t)i, TAG_RESUB, 0) < 0.5 ? 0 : 1;
    }
}

__global__ void advance_kernel(uint32_t* diter) { *diter += 1; }

static SMArgs sm_args(dpmm_ctx* c) {
    SMArgs a;
    a.stats = c->stats;
    a.L = c->st;
    a.shift_stats = c->shift_stats;
    a.m0s = c->center + c->d;
    a.psi0 = c->center + 2 * c->d;
    a.beta = c->center + c->d;
    a.kappa0 = c->kappa0;
    a.nu0 = c->nu0;
    a.logdet_psi0 = c->logdet_psi0;
    a.alpha = c->alpha;
    a.log_alpha = std::log(c->alpha);
    a.lg_alpha = std::lgamma(c->alpha);
    a.lg_half_alpha = std::lgamma(0.5 * c->alpha);
    a.lmvg_nu0 = 0.0;
    for (int j = 0; j < c->d; ++j) a.lmvg_nu0 += std::lgamma(0.5 * c->nu0 - 0.5 * j);
    a.half_d_log_kappa0 = 0.5 * c->d * std::log(c->kappa0);
    a.sum_beta = a.lg_sum_beta = a.sum_lg_beta = 0.0;
    if (c->kind == DPMM_PRIOR_DIRICHLET) {
        for (double b : c->beta) {
            a.sum_beta += b;
            a.sum_lg_beta += std::lgamma(b);
        }
        a.lg_sum_beta = std::lgamma(a.sum_beta);
    }
    a.stage = 0;
    a.kind = c->kind;
    a.K_max = c->K_max;
    a.dK = c->dK;
    return a;
}

cudaError_t launch_restats_gated(dpmm_ctx* c, const int* gate);

cudaError_t launch_splitmerge(dpmm_ctx* c, uint64_t seed, int labels_ran, int sm_enabled) {
    SMArgs s = sm_args(c);
    if (sm_enabled) {
        int items = 3 * c->K_max + c->K_max * (c->K_max - 1) / 2;
        // the Dirichlet marginal needs no matrix workspace; the NIW one stages the two
        // statistics blocks it reads when they fit
        size_t sm = 0;
        if (c->kind == DPMM_PRIOR_NIW) {
            sm = sizeof(double) * ((size_t)c->d * (c->d | 1) + 10 * c->d);
            const size_t st = sm + sizeof(double) * 2 * (size_t)c->st.E;
            if (st <= 160 * 1024) {
                sm = st;
                s.stage = 1;
            }
        }
        if (sm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(marginal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
        }
        // one wave of resident blocks, each taking items in turn (the items beyond the
        // current K launch no block)
        auto waves = [&](const void* fn, int threads, size_t smem) {
            int per = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per < 1) {
                cudaGetLastError();
                per = 1;
            }
            return (unsigned)std::min<int64_t>(items, (int64_t)per * c->num_sms);
        };
        prof_begin(c, "marginal");
        if (c->sparse)
            marginal_counts_kernel<CountsF32>
                <<<waves((const void*)marginal_counts_kernel<CountsF32>, 256, 0), 256, 0, c->stream>>>(
                    s, CountsF32{c->sp_cc, c->d}, c->sp_lgt, c->sp_lgt ? SP_LGT : 0, c->sp_lgb, c->Ltab);
        else if (c->kind == DPMM_PRIOR_DIRICHLET && c->prec != DPMM_PREC_FP64_PLAIN)  // dense counts
            marginal_counts_kernel<CountsStats>
                <<<waves((const void*)marginal_counts_kernel<CountsStats>, 256, 0), 256, 0, c->stream>>>(
                    s, CountsStats{c->stats, c->st}, c->sp_lgt, c->sp_lgt ? SP_LGT : 0, c->sp_lgb, c->Ltab);
        else
            marginal_kernel<<<waves((const void*)marginal_kernel, 128, sm), 128, sm, c->stream>>>(s, c->Ltab, c->derr);
        prof_end(c, "marginal");
        c->nlaunch += 1;
    }
    if (sm_enabled) {
        const int items = c->K_max + c->K_max * (c->K_max - 1) / 2;
        prof_begin(c, "hastings");
        hastings_kernel<<<(items + 31) / 32, 32, 0, c->stream>>>(s, c->Ltab, c->diter, seed, labels_ran ? 1 : 0,
                                                                   c->acc);
        prof_end(c, "hastings");
        c->nlaunch += 1;
    }
    DecArgs a;
    a.s = s;
    a.acc = c->acc;
    a.Ltab = c->Ltab;
    a.diter = c->diter;
    a.seed = seed;
    a.burn_out = c->burn_out;
    a.labels_ran = labels_ran;
    a.sm_enabled = sm_enabled;
    a.init_mode = (labels_ran == 2);
    a.labels_ran = labels_ran ? 1 : 0;
    a.age = c->age;
    a.dK = c->dK;
    a.relabel = c->relabel;
    a.counters = c->counters;
    a.shift_new = c->shift_new;
    a.shift32 = c->shift32;
    a.derr = c->derr;
    prof_begin(c, "decision");
    const int dyn = 32 * 1024;
    cudaError_t ea = cudaFuncSetAttribute(decision_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (ea != cudaSuccess) return ea;
    decision_kernel<<<1, 256, dyn, c->stream>>>(a, dyn);
    prof_end(c, "decision");
    c->nlaunch += 1;
    return cudaGetLastError();
}

cudaError_t launch_relabel(dpmm_ctx* c, uint64_t seed) {
    prof_begin(c, "relabel");
    const unsigned grid = (unsigned)std::min<int64_t>((c->N + 255) / 256, 8 * (int64_t)c->num_sms);
    relabel_kernel<<<grid, 256, 0, c->stream>>>(c->N, c->relabel, c->K_max, c->counters + 4,
                                                                         c->diter, seed, c->z, c->zbar, c->derr);
    prof_end(c, "relabel");
    c->nlaunch += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_restats_gated(c, c->counters + 4);
    return e;
}

cudaError_t launch_advance(dpmm_ctx* c) {
    advance_kernel<<<1, 1, 0, c->stream>>>(c->diter);
    c->nlaunch += 1;
    return cudaGetLastError();
}

}  // namespace dpmm
