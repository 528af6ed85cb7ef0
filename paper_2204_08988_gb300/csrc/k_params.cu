// k_params.cu -- steps (a)-(d) of the sweep (Sec. 4.1, Eqs. sample_weights,
// sample_sub_weights, sample_params, sample_sub_params) on the GPU: one warp draws the
// weights; one CTA per (sub-)cluster slot draws its parameters from the conjugate
// posterior of its sufficient statistics (in FP64; the NIW factorisation in FP32 on the
// reduced-precision paths, with an FP64 retry).
#include <math.h>

#include <algorithm>

#include "dpmm_internal.cuh"
#include "fp64_chol.cuh"

namespace dpmm {

struct StatView {
    const double* S;  // stats table
    StatLayout L;
    // M[j][l] of slot (k, h); h = -1 sums both sub-clusters (the cluster)
    __device__ double m(int k, int h, int j, int l) const {
        int e = L.ent(j, l);
        if (h >= 0) return S[(size_t)(2 * k + h) * L.E + e];
        return S[(size_t)(2 * k) * L.E + e] + S[(size_t)(2 * k + 1) * L.E + e];
    }
    __device__ double count(int k, int h) const { return m(k, h, L.d, L.d); }
};

__device__ inline double block_reduce_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    v = -INFINITY;
    for (int i = 0; i < nw; ++i) v = fmax(v, sh[i]);
    __syncthreads();
    return v;
}

__device__ inline double block_reduce_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    for (int i = 0; i < nw; ++i) v += sh[i];  // fixed order: deterministic
    __syncthreads();
    return v;
}

// Every random variate of steps (a)-(d) that does not depend on a Cholesky factor,
// one thread each, spread over the whole GPU (GB300's FP64 pipes are narrow, so FP64
// work must be spread over many SMs):
//   blockIdx.y < 3 K_max: slot s = blockIdx.y (NIW only): thread q < npair draws the
//     Box-Muller pair q of the slot's PARAM stream (normals 2q, 2q + 1) into W (entry
//     r*d + c, r < c; zero below the diagonal) or eps (normal d*d + j); thread
//     npair + j draws the Bartlett chi-square j into bart[s][j] (as sqrt);
//   blockIdx.y = 3 K_max: the 3K + 1 Gamma draws of steps (a), (b) into lgs.
struct VarArgs {
    StatView sv;
    const int* dK;
    const uint32_t* diter;
    uint64_t seed;
    double alpha, nu0;
    int kind, Kmax, niw;
    int f32;       // the slots' variates in FP32 arithmetic (NIW, reduced-precision paths)
    int f32w;      // the weights' Gamma draws in FP32 arithmetic (reduced-precision paths)
    double* W;     // p_W
    double* eps;   // 3 K_max x d
    double* bart;  // 3 K_max x d
    double* lgs;   // 3 K_max + 1
};

// Element q of the variates of slot s's NIW draw (Sec. 4.1 steps (c), (d)): for q < npair a
// pair of normals (the entries above W's diagonal, then eps), for npair <= q < npair + d the
// Bartlett diagonal B_jj = sqrt(chi^2(nu_n - d + j + 1)).  W, eps, bart: the slot's rows.
// f32: FP32 arithmetic on the leading bits of the same Philox words (the reduced-precision
// paths; an FP64 retry of the slot draws them again in FP64).
__device__ inline void slot_variate(const Key& key, int s, int d, double nun, int q, bool f32, double* W, double* eps,
                                    double* bart) {
    const int npair = (d * d + d + 1) / 2;
    const uint32_t NB = 64u * d;
    if (q < npair) {
        uint32_t w[4];
        key.block((uint32_t)s, TAG_PARAM, NB + (uint32_t)q, w);
        double nv2[2];
        if (f32) {
            const float rr = sqrtf(-2.f * logf(u01_f32(w[0])));
            float sn, cs;
            sincospif(2.f * u01_f32(w[2]), &sn, &cs);
            nv2[0] = rr * cs;
            nv2[1] = rr * sn;
        } else {
            const double u1 = u01_f64(w[0], w[1]), u2 = u01_f64(w[2], w[3]);
            const double rr = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);  // sin and cos of 2 pi u2
            nv2[0] = rr * cs;
            nv2[1] = rr * sn;
        }
        for (int o = 0; o < 2; ++o) {
            const int qq = 2 * q + o;
            if (qq < d * d) {
                const int r = qq / d, c = qq % d;
                W[qq] = r < c ? nv2[o] : 0.0;
            } else if (qq < d * d + d) {
                eps[qq - d * d] = nv2[o];
            }
        }
    } else if (q < npair + d) {
        const int j = q - npair;
        const double df = nun - d + (j + 1);
        if (f32) {
            const float lg = f_log_gamma(key, (uint32_t)s, TAG_PARAM, 64u * j, (float)(0.5 * df));
            bart[j] = (double)sqrtf(2.f * expf(lg));
        } else {
            const double lg = d_log_gamma(key, (uint32_t)s, TAG_PARAM, 64u * j, 0.5 * df);
            bart[j] = sqrt(2.0 * exp(lg));
        }
    }
}

__global__ void variates_kernel(VarArgs a) {
    const int K = *a.dK;
    const int d = a.sv.L.d;
    Key key{a.seed, a.diter[0], a.diter[1], a.diter[2]};
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if ((int)blockIdx.y == 3 * a.Kmax) {
        const int T = 3 * K + 1;
        if (q >= T) return;
        // Gamma draws of the weights: FP32 arithmetic on the reduced-precision paths
        auto lg = [&](uint32_t c0, uint32_t tag, uint32_t base, double shape) -> double {
            return a.f32w ? (double)f_log_gamma(key, c0, tag, base, (float)shape) : d_log_gamma(key, c0, tag, base, shape);
        };
        double v;
        if (q < K) v = lg((uint32_t)q, TAG_WEIGHT, 0, a.sv.count(q, -1));
        else if (q == K) v = lg(0xFFFFFFFFu, TAG_WEIGHT, 0, a.alpha);
        else {
            const int k = (q - K - 1) >> 1, h = (q - K - 1) & 1;
            v = lg((uint32_t)k, TAG_SUBW, 64u * h, a.sv.count(k, h) + 0.5 * a.alpha);
        }
        a.lgs[q] = v;
        return;
    }
    const int s = blockIdx.y;
    if (!a.niw || s >= 3 * K) return;
    const int k = s / 3, h = s % 3 - 1;
    slot_variate(key, s, d, a.nu0 + a.sv.count(k, h), q, a.f32 != 0, a.W + (size_t)s * d * d, a.eps + (size_t)s * d,
                 a.bart + (size_t)s * d);
}

// (a) (pi_1..pi_K, pi~) ~ Dir(N_1..N_K, alpha); (b) pibar_k ~ Dir(N_kl + a/2, N_kr + a/2):
// normalisation of the Gamma draws made by variates_kernel.  One warp: a wider block
// would only multiply the FP64 reduction work on GB300's narrow FP64 pipe.
template <typename T>
__global__ void __launch_bounds__(32) weights_kernel(const int* dK, const double* lgs, double* logw,
                                                     double* cweights) {
    const int K = *dK, lane = threadIdx.x;
    if constexpr (sizeof(T) == 4) {  // the reduced-precision paths: FP32 arithmetic
        float lmax = -INFINITY;
        for (int k = lane; k <= K; k += 32) lmax = fmaxf(lmax, (float)lgs[k]);
        for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        float s = 0.f;
        for (int k = lane; k <= K; k += 32) s += expf((float)lgs[k] - lmax);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float lse = lmax + logf(s);
        for (int k = lane; k < K; k += 32) {
            const float lw = (float)lgs[k] - lse;
            logw[3 * k] = lw;
            cweights[k] = expf(lw);
            const float gl = (float)lgs[K + 1 + 2 * k], gr = (float)lgs[K + 2 + 2 * k];
            const float m = fmaxf(gl, gr);
            const float l2 = m + log1pf(expf(-fabsf(gl - gr)));
            logw[3 * k + 1] = gl - l2;
            logw[3 * k + 2] = gr - l2;
        }
        return;
    }
    double lmax = -INFINITY;
    for (int k = lane; k <= K; k += 32) lmax = fmax(lmax, lgs[k]);
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    double s = 0.0;
    for (int k = lane; k <= K; k += 32) s += exp(lgs[k] - lmax);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double lse = lmax + log(s);
    for (int k = lane; k < K; k += 32) {
        const double lw = lgs[k] - lse;
        logw[3 * k] = lw;
        cweights[k] = exp(lw);
        const double gl = lgs[K + 1 + 2 * k], gr = lgs[K + 2 + 2 * k];
        const double m = fmax(gl, gr);
        const double l2 = m + log1p(exp(-fabs(gl - gr)));
        logw[3 * k + 1] = gl - l2;
        logw[3 * k + 2] = gr - l2;
    }
}

struct NiwPrior {
    double kappa0, nu0;
    const double* m0s;   // prior mean in storage coordinates (m0 - center), device
    const double* psi0;  // device, d x d
};

// (c), (d): (mu, Lambda) ~ NIW posterior of one slot.  Lambda = W W^T with
// W = U^-T B (Psi_n = U U^T, B upper-triangular Bartlett factor of Wishart(nu_n, I):
// B_jj^2 ~ chi^2(nu_n - d + j), j = 1..d, N(0,1) above the diagonal);
// mu = m_n + W^-T eps / sqrt(kappa_n).
//
// GB300's FP64 pipe retires about two operations per clock per SM with a 64-cycle
// dependent latency, so the kernel keeps FP64 work off the serial paths: the slot's
// statistics are staged in shared memory, every division is a reciprocal formed once,
// the factorisation takes one reciprocal square root per pivot, and the triangular
// solve for W runs right-looking (one parallel update of the rows above per step).
// T is the working type of the factorisation and the solves: double on the FP64 path;
// float on the reduced-precision paths (whose label scores are FP32 anyway), with the
// statistics, C = S2 - S1 S1^T / n and the outputs in FP64.  A slot whose FP32
// factorisation loses more than 10 bits of a pivot to cancellation (or meets a
// non-positive one) is flagged in retry[] and redone by the FP64 instantiation
// (launched with retry set, it takes only the flagged slots).
// Dynamic shared memory: (E doubles when staged) + (d*ld + 11*d (+ d*d when W fits)) T.
__device__ inline float log_t(float x) { return logf(x); }
__device__ inline double log_t(double x) { return log(x); }

template <typename T>
__global__ void niw_params_kernel(StatView sv, const double* shift_stats, NiwPrior pr, const int* dK,
                                  double* eps, double* bart, const double* logw, double* p_mu,
                                  double* p_W, double* p_logdetW, double* p_c, int* derr, int w_in_smem,
                                  int staged, int* retry, const uint32_t* diter, uint64_t seed) {
    extern __shared__ double smem[];
    const int d = sv.L.d, E = sv.L.E;
    const int K = *dK;
    const int s = blockIdx.x;
    if (s >= 3 * K) return;
    const bool retry_pass = sizeof(T) == 8 && retry != nullptr;
    if (retry_pass && retry[s] == 0) return;
    const int k = s / 3, h = s % 3 - 1;  // h = -1: the cluster
    const int ld = d | 1;         // odd row stride: column reads without bank conflicts
    double* S = smem;             // E: staged statistics
    T* A = (T*)(S + (staged ? E : 0));  // d x ld: Psi_n (lower), then the solve's multipliers
    T* mn = A + d * ld;           // d
    T* dg = mn + d;               // d: diagonal of Psi_n
    T* Bd = dg + d;               // d: Bartlett diagonal, then v
    T* acc = Bd + d;              // d: eps
    T* rd = acc + d;              // d: 1 / U_jj
    T* rw = rd + d;               // d: 1 / W_jj
    T* piv = rw + d;              // d: pivots
    T* cols = piv + d;            // 4 d: the factorisation's scaled panel columns
    double* Wg = p_W + (size_t)s * d * d;
    T* W = w_in_smem ? cols + 4 * d : (T*)Wg;  // d x d working copy (global only when T = double)
    __shared__ double sh[32];
    __shared__ double s_n, s_rn, s_kn, s_rkn;
    __shared__ int s_fail;
    const int tid = threadIdx.x, nt = blockDim.x;

    if (staged) {
        stage_slot(sv.S, E, k, h, S);
        __syncthreads();
    }
    auto M = [&](int j, int l) -> double { return staged ? S[sv.L.ent(j, l)] : sv.m(k, h, j, l); };
    if (tid == 0) {
        const double n = M(d, d);
        s_n = n;
        s_rn = n > 0 ? 1.0 / n : 0.0;
        s_kn = pr.kappa0 + n;
        s_rkn = 1.0 / s_kn;
        s_fail = 0;
    }
    __syncthreads();
    const double n = s_n, rn = s_rn, kn = s_kn, rkn = s_rkn;
    if (retry_pass) {  // the slot's variates again, in FP64 (the FP32 pass drew them in FP32)
        const Key key{seed, diter[0], diter[1], diter[2]};
        const int npair = (d * d + d + 1) / 2;
        for (int q = tid; q < npair + d; q += nt)
            slot_variate(key, s, d, pr.nu0 + n, q, false, p_W + (size_t)s * d * d, eps + (size_t)s * d,
                         bart + (size_t)s * d);
        __syncthreads();
    }
    const double* sh_k = shift_stats + (size_t)k * d;
    // xbar - m0 per coordinate (FP64), for the Psi_n build below; in the factorisation's
    // scratch columns, which it overwrites only after that build
    double* dxm = (double*)(((uintptr_t)cols + 7) & ~(uintptr_t)7);
    for (int j = tid; j < d; j += nt) {
        const double xbar = n > 0 ? sh_k[j] + M(j, d) * rn : 0.0;
        mn[j] = (T)((pr.kappa0 * pr.m0s[j] + n * xbar) * rkn);
        dxm[j] = xbar - pr.m0s[j];
        Bd[j] = (T)bart[(size_t)s * d + j];
        acc[j] = (T)eps[(size_t)s * d + j];
    }
    if (w_in_smem)  // the normals above the diagonal (zero below), drawn by variates_kernel
        for (int e0 = tid; e0 < d * d; e0 += 8 * nt) {  // eight loads in flight per thread
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = e0 + u * nt < d * d ? Wg[e0 + u * nt] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (e0 + u * nt < d * d) W[e0 + u * nt] = (T)v[u];
        }
    __syncthreads();
    // Psi_n = Psi0 + C + (kappa0 n / kappa_n)(xbar - m0)(xbar - m0)^T, C = S2 - S1 S1^T / n
    // (in FP64: the subtraction cancels); lower triangle only: the factorisation reads
    // nothing else
    const double f = n > 0 ? pr.kappa0 * n * rkn : 0.0;
    const int ntri = d * (d + 1) / 2;
    for (int e0 = tid; e0 < ntri; e0 += 4 * nt) {  // the Psi0 entries of four entries loaded first
        int jj[4], ll[4];
        double p0[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = min(e0 + u * nt, ntri - 1);
            tri_index(e, jj[u], ll[u]);  // l <= j
            p0[u] = pr.psi0[jj[u] * d + ll[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (e0 + u * nt >= ntri) break;
            const int j = jj[u], l = ll[u];
            double C = 0.0;
            if (n > 0) C = M(l, j) - M(l, d) * M(j, d) * rn;
            const T a = (T)(p0[u] + C + f * dxm[j] * dxm[l]);
            A[j * ld + l] = a;
            if (l == j) dg[j] = a;
        }
    }
    __syncthreads();
    chol_ldl_t<T>(A, d, ld, piv, rd, cols, dg, sizeof(T) == 4 ? T(1.0 / 1024) : T(0), &s_fail);
    if (s_fail) {
        if (sizeof(T) == 4) {  // redo this slot in FP64
            if (tid == 0) retry[s] = 1;
            return;
        }
        if (tid == 0) atomicExch(derr, (int)DPMM_ENUMERIC);
    }
    // U_ij = A_ij / sqrt(v_j) below the diagonal (U_jj = sqrt(v_j)); the solve below
    // needs V_ri = U_ri / U_rr = A_ri rd[i] rd[r], kept in place of A
    for (int e = tid; e < d * (d - 1) / 2; e += nt) {
        int r, i;
        tri_index(e, r, i);  // i <= r
        ++r;                 // strict lower triangle: i < r
        A[r * ld + i] *= rd[i] * rd[r];
    }
    // U^T W = B, right-looking: after step r, row r of W (unscaled) is final and the rows
    // above are updated with it; the rows are scaled by 1 / U_rr at the end
    for (int j = tid; j < d; j += nt) W[j * d + j] = Bd[j];
    __syncthreads();
    for (int r = d - 1; r > 0; --r) {
        const int w = d - r;  // columns c = r .. d-1
        const T* Wr = W + (size_t)r * d;
        const T* Vr = A + (size_t)r * ld;
        for (int e0 = tid; e0 < r * w; e0 += 2 * nt) {
            const int e1 = e0 + nt;
            const int i0 = e0 / w, c0 = r + e0 % w;  // row i < r
            const bool two = e1 < r * w;
            const int i1 = two ? e1 / w : i0, c1 = two ? r + e1 % w : c0;
            const T a0 = W[i0 * d + c0], v0 = Vr[i0], w0 = Wr[c0];
            const T a1 = W[i1 * d + c1], v1 = Vr[i1], w1 = Wr[c1];
            W[i0 * d + c0] = fma(-v0, w0, a0);
            if (two) W[i1 * d + c1] = fma(-v1, w1, a1);
        }
        __syncthreads();
    }
    for (int e = tid; e < d * d; e += nt) {
        const int r = e / d, c = e % d;
        if (c >= r) W[e] *= rd[r];
    }
    __syncthreads();
    for (int j = tid; j < d; j += nt) rw[j] = T(1) / W[j * d + j];
    __syncthreads();
    // W^T v = eps (forward substitution) by warp 0, lane m keeps sum_{j<m} W[j][m] v_j;
    // mu = m_n + v / sqrt(kappa_n)
    if (tid < 32) {
        const int ns = (d + 31) >> 5;
        T am[8];  // m = tid + 32 i, d <= 256
#pragma unroll
        for (int i = 0; i < 8; ++i) am[i] = T(0);
        for (int j = 0; j < d; ++j) {
            const int own = j & 31, slot = j >> 5;
            T mine = T(0);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i == slot) mine = am[i];
            T vj = T(0);
            if (tid == own) {
                vj = (acc[j] - mine) * rw[j];
                Bd[j] = vj;  // reuse as v
            }
            vj = __shfl_sync(0xffffffffu, vj, own);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int m = tid + 32 * i;
                if (i < ns && m > j && m < d) am[i] += W[j * d + m] * vj;
            }
        }
    }
    __syncthreads();
    double* mu = p_mu + (size_t)s * d;
    const T rsk = rsqrt_t((T)kn);
    for (int j = tid; j < d; j += nt) mu[j] = (double)(mn[j] + Bd[j] * rsk);
    if (w_in_smem)
        for (int e = tid; e < d * d; e += nt) Wg[e] = (double)W[e];
    double lgd = 0.0;
    for (int j = tid; j < d; j += nt) lgd += (double)log_t(W[j * d + j]);
    lgd = block_reduce_sum(lgd, sh);
    if (tid == 0) {
        p_logdetW[s] = lgd;
        p_c[s] = logw[s] + lgd - 0.5 * d * 1.8378770664093453;  // log(2 pi)
        if (retry_pass) retry[s] = 0;
    }
}

// theta ~ Dir(beta + counts), as log theta (log-space Gamma draws).  cc (compressed-row
// path only): the compact sub-cluster counts, read instead of the statistics table.
__global__ void dirichlet_params_kernel(StatView sv, const double* beta, const int* dK, const uint32_t* diter,
                                        uint64_t seed, const double* logw, double* p_logtheta, double* p_c,
                                        const float* cc) {
    __shared__ double sh[32];
    const int d = sv.L.d;
    const int K = *dK;
    const int s = blockIdx.x;
    if (s >= 3 * K) return;
    const int k = s / 3, h = s % 3 - 1;
    Key key{seed, diter[0], diter[1], diter[2]};
    double* lt = p_logtheta + (size_t)s * d;
    double mx = -INFINITY;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double cnt = cc ? (h < 0 ? (double)cc[(size_t)(2 * k) * d + j] + (double)cc[(size_t)(2 * k + 1) * d + j]
                                       : (double)cc[(size_t)(2 * k + h) * d + j])
                              : sv.m(k, h, j, d);
        double v = d_log_gamma(key, (uint32_t)s, TAG_PARAM, 64u * j, beta[j] + cnt);
        lt[j] = v;
        mx = fmax(mx, v);
    }
    mx = block_reduce_max(mx, sh);
    double sum = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) sum += exp(lt[j] - mx);
    double lse = mx + log(block_reduce_sum(sum, sh));
    for (int j = threadIdx.x; j < d; j += blockDim.x) lt[j] -= lse;
    if (threadIdx.x == 0) p_c[s] = logw[s];
}

// The same draw in FP32 (the reduced-precision paths): f_log_gamma, FP32 normalisation; log
// theta stored in the FP64 table and its FP32 mirror.  A slot's
// d categories (20,000 for document data) are spread over blockIdx.y chunks of
// DP_CHUNK; the first kernel draws and leaves each chunk's maximum and sum of
// exp(v - maximum), the second combines a slot's chunks in a fixed order and normalises.
constexpr int DP_CHUNK = 2048;

template <typename Src>
__global__ void dirichlet_draw_f32_kernel(int d, const double* beta, const int* dK, const uint32_t* diter,
                                          uint64_t seed, Src cnt, float* q_logtheta, float2* part) {
    __shared__ double sh[32];
    const int K = *dK;
    const int s = blockIdx.x;
    if (s >= 3 * K) return;
    const int k = s / 3, h = s % 3 - 1;
    const int j0 = blockIdx.y * DP_CHUNK, j1 = min(d, j0 + DP_CHUNK);
    Key key{seed, diter[0], diter[1], diter[2]};
    float* qt = q_logtheta + (size_t)s * d;
    float mx = -INFINITY;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const auto c = h < 0 ? cnt(2 * k, j) + cnt(2 * k + 1, j) : cnt(2 * k + h, j);
        const float v = f_log_gamma(key, (uint32_t)s, TAG_PARAM, 64u * j, (float)beta[j] + (float)c);
        qt[j] = v;
        mx = fmaxf(mx, v);
    }
    mx = (float)block_reduce_max((double)mx, sh);
    float sum = 0.f;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) sum += __expf(qt[j] - mx);
    sum = (float)block_reduce_sum((double)sum, sh);
    if (threadIdx.x == 0) part[(size_t)s * gridDim.y + blockIdx.y] = make_float2(mx, sum);
}

__global__ void dirichlet_norm_f32_kernel(int d, const int* dK, const double* logw, const float2* part,
                                          float* q_logtheta, double* p_logtheta, double* p_c) {
    const int K = *dK;
    const int s = blockIdx.x;
    if (s >= 3 * K) return;
    const int nc = gridDim.y;
    float mx = -INFINITY;
    for (int q = 0; q < nc; ++q) mx = fmaxf(mx, part[(size_t)s * nc + q].x);
    float sum = 0.f;
    for (int q = 0; q < nc; ++q) {
        const float2 p = part[(size_t)s * nc + q];
        sum += p.y * __expf(p.x - mx);
    }
    const float lse = mx + logf(sum);
    const int j0 = blockIdx.y * DP_CHUNK, j1 = min(d, j0 + DP_CHUNK);
    float* qt = q_logtheta + (size_t)s * d;
    double* lt = p_logtheta + (size_t)s * d;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const float v = qt[j] - lse;
        qt[j] = v;
        lt[j] = (double)v;
    }
    if (blockIdx.y == 0 && threadIdx.x == 0) p_c[s] = logw[s];
}

// FP32 mirrors of the drawn parameters for the reduced-precision paths, and the
// shift the next statistics are accumulated with (the cluster's drawn mean).
__global__ void derive_kernel(int kind, int d, int tf32, const int* dK, const double* p_logw, const double* p_mu,
                              const double* p_W, const double* p_c, const double* p_logtheta, float* q_mu,
                              float* q_W, float* q_c, float* q_b, double* p_b, float* q_logtheta, double* shift_new,
                              float* shift32) {
    const int K = *dK;
    const int s = blockIdx.x;
    if (s >= 3 * K) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (kind == DPMM_PRIOR_NIW) {
        const double* W = p_W + (size_t)s * d * d;
        const double* mu = p_mu + (size_t)s * d;
        for (int e0 = 0; e0 < d * d; e0 += 8 * nt) {  // eight loads in flight per thread
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * nt + tid;
                v[u] = e < d * d ? W[e] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * nt + tid;
                if (e < d * d) q_W[(size_t)s * d * d + e] = (float)v[u];
            }
        }
        for (int j = tid; j < d; j += nt) {
            q_mu[(size_t)s * d + j] = (float)mu[j];
            // b_j = sum_l mu_l W_lj (l <= j: W is upper triangular), with W as the tensor
            // cores see it, in the order l = 0, 1, ...; a fixed trip count lets the loads of
            // several rows be in flight at once (the FMA chain is the only serial part)
            double b = 0.0;
#pragma unroll 8
            for (int l = 0; l < d; ++l) {
                const double w = W[l * d + j], m = mu[l];
                if (l <= j) b = fma(m, tf32 ? (double)round_tf32((float)w) : w, b);
            }
            q_b[(size_t)s * d + j] = (float)b;
            p_b[(size_t)s * d + j] = b;  // read by the tensor-core image builds
            if (s % 3 == 0) {
                shift_new[(size_t)(s / 3) * d + j] = (double)(float)mu[j];
                shift32[(size_t)(s / 3) * d + j] = (float)mu[j];
            }
        }
    } else {  // blockIdx.y: chunks of 4096 categories
        const int j0 = blockIdx.y * 4096, j1 = min(d, j0 + 4096);
        for (int j = j0 + tid; j < j1; j += nt) q_logtheta[(size_t)s * d + j] = (float)p_logtheta[(size_t)s * d + j];
    }
    if (tid == 0 && blockIdx.y == 0) q_c[s] = (float)p_c[s];
}

static StatView make_sv(dpmm_ctx* c) { return StatView{c->stats, c->st}; }

cudaError_t launch_weights(dpmm_ctx* c, uint64_t seed) {
    VarArgs a{make_sv(c), c->dK, c->diter, seed, c->alpha, c->nu0, c->kind, c->K_max, c->kind == DPMM_PRIOR_NIW,
              c->kind == DPMM_PRIOR_NIW && c->prec != DPMM_PREC_FP64_PLAIN, c->prec != DPMM_PREC_FP64_PLAIN, c->p_W,
              c->eps, c->bart, c->lgs};
    const int d = c->d;
    const int per_slot = c->kind == DPMM_PRIOR_NIW ? (d * d + d + 1) / 2 + d : 0;
    const int per = std::max(per_slot, 3 * c->K_max + 1);
    dim3 grid((per + 127) / 128, 3 * c->K_max + 1);
    prof_begin(c, "variates");
    variates_kernel<<<grid, 128, 0, c->stream>>>(a);
    prof_end(c, "variates");
    prof_begin(c, "weights");
    if (c->prec == DPMM_PREC_FP64_PLAIN) weights_kernel<double><<<1, 32, 0, c->stream>>>(c->dK, c->lgs, c->p_logw, c->cweights);
    else weights_kernel<float><<<1, 32, 0, c->stream>>>(c->dK, c->lgs, c->p_logw, c->cweights);
    prof_end(c, "weights");
    c->nlaunch += 2;
    return cudaGetLastError();
}

cudaError_t launch_params(dpmm_ctx* c, uint64_t seed) {
    if (c->kind == DPMM_PRIOR_NIW) {
        const size_t dd = (size_t)c->d * c->d, E = (size_t)c->st.E, dl = (size_t)c->d * (c->d | 1);
        NiwPrior pr{c->kappa0, c->nu0, c->center + c->d, c->center + 2 * c->d};
        // shared memory of the T instantiation: E doubles (staged), then d*ld + 7 d (+ d*d) T
        auto plan = [&](size_t tsz, int& staged, int& w_in_smem) {
            size_t sm = tsz * (dl + 11 * (size_t)c->d);
            staged = w_in_smem = 0;
            if (sm + 8 * E <= 200 * 1024) {
                sm += 8 * E;
                staged = 1;
            }
            if (sm + tsz * dd <= 200 * 1024) {
                sm += tsz * dd;
                w_in_smem = 1;
            }
            return sm;
        };
        int st64, w64, st32, w32;
        const size_t sm64 = plan(8, st64, w64), sm32 = plan(4, st32, w32);
        const bool fp32 = c->prec != DPMM_PREC_FP64_PLAIN && w32;  // FP32 needs W in shared memory
        cudaError_t e = cudaFuncSetAttribute(niw_params_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm64);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(niw_params_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32);
        if (e != cudaSuccess) return e;
        prof_begin(c, "niw_params");
        if (fp32) {
            niw_params_kernel<float><<<3 * c->K_max, 128, sm32, c->stream>>>(
                make_sv(c), c->shift_stats, pr, c->dK, c->eps, c->bart, c->p_logw, c->p_mu, c->p_W, c->p_logdetW,
                c->p_c, c->derr, w32, st32, c->retry, c->diter, seed);
            c->nlaunch += 1;
        }
        // the FP64 path, or the FP64 retry of slots whose FP32 factorisation failed
        niw_params_kernel<double><<<3 * c->K_max, 128, sm64, c->stream>>>(
            make_sv(c), c->shift_stats, pr, c->dK, c->eps, c->bart, c->p_logw, c->p_mu, c->p_W, c->p_logdetW, c->p_c,
            c->derr, w64, st64, fp32 ? c->retry : nullptr, c->diter, seed);
        prof_end(c, "niw_params");
        c->nlaunch += 1;
    } else {
        prof_begin(c, "dirichlet_params");
        if (c->prec != DPMM_PREC_FP64_PLAIN) {  // the reduced-precision paths: FP32 draws
            const dim3 grid(3 * c->K_max, (c->d + DP_CHUNK - 1) / DP_CHUNK);
            if (c->sparse)
                dirichlet_draw_f32_kernel<CountsF32><<<grid, 256, 0, c->stream>>>(
                    c->d, c->center + c->d, c->dK, c->diter, seed, CountsF32{c->sp_cc, c->d}, c->q_logtheta,
                    (float2*)c->sp_part);
            else
                dirichlet_draw_f32_kernel<CountsStats><<<grid, 256, 0, c->stream>>>(
                    c->d, c->center + c->d, c->dK, c->diter, seed, CountsStats{c->stats, c->st}, c->q_logtheta,
                    (float2*)c->sp_part);
            dirichlet_norm_f32_kernel<<<grid, 256, 0, c->stream>>>(c->d, c->dK, c->p_logw, (const float2*)c->sp_part,
                                                                  c->q_logtheta, c->p_logtheta, c->p_c);
            c->nlaunch += 1;
        } else
            dirichlet_params_kernel<<<3 * c->K_max, 256, 0, c->stream>>>(make_sv(c), c->center + c->d, c->dK,
                                                                         c->diter, seed, c->p_logw, c->p_logtheta,
                                                                         c->p_c, c->sparse ? c->sp_cc : nullptr);
        prof_end(c, "dirichlet_params");
        c->nlaunch += 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_derive(dpmm_ctx* c) {
    prof_begin(c, "derive");
    const dim3 dgrid(3 * c->K_max, c->kind == DPMM_PRIOR_NIW ? 1 : (c->d + 4095) / 4096);
    derive_kernel<<<dgrid, 128, 0, c->stream>>>(c->kind, c->d, c->prec == DPMM_PREC_TF32, c->dK, c->p_logw, c->p_mu, c->p_W, c->p_c,
                                                       c->p_logtheta, c->q_mu, c->q_W, c->q_c, c->q_b, c->p_b,
                                                       c->q_logtheta, c->shift_new, c->shift32);
    prof_end(c, "derive");
    c->nlaunch += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c->sparse) e = sparse_prepare(c);
    if (e == cudaSuccess && tc_supported(c)) e = tc_prepare(c);
    if (e == cudaSuccess && substats_tc_supported(c)) e = substats_tc_prepare(c);
    if (e == cudaSuccess && x3_supported(c)) e = x3_prepare(c);
    return e;
}

}  // namespace dpmm
