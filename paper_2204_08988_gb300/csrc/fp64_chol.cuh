// fp64_chol.cuh -- FP64 building blocks of the parameter and split/merge steps: staging a
// (sub-)cluster's statistics block in shared memory and a right-looking Cholesky (LDL)
// factorisation written for GB300's FP64 pipe (about two operations per clock per SM,
// 64-cycle dependent latency): the only serial work per pivot is one reciprocal square
// root, and the block meets its barriers once per panel of four pivots.
#pragma once
#include "dpmm_internal.cuh"

namespace dpmm {

// out[e] = statistics entry e of slot (k, h) of the table S (E entries per sub-cluster);
// h = -1 sums the two sub-clusters (the cluster).  Every thread of the block calls it.
__device__ inline void stage_slot(const double* S, int E, int k, int h, double* out) {
    const double* s0 = S + (size_t)(2 * k + (h < 0 ? 0 : h)) * E;
    const double* s1 = S + (size_t)(2 * k + 1) * E;
    const int nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < E; e0 += 4 * nt) {  // four entries' loads in flight per thread
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * nt;
            a[u] = e < E ? s0[e] : 0.0;
            b[u] = e < E && h < 0 ? s1[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e0 + u * nt < E) out[e0 + u * nt] = h < 0 ? a[u] + b[u] : a[u];
    }
}

// Row i0 and column l0 (l0 <= i0) of entry e of a lower triangle enumerated row by row.
__device__ inline void tri_index(int e, int& i0, int& l0) {
    int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    if ((i + 1) * (i + 2) / 2 <= e) ++i;
    if (i * (i + 1) / 2 > e) --i;
    i0 = i;
    l0 = e - i * (i + 1) / 2;
}

__device__ inline float rsqrt_t(float x) { return rsqrtf(x); }
__device__ inline double rsqrt_t(double x) { return rsqrt(x); }

// In-place factorisation of the symmetric matrix whose lower triangle is in A (d x d,
// row-major with row stride ld, shared memory; an odd ld keeps the column reads free of
// bank conflicts), in working type T.  Pivot j is v_j = the (j, j) entry of the Schur
// complement; the update is A_il -= (A_ij / v_j) A_lj for j < l <= i, so column j keeps its
// unscaled values.  On return piv[j] = v_j and rs[j] = 1 / sqrt(v_j): Psi = U U^T with
// U_jj = sqrt(v_j), U_ij = A_ij rs[j] (i > j), and log|Psi| = sum_j log v_j.
//
// Blocked by panels of four pivots, so that the block meets two barriers per panel
// instead of two per pivot: warp 0 forms a panel's pivots, its scaled columns
// cols[q][i] = A_i,j0+q / v_j0+q and the updates inside the panel's columns; then every
// thread applies the panel's four rank-one updates to the rest of the lower triangle, in
// pivot order.  Every entry receives the same fused multiply-adds in the same order as in
// the unblocked algorithm, so the results are the same bits.
// A pivot v_j that is not above rel * dg[j] (rel = 0: not positive, or NaN) sets *fail
// (shared memory) and/or the device error word *derr (DPMM_ENUMERIC) and is replaced by
// the smallest normal value of T.  cols: 4 d values of T (shared memory), scratch.
template <typename T>
__device__ inline void chol_ldl_blk(T* A, int d, int ld, T* piv, T* rs, T* cols, const T* dg, T rel, int* fail,
                                    int* derr) {
    const int tid = threadIdx.x;
    for (int j0 = 0; j0 < d; j0 += 4) {
        const int pw = min(4, d - j0), j1 = j0 + pw;
        if (tid < 32) {
            for (int q = 0; q < pw; ++q) {
                const int j = j0 + q;
                T v = A[j * ld + j];
                if (!(v > (rel > T(0) ? rel * dg[j] : T(0)))) {
                    if (tid == 0) {
                        if (fail) *fail = 1;
                        if (derr) atomicExch(derr, (int)DPMM_ENUMERIC);
                    }
                    v = sizeof(T) == 4 ? T(1.17549435e-38f) : T(2.2250738585072014e-308);
                }
                const T r = rsqrt_t(v), inv = r * r;
                T* col = cols + (size_t)q * d;
                for (int i = j + 1 + tid; i < d; i += 32) col[i] = A[i * ld + j] * inv;
                if (tid == 0) {
                    piv[j] = v;
                    rs[j] = r;
                }
                __syncwarp();
                // the panel's later columns, every row at or below the column's diagonal
                for (int l = j + 1; l < j1; ++l) {
                    const T alj = A[l * ld + j];
                    for (int i = l + tid; i < d; i += 32) A[i * ld + l] = fma(-col[i], alj, A[i * ld + l]);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // the rest of the lower triangle: entries (i, l), j1 <= l <= i < d
        const int m = d - j1;
        for (int e = tid; e < m * (m + 1) / 2; e += blockDim.x) {
            int i, l;
            tri_index(e, i, l);
            i += j1;
            l += j1;
            T a = A[i * ld + l];
            for (int q = 0; q < pw; ++q) a = fma(-cols[(size_t)q * d + i], A[l * ld + j0 + q], a);
            A[i * ld + l] = a;
        }
        __syncthreads();
    }
}

// FP64, a non-positive pivot reported as DPMM_ENUMERIC (split/merge marginals).
__device__ inline void chol_ldl(double* A, int d, int ld, double* piv, double* rs, double* cols, int* derr) {
    chol_ldl_blk<double>(A, d, ld, piv, rs, cols, nullptr, 0.0, nullptr, derr);
}

// The factorisation above for the parameter draws of the reduced-precision paths (T =
// float) and their FP64 retry (T = double): with rel = 2^-10 an FP32 factorisation is
// flagged in *fail (and redone in FP64) once cancellation has taken more than 10 of the
// 24 bits of a pivot.
template <typename T>
__device__ inline void chol_ldl_t(T* A, int d, int ld, T* piv, T* rs, T* cols, const T* dg, T rel, int* fail) {
    chol_ldl_blk<T>(A, d, ld, piv, rs, cols, dg, rel, fail, nullptr);
}

}  // namespace dpmm
