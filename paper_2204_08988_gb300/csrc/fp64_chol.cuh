// fp64_chol.cuh -- FP64 building blocks of the parameter and split/merge steps: staging a
// (sub-)cluster's statistics block in shared memory and a right-looking Cholesky
// factorisation written for GB300's FP64 pipe (about two operations per clock per SM,
// 64-cycle dependent latency): the only serial work per pivot is one reciprocal square
// root; the trailing update (balanced row pairs) has no square roots or divisions in its
// indexing and issues its loads in batches so that independent FMAs overlap.
#pragma once
#include "dpmm_internal.cuh"

namespace dpmm {

// out[e] = statistics entry e of slot (k, h) of the table S (E entries per sub-cluster);
// h = -1 sums the two sub-clusters (the cluster).  Every thread of the block calls it.
__device__ inline void stage_slot(const double* S, int E, int k, int h, double* out) {
    const double* s0 = S + (size_t)(2 * k + (h < 0 ? 0 : h)) * E;
    const double* s1 = S + (size_t)(2 * k + 1) * E;
    for (int e = threadIdx.x; e < E; e += blockDim.x) out[e] = h < 0 ? s0[e] + s1[e] : s0[e];
}

// Row i0 and column l0 (l0 <= i0) of entry e of a lower triangle enumerated row by row.
__device__ inline void tri_index(int e, int& i0, int& l0) {
    int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    if ((i + 1) * (i + 2) / 2 <= e) ++i;
    if (i * (i + 1) / 2 > e) --i;
    i0 = i;
    l0 = e - i * (i + 1) / 2;
}

// Trailing update of pivot j: A_il -= col_i A_lj for j < l <= i < d.  Rows are taken in
// pairs (j + 1 + p, d - 1 - p), which together hold m + 1 entries (m = d - j - 1), so every
// pair carries the same work; each pair is split over S threads (entries s, s + S, ...,
// consecutive threads on consecutive columns of a row), and each thread keeps four
// entries' loads in flight.  No index needs a square root or a division.  Every entry
// gets the single FMA fma(-col_i, A_lj, A_il), as in any enumeration order.
template <typename T>
__device__ inline void chol_update(T* A, int d, int ld, int j, const T* col) {
    const int m = d - j - 1;
    if (m <= 0) return;
    const int np = (m + 1) >> 1, nt = blockDim.x;
    int S = nt / np;
    S = S < 1 ? 1 : (S > 8 ? 8 : S);
    for (int w = threadIdx.x; w < np * S; w += nt) {
        const int p = w / S, s = w - p * S;
        const int r1 = j + 1 + p, r2 = d - 1 - p;
        const int n1 = r1 - j, n = r2 > r1 ? n1 + (r2 - j) : n1;
        const T c1 = col[r1], c2 = col[r2];
        for (int e0 = s; e0 < n; e0 += 4 * S) {
            T av[4], cl[4];
            int at[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * S;
                at[u] = -1;
                if (e < n) {
                    const bool first = e < n1;
                    const int i = first ? r1 : r2, l = j + 1 + (first ? e : e - n1);
                    at[u] = i * ld + l;
                    av[u] = A[at[u]];
                    cl[u] = A[l * ld + j];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * S;
                if (at[u] >= 0) A[at[u]] = fma(-(e < n1 ? c1 : c2), cl[u], av[u]);
            }
        }
    }
}

// In-place factorisation of the symmetric matrix whose lower triangle is in A (d x d,
// row-major with row stride ld, shared memory; an odd ld keeps the column reads free of
// bank conflicts).  Pivot j is v_j = the (j, j) entry of the Schur complement;
// the update is A_il -= (A_ij / v_j) A_lj for j < l <= i, so column j keeps its unscaled
// values.  On return piv[j] = v_j and rs[j] = 1 / sqrt(v_j): Psi = U U^T with
// U_jj = sqrt(v_j), U_ij = A_ij rs[j] (i > j), and log|Psi| = sum_j log v_j.  A pivot
// that is not positive (or NaN) sets *derr = DPMM_ENUMERIC and is replaced by 1e-300.
// col (d doubles of shared memory) is scratch.  Every thread of the block calls it; two
// barriers per pivot.  Each FP64 warp instruction costs the pipe about the same whether
// or not its lanes are busy, so warp 0 forms the pivot and the scaled column (one lane
// per row) and the update touches only the lower triangle, one FMA per entry.
__device__ inline void chol_ldl(double* A, int d, int ld, double* piv, double* rs, double* col, int* derr) {
    const int tid = threadIdx.x;
    for (int j = 0; j < d; ++j) {
        if (tid < 32) {
            double v = A[j * ld + j];
            if (!(v > 0.0)) {
                if (tid == 0) atomicExch(derr, (int)DPMM_ENUMERIC);
                v = 1e-300;
            }
            const double r = rsqrt(v), inv = r * r;
            for (int i = j + 1 + tid; i < d; i += 32) col[i] = A[i * ld + j] * inv;
            if (tid == 0) {
                piv[j] = v;
                rs[j] = r;
            }
        }
        __syncthreads();
        chol_update<double>(A, d, ld, j, col);
        __syncthreads();
    }
}

__device__ inline float rsqrt_t(float x) { return rsqrtf(x); }
__device__ inline double rsqrt_t(double x) { return rsqrt(x); }

// The factorisation above in working type T, for the parameter draws of the reduced-
// precision paths (T = float) and their FP64 retry (T = double).  A pivot v_j that is not
// above rel * dg[j] (dg: the matrix's own diagonal; rel = 0: not positive, or NaN) sets
// *fail (shared memory) and is replaced by the smallest normal value of T, so that the
// caller can redo the slot in FP64.  With rel = 2^-10 an FP32 factorisation is redone
// once cancellation has taken more than 10 of the 24 bits of a pivot.
template <typename T>
__device__ inline void chol_ldl_t(T* A, int d, int ld, T* piv, T* rs, T* col, const T* dg, T rel, int* fail) {
    const int tid = threadIdx.x;
    for (int j = 0; j < d; ++j) {
        if (tid < 32) {
            T v = A[j * ld + j];
            if (!(v > (rel > T(0) ? rel * dg[j] : T(0)))) {
                if (tid == 0) *fail = 1;
                v = sizeof(T) == 4 ? T(1.17549435e-38f) : T(2.2250738585072014e-308);
            }
            const T r = rsqrt_t(v), inv = r * r;
            for (int i = j + 1 + tid; i < d; i += 32) col[i] = A[i * ld + j] * inv;
            if (tid == 0) {
                piv[j] = v;
                rs[j] = r;
            }
        }
        __syncthreads();
        chol_update<T>(A, d, ld, j, col);
        __syncthreads();
    }
}

}  // namespace dpmm
