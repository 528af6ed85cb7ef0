// k_sparse.cu -- the label step (Sec. 4.1 steps (e), (f); Eqs. sample_labels,
// sample_sub_labels) and the sufficient statistics of the multinomial model for
// high-dimensional count data (Sec. 5.3's document-word shapes: d up to 65,536), with
// the points held as compressed rows (CSR: per point its nonzero categories in
// increasing order and their counts).
//
// A document touches a few hundred of d = 20,000 categories, so a dense row would be
// read almost entirely as zeros; the compressed rows read only the nonzeros (8 bytes
// each), and the multinomial score sum_j x_ij log theta_kj is a sum over them.  Adding
// the zero terms changes no sum, so the FP64 path, which adds the nonzero terms in
// increasing j without fused multiply-adds, forms exactly the sums of a loop over all j.
//
//   sparse_sweep_kernel : one warp per point.  Mode 0: lane l scores clusters
//       l, l + 32, ... (cluster log theta stored transposed, category-major, so one
//       category's K values are contiguous), Gumbel-max over the clusters that can win
//       (exact: the others' score plus the largest Gumbel is below the best score plus
//       the smallest), then the two sub-cluster scores of the chosen cluster and z-bar;
//       mode 1: z-bar only; mode 2: neither.  Every mode adds the point's counts into
//       the compact count table of its sub-cluster (FP32, 2 K_max x d, read by the
//       parameter draws and the split/merge step) with atomic adds of integers (exact,
//       so the order of the additions does not matter).
//   sparse_zero_kernel  : clears the entries of the 2K sub-clusters those adds touch.
//   sparse_fill_kernel  : copies the compact counts into the FP64 statistics table.
//   csr_*               : the compressed rows of a dense input (count, scan, fill).
#include <math.h>

#include <cuda_bf16.h>

#include <algorithm>

#include "dpmm_internal.cuh"

namespace dpmm {

// ------------------------------------------------------------------ compressed rows
template <typename IN>
__device__ inline double in_val(const IN* p) { return (double)*p; }
template <>
__device__ inline double in_val<__nv_bfloat16>(const __nv_bfloat16* p) { return (double)__bfloat162float(*p); }

// per row (one warp): the number of nonzero entries; a negative or non-integer count
// sets *bad
template <typename IN>
__global__ void csr_count_kernel(const IN* X, int64_t N, int d, int* cnt, int* bad) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < N; i += nw) {
        int n = 0;
        for (int j = lane; j < d; j += 32) {
            const double v = in_val(X + i * d + j);
            if (!(v >= 0.0) || v != rint(v) || v > 16777216.0) *bad = 1;  // counts: integers, exact in FP32
            n += v != 0.0;
        }
        for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        if (lane == 0) cnt[i] = n;
    }
}

// exclusive prefix sum of cnt[0..N) into ptr[0..N] (one CTA of 1024 threads; runs once
// per data set)
__global__ void csr_scan_kernel(const int* cnt, int64_t N, int64_t* ptr) {
    __shared__ int64_t part[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < N; base += 1024) {
        const int64_t i = base + tid;
        int64_t v = i < N ? cnt[i] : 0, x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) part[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t p = part[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p += y;
            }
            part[lane] = p;
        }
        __syncthreads();
        const int64_t incl = x + (w > 0 ? part[w - 1] : 0) + carry;
        if (i < N) ptr[i] = incl - v;
        __syncthreads();
        if (tid == 1023) carry = incl;
        __syncthreads();
    }
    if (tid == 0) ptr[N] = carry;
}

// per row (one warp): the nonzeros in increasing category order
template <typename IN>
__global__ void csr_fill_kernel(const IN* X, int64_t N, int d, const int64_t* ptr, int* idx, int* val) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < N; i += nw) {
        int64_t pos = ptr[i];
        for (int j0 = 0; j0 < d; j0 += 32) {
            const int j = j0 + lane;
            const double v = j < d ? in_val(X + i * d + j) : 0.0;
            const unsigned m = __ballot_sync(0xffffffffu, v != 0.0);
            if (v != 0.0) {
                const int64_t q = pos + __popc(m & ((1u << lane) - 1u));
                idx[q] = j;
                val[q] = (int)v;
            }
            pos += __popc(m);
        }
    }
}

// ------------------------------------------------------------------ parameters
// cluster log theta, category-major: lt_t[j * ks + k] = log theta_{3k, j}; c_t[k] = log pi_k
template <typename T>
__global__ void sparse_ltT_kernel(const int* dK, int d, int ks, const double* p_logtheta, const double* p_c, T* lt_t,
                                  T* c_t) {
    const int K = *dK;
    const int64_t total = (int64_t)d * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / K), k = (int)(e % K);
        lt_t[(size_t)j * ks + k] = (T)p_logtheta[(size_t)3 * k * d + j];
    }
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < K; k += blockDim.x) c_t[k] = (T)p_c[3 * k];
}

// ------------------------------------------------------------------ arithmetic
// FP64: multiply and add rounded separately (a loop over all j in C does the same);
// FP32: fused
__device__ inline double madd(double acc, double c, double l) { return __dadd_rn(acc, __dmul_rn(c, l)); }
__device__ inline float madd(float acc, float c, float l) { return fmaf(c, l, acc); }

template <typename T>
__device__ inline T gumbel_sp(uint32_t a, uint32_t b);
template <>
__device__ inline double gumbel_sp<double>(uint32_t a, uint32_t b) { return -log(-log(u01_f64(a, b))); }
template <>
__device__ inline float gumbel_sp<float>(uint32_t a, uint32_t) { return -__logf(-logf(u01_f32(a))); }
// a cluster whose score is more than WIN below the best cannot win: WIN >= the largest
// minus the smallest Gumbel value the uniforms allow (FP64: 36.74 + 3.61; FP32:
// 16.64 + 2.82), rounded up
template <typename T>
__device__ inline T gwin();
template <>
__device__ inline double gwin<double>() { return 41.0; }
template <>
__device__ inline float gwin<float>() { return 20.5f; }

template <typename T>
struct SpArgs {
    int64_t N;
    int d, ks, mode;
    const int64_t* ptr;
    const int* idx;
    const int* val;
    const T* lt_t;          // d x ks, cluster slots
    const T* c_t;           // K: log pi_k
    const double* p_logtheta;  // slots x d (sub-cluster scores, FP64 table)
    const float* q_logtheta;   // slots x d (FP32 mirror)
    const double* p_c;
    const int* dK;
    const uint32_t* diter;
    uint64_t seed;
    const int* gate;
    int32_t* z;
    uint8_t* zbar;
    double* S;              // statistics table (FIRST layout)
    StatLayout L;
    float* cc;              // 2 K_max x d compact counts
    double* scores;         // optional N x K (test hook)
};

template <typename T>
__device__ inline const T* slot_lt(const SpArgs<T>& a, int s);
template <>
__device__ inline const double* slot_lt<double>(const SpArgs<double>& a, int s) { return a.p_logtheta + (size_t)s * a.d; }
template <>
__device__ inline const float* slot_lt<float>(const SpArgs<float>& a, int s) { return a.q_logtheta + (size_t)s * a.d; }

constexpr int SP_WARPS = 8;  // warps per CTA (256 threads)
constexpr int SP_DEPTH = 16; // table rows in flight per lane in the cluster-score loop

template <typename T, int KQ>
__global__ void __launch_bounds__(256) sparse_sweep_kernel(SpArgs<T> a) {
    if (a.gate && *a.gate == 0) return;
    // per warp: the (category, count) pairs of 32 nonzeros, read back as broadcasts
    __shared__ int2 pairs[SP_WARPS][32];
    const int K = *a.dK;
    const int lane = threadIdx.x & 31;
    int2* pr = pairs[threadIdx.x >> 5];
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const Key key{a.seed, a.diter[0], a.diter[1], a.diter[2]};
    for (int64_t i = w0; i < a.N; i += nw) {
        const int64_t r0 = a.ptr[i], r1 = a.ptr[i + 1];
        int zi, hi = 0;
        if (a.mode == 0 || a.mode == 3) {
            T acc[KQ];
#pragma unroll
            for (int q = 0; q < KQ; ++q) acc[q] = T(0);
            for (int64_t p0 = r0; p0 < r1; p0 += 32) {
                const int n = (int)min((int64_t)32, r1 - p0);
                __syncwarp();
                if (lane < n) pr[lane] = make_int2(a.idx[p0 + lane], a.val[p0 + lane]);
                __syncwarp();
#pragma unroll
                for (int u = 0; u < KQ; ++u) {
                    if (32 * u >= K) break;
                    // lane k reads log theta_{k, j_q} (the table is category-major: one
                    // category's K values are contiguous, so the warp reads one row segment
                    // per nonzero); SP_DEPTH nonzeros' reads are issued before they are added,
                    // and the additions run in increasing q: those of a loop over the
                    // nonzeros one at a time
                    const int k = lane + 32 * u;
                    const bool on = k < K;
                    const T* col = a.lt_t + k;
                    T sk = acc[u];
                    for (int q0 = 0; q0 < n; q0 += SP_DEPTH) {
                        T lv[SP_DEPTH];
                        int cq[SP_DEPTH];
#pragma unroll
                        for (int v = 0; v < SP_DEPTH; ++v) {
                            const int2 jc = pr[min(q0 + v, n - 1)];
                            cq[v] = jc.y;
                            lv[v] = on ? col[(size_t)jc.x * a.ks] : T(0);
                        }
#pragma unroll
                        for (int v = 0; v < SP_DEPTH; ++v)
                            if (q0 + v < n) sk = madd(sk, (T)cq[v], lv[v]);
                    }
                    acc[u] = sk;
                }
            }
        // scores log pi_k + log f(x_i; theta_k) and the exact Gumbel-max
            T sc[KQ], best = -INFINITY;
#pragma unroll
            for (int u = 0; u < KQ; ++u) {
                const int k = lane + 32 * u;
                sc[u] = k < K ? a.c_t[k] + acc[u] : (T)-INFINITY;
                if (a.scores && k < K) a.scores[i * K + k] = (double)sc[u];
                best = sc[u] > best ? sc[u] : best;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, o);
                best = ob > best ? ob : best;
            }
            const T lim = best - gwin<T>();
            T vb = -INFINITY;
            int kb = 0x7fffffff;
#pragma unroll
            for (int u = 0; u < KQ; ++u) {
                const int k = lane + 32 * u;
                if (k < K && sc[u] >= lim) {
                    uint32_t w[4];
                    key.block((uint32_t)i, TAG_Z, (uint32_t)(k >> 1), w);
                    const T v = sc[u] + ((k & 1) ? gumbel_sp<T>(w[2], w[3]) : gumbel_sp<T>(w[0], w[1]));
                    if (v > vb) {  // k increases along u: ties keep the lower index
                        vb = v;
                        kb = k;
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {  // argmax, ties to the lower cluster index
                const T ov = __shfl_xor_sync(0xffffffffu, vb, o);
                const int ok = __shfl_xor_sync(0xffffffffu, kb, o);
                if (ov > vb || (ov == vb && ok < kb)) {
                    vb = ov;
                    kb = ok;
                }
            }
            zi = kb < K ? kb : 0;
            if (lane == 0) a.z[i] = zi;
            if (a.mode == 3) continue;  // labels only (the score hook)
        } else {
            zi = a.z[i];
        }
        if ((unsigned)zi >= (unsigned)K) continue;  // never for consistent labels
        if (a.mode <= 1) {
            // the two sub-cluster scores of cluster zi: sequential on lane 0 for FP64 (the
            // sum in increasing j, as over all j), lane-parallel for FP32
            const T* ll = slot_lt<T>(a, 3 * zi + 1);
            const T* lr = slot_lt<T>(a, 3 * zi + 2);
            T sl = T(0), sr = T(0);
            if (sizeof(T) == 8) {
                // lane q loads its nonzero's two values; every lane then adds them in
                // increasing q (the order of the loop over all j), so lane 0 holds the sums
                for (int64_t p0 = r0; p0 < r1; p0 += 32) {
                    const int n = (int)min((int64_t)32, r1 - p0);
                    T c = T(0), vl = T(0), vr = T(0);
                    if (lane < n) {
                        const int j = a.idx[p0 + lane];
                        c = (T)a.val[p0 + lane];
                        vl = ll[j];
                        vr = lr[j];
                    }
                    for (int q = 0; q < n; ++q) {
                        const T cq = __shfl_sync(0xffffffffu, c, q);
                        sl = madd(sl, cq, __shfl_sync(0xffffffffu, vl, q));
                        sr = madd(sr, cq, __shfl_sync(0xffffffffu, vr, q));
                    }
                }
            } else {
                // lane-parallel partial sums, eight nonzeros' loads in flight per lane
                for (int64_t p0 = r0 + lane; p0 < r1; p0 += 256) {
                    T c[8], tl[8], tr[8];
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const int64_t p = p0 + 32 * v;
                        c[v] = T(0);
                        tl[v] = tr[v] = T(0);
                        if (p < r1) {
                            const int j = a.idx[p];
                            c[v] = (T)a.val[p];
                            tl[v] = ll[j];
                            tr[v] = lr[j];
                        }
                    }
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        if (p0 + 32 * v < r1) {
                            sl = madd(sl, c[v], tl[v]);
                            sr = madd(sr, c[v], tr[v]);
                        }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    sl += __shfl_xor_sync(0xffffffffu, sl, o);
                    sr += __shfl_xor_sync(0xffffffffu, sr, o);
                }
            }
            if (lane == 0) {
                uint32_t w[4];
                key.block((uint32_t)i, TAG_ZBAR, 0u, w);
                const T vl = ((T)a.p_c[3 * zi + 1] + sl) + gumbel_sp<T>(w[0], w[1]);
                const T vr = ((T)a.p_c[3 * zi + 2] + sr) + gumbel_sp<T>(w[2], w[3]);
                hi = vr > vl ? 1 : 0;
                a.zbar[i] = (uint8_t)hi;
            }
            hi = __shfl_sync(0xffffffffu, hi, 0);
        } else {
            hi = a.zbar[i] ? 1 : 0;
        }
        // statistics: integer counts, exact in any order, added to the compact table (FP32,
        // exact up to 2^24 per entry); sparse_fill_kernel copies it into the FP64 table
        const int s = 2 * zi + hi;
        float* cs = a.cc + (size_t)s * a.d;
        for (int64_t p0 = r0 + lane; p0 < r1; p0 += 256) {
            int j[8], v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t p = p0 + 32 * u;
                j[u] = p < r1 ? a.idx[p] : -1;
                v[u] = p < r1 ? a.val[p] : 0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (j[u] >= 0) atomicAdd(cs + j[u], (float)v[u]);
        }
        if (lane == 0) atomicAdd(a.S + (size_t)s * a.L.E + a.L.ent(a.d, a.d), 1.0);
    }
}

// the entries the adds above touch, for the 2K sub-clusters (grid: y = sub-cluster slot,
// 2 K_max rows; x strides over the d + 1 entries of a slot)
__global__ void sparse_zero_kernel(const int* dK, const int* gate, StatLayout L, double* S, float* cc) {
    if (gate && *gate == 0) return;
    const int s = blockIdx.y, d = L.d;
    if (s >= 2 * *dK) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= d; j += gridDim.x * blockDim.x) {
        S[(size_t)s * L.E + L.ent(j, d)] = 0.0;
        if (j < d) cc[(size_t)s * d + j] = 0.f;
    }
}

// the FP64 statistics of the 2K sub-clusters from the compact counts (exact: integers)
__global__ void sparse_fill_kernel(const int* dK, const int* gate, StatLayout L, double* S, const float* cc) {
    if (gate && *gate == 0) return;
    const int s = blockIdx.y, d = L.d;
    if (s >= 2 * *dK) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x)
        S[(size_t)s * L.E + L.ent(j, d)] = (double)cc[(size_t)s * d + j];
}

// x blocks of the zero and fill grids: enough 256-thread blocks to cover a slot's entries
static dim3 slot_grid(const dpmm_ctx* c) {
    return dim3((unsigned)std::min(16, (c->d + 1 + 255) / 256), (unsigned)(2 * c->K_max));
}

// ------------------------------------------------------------------ host
bool sparse_path(const dpmm_ctx* c) { return c->kind == DPMM_PRIOR_DIRICHLET && c->d > SPARSE_MIN_D; }

template <typename IN>
static cudaError_t build_csr_t(dpmm_ctx* c, const IN* X, int* bad) {
    const int64_t N = c->N;
    int* cnt = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&cnt, sizeof(int) * N, c->stream);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>((N + 7) / 8, 8 * (int64_t)c->num_sms);
    csr_count_kernel<IN><<<grid, 256, 0, c->stream>>>(X, N, c->d, cnt, bad);
    csr_scan_kernel<<<1, 1024, 0, c->stream>>>(cnt, N, c->csr_ptr);
    cudaFreeAsync(cnt, c->stream);
    int64_t nnz = 0;
    e = cudaMemcpyAsync(&nnz, c->csr_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    if (c->csr_idx) cudaFree(c->csr_idx);
    if (c->csr_val) cudaFree(c->csr_val);
    c->csr_idx = c->csr_val = nullptr;
    c->nnz = nnz;
    e = cudaMalloc((void**)&c->csr_idx, sizeof(int) * std::max<int64_t>(nnz, 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->csr_val, sizeof(int) * std::max<int64_t>(nnz, 1));
    if (e != cudaSuccess) return e;
    csr_fill_kernel<IN><<<grid, 256, 0, c->stream>>>(X, N, c->d, c->csr_ptr, c->csr_idx, c->csr_val);
    c->nlaunch += 3;
    return cudaGetLastError();
}

cudaError_t sparse_build_dense(dpmm_ctx* c, const void* X, dpmm_dtype dt, int* bad) {
    switch (dt) {
        case DPMM_F64: return build_csr_t(c, (const double*)X, bad);
        case DPMM_F32: return build_csr_t(c, (const float*)X, bad);
        case DPMM_BF16: return build_csr_t(c, (const __nv_bfloat16*)X, bad);
        default: return build_csr_t(c, (const int32_t*)X, bad);
    }
}

cudaError_t sparse_prepare(dpmm_ctx* c) {
    const bool f64 = c->prec == DPMM_PREC_FP64_PLAIN;
    const int ks = (c->K_max + 31) / 32 * 32;
    const int grid = 4 * c->num_sms;
    prof_begin(c, "derive_sparse");
    if (f64)
        sparse_ltT_kernel<double><<<grid, 256, 0, c->stream>>>(c->dK, c->d, ks, c->p_logtheta, c->p_c,
                                                              (double*)c->sp_ltT, (double*)c->sp_ct);
    else
        sparse_ltT_kernel<float><<<grid, 256, 0, c->stream>>>(c->dK, c->d, ks, c->p_logtheta, c->p_c,
                                                             (float*)c->sp_ltT, (float*)c->sp_ct);
    prof_end(c, "derive_sparse");
    c->nlaunch += 1;
    return cudaGetLastError();
}

template <typename T, int KQ>
static cudaError_t launch_sp(dpmm_ctx* c, const SpArgs<T>& a, int grid) {
    sparse_sweep_kernel<T, KQ><<<grid, 32 * SP_WARPS, 0, c->stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t sparse_sweep_t(dpmm_ctx* c, uint64_t seed, int mode, const int* gate) {
    SpArgs<T> a;
    a.N = c->N;
    a.d = c->d;
    a.ks = (c->K_max + 31) / 32 * 32;
    a.mode = mode;
    a.ptr = c->csr_ptr;
    a.idx = c->csr_idx;
    a.val = c->csr_val;
    a.lt_t = (const T*)c->sp_ltT;
    a.c_t = (const T*)c->sp_ct;
    a.p_logtheta = c->p_logtheta;
    a.q_logtheta = c->q_logtheta;
    a.p_c = c->p_c;
    a.dK = c->dK;
    a.diter = c->diter;
    a.seed = seed;
    a.gate = gate;
    a.z = c->z;
    a.zbar = c->zbar;
    a.S = c->stats;
    a.L = c->st;
    a.cc = c->sp_cc;
    a.scores = (mode == 0 || mode == 3) ? c->dbg_scores : nullptr;
    const int grid = (int)std::min<int64_t>((c->N + 7) / 8, 16 * (int64_t)c->num_sms);
    const int kq = (c->K_max + 31) / 32;
    if (kq <= 1) return launch_sp<T, 1>(c, a, grid);
    if (kq <= 2) return launch_sp<T, 2>(c, a, grid);
    if (kq <= 4) return launch_sp<T, 4>(c, a, grid);
    return launch_sp<T, 8>(c, a, grid);
}

// mode 0: labels, sub-labels and statistics; 1: sub-labels and statistics; 2: statistics;
// 3: labels only (no statistics)
cudaError_t launch_sparse(dpmm_ctx* c, uint64_t seed, int mode, const int* gate) {
    const char* name = mode == 0 ? "labels_sparse" : (mode == 1 ? "substats_sparse" : (mode == 2 ? "restats_sparse" : "labels_sparse"));
    cudaError_t e = cudaSuccess;
    if (mode != 3) {
        prof_begin(c, "zero_sparse");
        sparse_zero_kernel<<<slot_grid(c), 256, 0, c->stream>>>(c->dK, gate, c->st, c->stats, c->sp_cc);
        prof_end(c, "zero_sparse");
        c->nlaunch += 1;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    prof_begin(c, name);
    e = c->prec == DPMM_PREC_FP64_PLAIN ? sparse_sweep_t<double>(c, seed, mode, gate)
                                        : sparse_sweep_t<float>(c, seed, mode, gate);
    prof_end(c, name);
    c->nlaunch += 1;
    if (e != cudaSuccess || mode == 3) return e;
    prof_begin(c, "fill_sparse");
    sparse_fill_kernel<<<slot_grid(c), 256, 0, c->stream>>>(c->dK, gate, c->st, c->stats, c->sp_cc);
    prof_end(c, "fill_sparse");
    c->nlaunch += 1;
    return cudaGetLastError();
}

}  // namespace dpmm
