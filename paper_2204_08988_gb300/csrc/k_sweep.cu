// k_sweep.cu -- the label step and the sufficient statistics (Sec. 4.1 steps (e),
// (f); Sec. 4.4 "updating the sufficient statistics" in three steps).
//
//   labels_simt  : z_i = argmax_k [log pi_k + log f(x_i; theta_k) + G_ik] on CUDA
//                  cores (FP64 parity path, FP32 for small d), one thread per point,
//                  cluster parameters staged in shared memory and read by broadcast.
//   hist/scan/scatter : stable counting sort of the points by cluster (tiles of 256
//                  points), so that the next kernel sees each cluster as one run.
//   substats     : per sorted run, z-bar_i from the two sub-clusters of z_i, then the
//                  per-sub-cluster sums of xt xt^T (xt = [x - shift_k, 1]) as 4x4
//                  register blocks, one partial record per (CTA, cluster) run.
//   combine      : sums each cluster's records in CTA order (deterministic).
#include <math.h>

#include <cuda_bf16.h>

#include <algorithm>

#include "dpmm_internal.cuh"

namespace dpmm {

template <typename T, typename XT>
__device__ inline T ldx(const XT* p) { return (T)(*p); }
template <>
__device__ inline float ldx<float, __nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <typename T>
struct ParamView {
    const T* W;      // slots x d x d
    const T* mu;     // slots x d
    const T* c;      // slots
    const T* lt;     // slots x d (multinomial)
};

template <typename T>
__device__ inline T gumbel_of(uint32_t w0, uint32_t w1);
template <>
__device__ inline double gumbel_of<double>(uint32_t a, uint32_t b) {
    return -log(-log(u01_f64(a, b)));
}
template <>
__device__ inline float gumbel_of<float>(uint32_t a, uint32_t) {
    // the inner log must be accurate near u = 1 (-log u is as small as 6e-8 there)
    return -__logf(-logf(u01_f32(a)));
}
template <typename T>
__device__ inline T gmax();
template <>
__device__ inline double gmax<double>() { return GUMBEL_MAX_F64; }
template <>
__device__ inline float gmax<float>() { return GUMBEL_MAX_F32; }

// ------------------------------------------------------------------ labels (simt)
// Dynamic shared memory: CB clusters x (d*d + d + 1) T (d + 1 for multinomial), then
// blockDim x (d + 1) T point rows.
template <typename T, typename XT, bool SCORES>
__global__ void __launch_bounds__(256) labels_simt_kernel(int kind, int d, int xs, int64_t N, const XT* __restrict__ X,
                                                          ParamView<T> pv, const int* dK, const uint32_t* diter,
                                                          uint64_t seed, int CB, const int* gate,
                                                          double* scores, int32_t* z) {
    if (gate && *gate == 0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sW = (T*)smraw;
    const int per = kind == DPMM_PRIOR_NIW ? d * d + d + 1 : d + 1;
    T* sx = sW + (size_t)CB * per;
    const int K = *dK;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t ntiles = (N + nt - 1) / nt;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {  // grid-stride over point tiles
    __syncthreads();
    const int64_t i = tile * nt + tid;
    const bool live = i < N;
    T* xr = sx + (size_t)tid * (d + 1);
    if (live)
        for (int j = 0; j < d; ++j) xr[j] = ldx<T, XT>(X + i * xs + j);
    Key key{seed, diter[0], diter[1], diter[2]};
    T best = -INFINITY;
    int zb = 0;
    uint32_t w[4];
    int wblk = -1;
    for (int k0 = 0; k0 < K; k0 += CB) {
        const int nc = min(CB, K - k0);
        __syncthreads();
        for (int e = tid; e < nc * per; e += nt) {
            int cc = e / per, r = e % per;
            int s = 3 * (k0 + cc);
            T v;
            if (kind == DPMM_PRIOR_NIW) {
                if (r < d * d) v = pv.W[(size_t)s * d * d + r];
                else if (r < d * d + d) v = pv.mu[(size_t)s * d + (r - d * d)];
                else v = pv.c[s];
            } else {
                v = (r < d) ? pv.lt[(size_t)s * d + r] : pv.c[s];
            }
            sW[e] = v;
        }
        __syncthreads();
        if (!live) continue;
        for (int cc = 0; cc < nc; ++cc) {
            const T* Wk = sW + (size_t)cc * per;
            T sc;
            if (kind == DPMM_PRIOR_NIW) {
                const T* mk = Wk + d * d;
                T q = 0;
                for (int j = 0; j < d; ++j) {
                    T y = 0;
                    for (int l = 0; l <= j; ++l) y += Wk[l * d + j] * (xr[l] - mk[l]);
                    q += y * y;
                }
                sc = Wk[d * d + d] - (T)0.5 * q;
            } else {
                T a = 0;
                for (int j = 0; j < d; ++j) a += xr[j] * Wk[j];
                sc = Wk[d] + a;
            }
            const int k = k0 + cc;
            if constexpr (SCORES) scores[i * K + k] = (double)sc;
            if (sc + gmax<T>() > best) {  // otherwise k cannot win the argmax
                if ((k >> 1) != wblk) {
                    key.block((uint32_t)i, TAG_Z, (uint32_t)(k >> 1), w);
                    wblk = k >> 1;
                }
                T g = (k & 1) ? gumbel_of<T>(w[2], w[3]) : gumbel_of<T>(w[0], w[1]);
                T v = sc + g;
                if (v > best) {
                    best = v;
                    zb = k;
                }
            }
        }
    }
    if (live) z[i] = zb;
    }
}

// ------------------------------------------------------------------ counting sort
// Stable counting sort of the points by cluster (the order the statistics step visits
// them in), in tiles of SORT_TILE points: four rounds of 256, one point per thread per
// round, so that a tile's points are ranked in index order (round, warp, lane).
__global__ void hist_kernel(const int32_t* z, int64_t N, int T_tiles, int Kmax, const int* gate, int* hist) {
    if (gate && *gate == 0) return;
    extern __shared__ int cnt[];
    const int t = blockIdx.x;
    for (int k = threadIdx.x; k < Kmax; k += blockDim.x) cnt[k] = 0;
    int zq[SORT_TILE / 256];
#pragma unroll
    for (int q = 0; q < SORT_TILE / 256; ++q) {
        const int64_t i = (int64_t)t * SORT_TILE + q * 256 + threadIdx.x;
        zq[q] = i < N ? z[i] : -1;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < SORT_TILE / 256; ++q)
        if ((unsigned)zq[q] < (unsigned)Kmax) atomicAdd(&cnt[zq[q]], 1);  // labels are always in range
    __syncthreads();
    for (int k = threadIdx.x; k < Kmax; k += blockDim.x) hist[(size_t)k * T_tiles + t] = cnt[k];
}

// Exclusive scan of each cluster's row of tile counts (block k), row total into tot[k];
// the last block to finish turns the totals into the clusters' starts (exclusive prefix,
// tot[K] = N) and re-arms the counter *done for the next launch.
__global__ void scan_kernel(int* hist, int T_tiles, const int* dK, const int* gate, int* tot, int* done) {
    if (gate && *gate == 0) return;
    const int k = blockIdx.x, K = *dK;
    __shared__ int wsum[32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (k < K) {
        int* row = hist + (size_t)k * T_tiles;
        const int per = (T_tiles + blockDim.x - 1) / blockDim.x;
        const int a = threadIdx.x * per, b = min(T_tiles, a + per);
        int s = 0;
        for (int t = a; t < b; ++t) s += row[t];
        // block exclusive scan of s
        int x = s;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int nw = blockDim.x >> 5;
            int v = lane < nw ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            if (lane < nw) wsum[lane] = v;
        }
        __syncthreads();
        int excl = x - s + (w > 0 ? wsum[w - 1] : 0);
        for (int t = a; t < b; ++t) {
            int v = row[t];
            row[t] = excl;
            excl += v;
        }
        if (threadIdx.x == blockDim.x - 1) {
            tot[k] = excl;
            __threadfence();
        }
    } else if (threadIdx.x == 0) {
        tot[k] = 0;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || w != 0) return;
    __threadfence();
    int acc = 0;
    for (int k0 = 0; k0 < K; k0 += 32) {
        const int v = k0 + lane < K ? __ldcg(tot + k0 + lane) : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (k0 + lane < K) tot[k0 + lane] = acc + x - v;
        acc += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) {
        tot[K] = acc;
        *done = 0;
    }
}

__global__ void scatter_kernel(const int32_t* z, int64_t N, int T_tiles, const int* hist, const int* starts,
                               const int* gate, int Kmax, int* idx) {
    if (gate && *gate == 0) return;
    extern __shared__ int wc[];  // 8 warps x Kmax counts of the round, then Kmax running bases
    int* base = wc + 8 * Kmax;
    const int t = blockIdx.x;
    for (int e = threadIdx.x; e < 8 * Kmax; e += blockDim.x) wc[e] = 0;
    for (int k = threadIdx.x; k < Kmax; k += blockDim.x) base[k] = starts[k] + hist[(size_t)k * T_tiles + t];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int zq[SORT_TILE / 256];
#pragma unroll
    for (int q = 0; q < SORT_TILE / 256; ++q) {
        const int64_t i = (int64_t)t * SORT_TILE + q * 256 + threadIdx.x;
        zq[q] = i < N ? z[i] : -1;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < SORT_TILE / 256; ++q) {
        const int64_t i = (int64_t)t * SORT_TILE + q * 256 + threadIdx.x;
        const bool live = (unsigned)zq[q] < (unsigned)Kmax;  // labels are always in range
        const int k = live ? zq[q] : -1 - lane;             // dead lanes never match live ones
        const unsigned m = __match_any_sync(0xffffffffu, k);
        const int r = __popc(m & ((1u << lane) - 1u));
        if (live && r == 0) wc[w * Kmax + k] = __popc(m);
        __syncthreads();
        if (live) {
            int before = 0;
            for (int v = 0; v < w; ++v) before += wc[v * Kmax + k];
            idx[base[k] + before + r] = (int)i;
        }
        __syncthreads();
        // the bases move past this round's points; the counts are cleared for the next
        for (int kk = threadIdx.x; kk < Kmax; kk += blockDim.x) {
            int s = 0;
            for (int v = 0; v < 8; ++v) {
                s += wc[v * Kmax + kk];
                wc[v * Kmax + kk] = 0;
            }
            base[kk] += s;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ sub-labels + stats
// Starts of the runs of equal labels among kq[0..np) (np <= blockDim), by warp ballots:
// runs[0..n) are the starts, runs[n] = np, *nruns = n.  All threads must call it.
__device__ inline void find_runs(const int* kq, int np, int* runs, int* nruns, int* wcnt) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = (blockDim.x + 31) >> 5;
    const bool f = tid < np && (tid == 0 || kq[tid] != kq[tid - 1]);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[w] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int v = 0; v < nw; ++v) {
        if (v < w) before += wcnt[v];
        total += wcnt[v];
    }
    if (f) runs[before + __popc(m & ((1u << lane) - 1u))] = tid;
    if (tid == 0) {
        runs[total] = np;
        *nruns = total;
    }
    __syncthreads();
}


template <typename T>
struct SubArgs {
    int kind, d, xs;
    int64_t N;
    const void* X;
    ParamView<T> pv;
    const T* shift;  // K_max x d, storage coordinates
    const int32_t* z;
    uint8_t* zbar;
    const int* idx;
    const int* dK;
    const uint32_t* diter;
    const int* gate;
    uint64_t seed;
    int draw;        // 1: draw z-bar; 0: keep
    int P;           // points per tile
    int G;           // point groups per block
    int64_t R;       // points per CTA
    StatLayout L;
    double* rec;     // (G2 + K_max) x 2 x E
};

template <typename T, typename XT>
__device__ inline T sub_score(const SubArgs<T>& a, int s, const T* xr) {
    const int d = a.d;
    if (a.kind == DPMM_PRIOR_NIW) {
        const T* W = a.pv.W + (size_t)s * d * d;
        const T* mu = a.pv.mu + (size_t)s * d;
        T q = 0;
        for (int j = 0; j < d; ++j) {
            T y = 0;
            for (int l = 0; l <= j; ++l) y += __ldg(W + l * d + j) * (xr[l] - __ldg(mu + l));
            q += y * y;
        }
        return __ldg(a.pv.c + s) - (T)0.5 * q;
    }
    const T* lt = a.pv.lt + (size_t)s * d;
    T acc = 0;
    for (int j = 0; j < d; ++j) acc += xr[j] * __ldg(lt + j);
    return __ldg(a.pv.c + s) + acc;
}

// Dynamic shared memory: P x dp T (point rows), P ints (k), P bytes (h), then the
// flush buffer G x nblk x 32 T.
template <typename T, typename XT, int MAXT>
__global__ void __launch_bounds__(MAXT) substats_kernel(SubArgs<T> a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int d = a.d, dp = a.L.dp, P = a.P, G = a.G, nblk = a.L.nblk;
    T* xs = (T*)smraw;
    int* kq = (int*)(xs + (size_t)P * dp);
    int* runs = kq + P;          // run starts, P + 1
    int* nruns = runs + P + 1;
    unsigned char* hq = (unsigned char*)(nruns + 1);
    T* red = (T*)(smraw + (((size_t)P * dp * sizeof(T) + (2 * P + 2) * sizeof(int) + P + 15) / 16) * 16);

    const int tid = threadIdx.x, nt = blockDim.x;
    const int g = blockIdx.x;
    const int64_t p0 = (int64_t)g * a.R, p1 = min(a.N, p0 + a.R);
    Key key{a.seed, a.diter[0], a.diter[1], a.diter[2]};
    const XT* X = (const XT*)a.X;

    // register block of this thread
    const bool worker = tid < nblk * G;
    const int myblk = worker ? tid % nblk : 0, grp = worker ? tid / nblk : 0;
    int jb = 0, lb = 0;
    a.L.blk_coords(myblk, jb, lb);
    T acc[16], accr[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = accr[e] = 0;
    int cur = -1;

    auto flush = [&](int k) {
        __syncthreads();
        if (worker) {
            T* r = red + ((size_t)grp * nblk + myblk) * 32;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                r[e] = acc[e];
                r[16 + e] = accr[e];
            }
        }
        __syncthreads();
        double* out = a.rec + (size_t)(g + k) * 2 * a.L.E;
        for (int e = tid; e < nblk * 16; e += nt) {
            int b = e >> 4, q = e & 15;
            double all = 0.0, rr = 0.0;
            for (int gg = 0; gg < G; ++gg) {
                all += (double)red[((size_t)gg * nblk + b) * 32 + q];
                rr += (double)red[((size_t)gg * nblk + b) * 32 + 16 + q];
            }
            out[b * 16 + q] = all - rr;       // sub-cluster l
            out[a.L.E + b * 16 + q] = rr;     // sub-cluster r
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = accr[e] = 0;
    };

    for (int64_t base = p0; base < p1; base += P) {
        const int np = (int)min((int64_t)P, p1 - base);
        __syncthreads();
        if (tid < np) {
            const int i = a.idx[base + tid];
            const int k = a.z[i];
            T* xr = xs + (size_t)tid * dp;
            for (int j = 0; j < d; ++j) xr[j] = ldx<T, XT>(X + (int64_t)i * a.xs + j);
            int h;
            if (a.draw) {
                uint32_t w[4];
                key.block((uint32_t)i, TAG_ZBAR, 0, w);
                T vl = sub_score<T, XT>(a, 3 * k + 1, xr) + gumbel_of<T>(w[0], w[1]);
                T vr = sub_score<T, XT>(a, 3 * k + 2, xr) + gumbel_of<T>(w[2], w[3]);
                h = vr > vl ? 1 : 0;
                a.zbar[i] = (uint8_t)h;
            } else {
                h = a.zbar[i];
            }
            const T* sh = a.shift + (size_t)k * d;
            for (int j = 0; j < d; ++j) xr[j] -= sh[j];
            xr[d] = 1;
            for (int j = d + 1; j < dp; ++j) xr[j] = 0;
            kq[tid] = k;
            hq[tid] = (unsigned char)h;
        }
        __syncthreads();
        {
            __shared__ int wcnt[32];
            find_runs(kq, np, runs, nruns, wcnt);
        }
        const int nr = *nruns;
        for (int r = 0; r < nr; ++r) {
            const int qs = runs[r], qe = runs[r + 1];
            const int k = kq[qs];
            if (k != cur) {
                if (cur >= 0) flush(cur);
                cur = k;
            }
            if (worker) {
                for (int q = qs + grp; q < qe; q += G) {
                    const T* xr = xs + (size_t)q * dp;
                    T xj[4], xl[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        xj[u] = xr[jb * 4 + u];
                        xl[u] = xr[lb * 4 + u];
                    }
                    const T hm = hq[q] ? (T)1 : (T)0;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            T pr = xj[u] * xl[v];
                            acc[u * 4 + v] += pr;
                            accr[u * 4 + v] += hm * pr;
                        }
                }
            }
        }
    }
    if (cur >= 0) flush(cur);
}

// FP32 variant for d <= DV (DV = 32 or 64): the sub-cluster parameters of the current
// cluster run are staged in shared memory (factor transposed and zero-padded to
// DV x DV, so row j holds W[l][j] for l <= j), the point's x - mu sits in registers,
// and each sub-cluster score costs d(d+1)/2 FMAs fed by float4 broadcast loads.
// Statistics: one 4x4 register block per worker thread and one accumulator set per
// sub-cluster (the branch on h is uniform within a warp: a warp's lanes share the
// point).  Dynamic shared memory: P x dp point rows, P ints (k), P + 2 ints (runs),
// P bytes (h), then 2 DV x DV + 2 DV + 2 + d floats (staged parameters), then the
// flush buffer G x nblk x 32 floats.
template <int DV, typename XT>
__global__ void __launch_bounds__(256) substats_f32_kernel(SubArgs<float> a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int d = a.d, dp = a.L.dp, P = a.P, G = a.G, nblk = a.L.nblk;
    float* xs = (float*)smraw;
    int* kq = (int*)(xs + (size_t)P * dp);
    int* runs = kq + P;
    int* nruns = runs + P + 1;
    unsigned char* hq = (unsigned char*)(nruns + 1);
    float* stg = (float*)(smraw + (((size_t)P * dp * 4 + (2 * P + 2) * sizeof(int) + P + 15) / 16) * 16);
    float* WT0 = stg;                 // DV x DV
    float* WT1 = WT0 + DV * DV;       // DV x DV
    float* mu0 = WT1 + DV * DV;       // DV
    float* mu1 = mu0 + DV;            // DV
    float* cc = mu1 + DV;             // 2
    float* shf = cc + 2;              // d (cluster shift)
    float* red = (float*)(((uintptr_t)(shf + DV) + 15) & ~(uintptr_t)15);
    __shared__ int staged;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int g = blockIdx.x;
    const int64_t p0 = (int64_t)g * a.R, p1 = min(a.N, p0 + a.R);
    Key key{a.seed, a.diter[0], a.diter[1], a.diter[2]};
    const XT* X = (const XT*)a.X;
    const bool worker = tid < nblk * G;
    const int myblk = worker ? tid % nblk : 0, grp = worker ? tid / nblk : 0;
    int jb = 0, lb = 0;
    a.L.blk_coords(myblk, jb, lb);
    float acc0[16], acc1[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc0[e] = acc1[e] = 0.f;
    int cur = -1;
    if (tid == 0) staged = -1;

    auto flush = [&](int k) {
        __syncthreads();
        if (worker) {
            float* r = red + ((size_t)grp * nblk + myblk) * 32;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                r[e] = acc0[e];
                r[16 + e] = acc1[e];
            }
        }
        __syncthreads();
        double* out = a.rec + (size_t)(g + k) * 2 * a.L.E;
        for (int e = tid; e < nblk * 16; e += nt) {
            int b = e >> 4, q = e & 15;
            double s0 = 0.0, s1 = 0.0;
            for (int gg = 0; gg < G; ++gg) {
                s0 += (double)red[((size_t)gg * nblk + b) * 32 + q];
                s1 += (double)red[((size_t)gg * nblk + b) * 32 + 16 + q];
            }
            out[b * 16 + q] = s0;
            out[a.L.E + b * 16 + q] = s1;
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) acc0[e] = acc1[e] = 0.f;
    };

    for (int64_t base = p0; base < p1; base += P) {
        const int np = (int)min((int64_t)P, p1 - base);
        __syncthreads();
        int i = 0;
        float v[DV];
        if (tid < np) {
            i = a.idx[base + tid];
            kq[tid] = a.z[i];
            if constexpr (sizeof(XT) == 4) {  // rows are 16-byte aligned (stride a multiple of 4 floats)
                const float4* xr4 = (const float4*)(X + (int64_t)i * a.xs);
#pragma unroll
                for (int j4 = 0; j4 < DV / 4; ++j4) {
                    const float4 q = j4 * 4 < d ? xr4[j4] : make_float4(0.f, 0.f, 0.f, 0.f);
                    v[4 * j4] = q.x;
                    v[4 * j4 + 1] = q.y;
                    v[4 * j4 + 2] = q.z;
                    v[4 * j4 + 3] = q.w;
                }
#pragma unroll
                for (int j = 0; j < DV; ++j)
                    if (j >= d) v[j] = 0.f;
            } else {
#pragma unroll
                for (int j = 0; j < DV; ++j) v[j] = j < d ? ldx<float, XT>(X + (int64_t)i * a.xs + j) : 0.f;
            }
        }
        __syncthreads();
        {
            __shared__ int wcnt2[32];
            find_runs(kq, np, runs, nruns, wcnt2);
        }
        const int nr = *nruns;
        for (int r = 0; r < nr; ++r) {
            const int qs = runs[r], qe = runs[r + 1];
            const int k = kq[qs];
            if (k != staged) {  // uniform: stage this cluster's two sub-clusters
                __syncthreads();
                for (int e = tid; e < 2 * DV * DV; e += nt) {
                    const int h = e / (DV * DV), jj = (e / DV) % DV, l = e % DV;
                    const int s = 3 * k + 1 + h;
                    stg[e] = (jj < d && l <= jj) ? a.pv.W[((size_t)s * d + l) * d + jj] : 0.f;
                }
                for (int e = tid; e < 2 * DV; e += nt) {
                    const int h = e / DV, j = e % DV;
                    mu0[e] = j < d ? a.pv.mu[(size_t)(3 * k + 1 + h) * d + j] : 0.f;
                }
                if (tid < 2) cc[tid] = a.pv.c[3 * k + 1 + tid];
                for (int j = tid; j < d; j += nt) shf[j] = a.shift[(size_t)k * d + j];
                __syncthreads();
                if (tid == 0) staged = k;
            }
            if (tid >= qs && tid < qe) {
                int h;
                if (a.draw) {
                    float sc[2];
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const float* WT = hh ? WT1 : WT0;
                        const float* mu = hh ? mu1 : mu0;
                        float t[DV];
#pragma unroll
                        for (int l = 0; l < DV; ++l) t[l] = v[l] - mu[l];
                        float q = 0.f;
#pragma unroll
                        for (int j = 0; j < DV; ++j) {
                            if (j < d) {
                                float y = 0.f;
#pragma unroll
                                for (int l4 = 0; l4 <= j / 4; ++l4) {
                                    const float4 w = *(const float4*)(WT + j * DV + l4 * 4);
                                    y = fmaf(w.x, t[l4 * 4], y);
                                    y = fmaf(w.y, t[l4 * 4 + 1], y);
                                    y = fmaf(w.z, t[l4 * 4 + 2], y);
                                    y = fmaf(w.w, t[l4 * 4 + 3], y);
                                }
                                q = fmaf(y, y, q);
                            }
                        }
                        sc[hh] = cc[hh] - 0.5f * q;
                    }
                    uint32_t w[4];
                    key.block((uint32_t)i, TAG_ZBAR, 0, w);
                    const float vl = sc[0] + gumbel_of<float>(w[0], w[1]);
                    const float vr = sc[1] + gumbel_of<float>(w[2], w[3]);
                    h = vr > vl ? 1 : 0;
                    a.zbar[i] = (uint8_t)h;
                } else {
                    h = a.zbar[i];
                }
                // the centred row, then 1, then zeros, as float4 stores (conflict-free at any
                // row stride that is a multiple of 4 floats)
                float4* xr4 = (float4*)(xs + (size_t)tid * dp);
#pragma unroll
                for (int j4 = 0; j4 < (DV + 4) / 4; ++j4) {
                    if (j4 * 4 < dp) {
                        float e[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = 4 * j4 + u;
                            e[u] = j < d ? v[j < DV ? j : 0] - shf[j < DV ? j : 0] : (j == d ? 1.f : 0.f);
                        }
                        xr4[j4] = make_float4(e[0], e[1], e[2], e[3]);
                    }
                }
                hq[tid] = (unsigned char)h;
            }
        }
        __syncthreads();
        for (int r = 0; r < nr; ++r) {
            const int qs = runs[r], qe = runs[r + 1];
            const int k = kq[qs];
            if (k != cur) {
                if (cur >= 0) flush(cur);
                cur = k;
            }
            if (worker) {
                for (int q = qs + grp; q < qe; q += G) {
                    const float* xr = xs + (size_t)q * dp;
                    const float4 xj = *(const float4*)(xr + jb * 4);
                    const float4 xl = *(const float4*)(xr + lb * 4);
                    const float aj[4] = {xj.x, xj.y, xj.z, xj.w}, al[4] = {xl.x, xl.y, xl.z, xl.w};
                    if (hq[q]) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int w2 = 0; w2 < 4; ++w2) acc1[u * 4 + w2] = fmaf(aj[u], al[w2], acc1[u * 4 + w2]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int w2 = 0; w2 < 4; ++w2) acc0[u * 4 + w2] = fmaf(aj[u], al[w2], acc0[u * 4 + w2]);
                    }
                }
            }
        }
    }
    if (cur >= 0) flush(cur);
}

// FP32 variant for 64 < d <= 128 (Gaussian).  Per batch of WP = 64 points (sorted by
// cluster): each sub-cluster score is the squared norm of (x - mu_h) W_h
// = (x - shift) W_h - bh, with bh = (mu_h - shift)^T W_h formed once per cluster run and
// shift the cluster's statistics centre; both products run at once over the shifted rows
// (warps 0-7 sub-cluster 0, warps 8-15 sub-cluster 1; each thread owns 8 points x 4
// columns; per K step two broadcast float4 loads of (x - shift)^T and one float4 of W
// feed 32 FMAs; W is staged once per cluster run, zero below the diagonal and beyond d,
// so the loop needs no triangular bound).  Statistics: one 4x4 register block per
// worker thread (nblk <= 561 workers, so every block has one owner and is written
// straight to the records) and one accumulator set per sub-cluster (warp-uniform
// branch on h).  Dynamic shared memory: 2 x 128 x 128 floats (W_l, W_r), 128 x WP
// (x - mu_h)^T, WP x dp point rows, WP x 2 scores, then ints and bytes.
constexpr int WP = 64;
constexpr int WIDE_T = 576;

template <typename XT>
__global__ void __launch_bounds__(WIDE_T, 1) substats_wide_kernel(SubArgs<float> a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int d = a.d, dp = a.L.dp, nblk = a.L.nblk;
    float* Ws = (float*)smraw;              // 2 x 128 x 128: W_h[l][j]
    float* Tt = Ws + 2 * 128 * 128;         // 128 x WP: (x_p - shift)_l at Tt[l * WP + p]
    float* xs = Tt + 128 * WP;              // WP x dp
    float* qv = xs + WP * dp;               // WP x 2
    float* mus = qv + 2 * WP;               // 2 x 128
    float* bh = mus + 256;                  // 2 x 128
    float* shf = bh + 256;                  // 128
    float* cc = shf + 128;                  // 2 (+2 pad)
    int* kq = (int*)(cc + 4);               // WP
    int* runs = kq + WP;                    // WP + 1
    int* nruns = runs + WP + 1;             // 1
    unsigned char* hq = (unsigned char*)(nruns + 1);  // WP
    __shared__ int staged;
    __shared__ int wcnt[32];

    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    const int64_t p0 = (int64_t)g * a.R, p1 = min(a.N, p0 + a.R);
    Key key{a.seed, a.diter[0], a.diter[1], a.diter[2]};
    const XT* X = (const XT*)a.X;
    const bool worker = tid < nblk;
    int jb = 0, lb = 0;
    a.L.blk_coords(worker ? tid : 0, jb, lb);
    float acc0[16], acc1[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc0[e] = acc1[e] = 0.f;
    int cur = -1;
    if (tid == 0) staged = -1;

    auto flush = [&](int k) {  // every block has a single owner: no reduction
        if (worker) {
            double* out = a.rec + (size_t)(g + k) * 2 * a.L.E + (size_t)tid * 16;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                out[e] = (double)acc0[e];
                out[a.L.E + e] = (double)acc1[e];
            }
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) acc0[e] = acc1[e] = 0.f;
    };

    for (int64_t base = p0; base < p1; base += WP) {
        const int np = (int)min((int64_t)WP, p1 - base);
        __syncthreads();
        if (tid < np) kq[tid] = a.z[a.idx[base + tid]];
        // raw rows, one warp per row (d <= 128: one float4 per lane)
        for (int r = warp; r < np; r += nt / 32) {
            const int i = a.idx[base + r];
            float* xr = xs + (size_t)r * dp;
            if constexpr (sizeof(XT) == 4) {
                if (lane * 4 < d) *(float4*)(xr + lane * 4) = *(const float4*)(X + (int64_t)i * a.xs + lane * 4);
            } else {
                for (int j = lane; j < d; j += 32) xr[j] = ldx<float, XT>(X + (int64_t)i * a.xs + j);
            }
        }
        __syncthreads();
        find_runs(kq, np, runs, nruns, wcnt);
        const int nr = *nruns;
        for (int r = 0; r < nr; ++r) {
            const int qs = runs[r], qe = runs[r + 1];
            const int k = kq[qs];
            if (k != staged) {  // uniform: stage the cluster's two sub-clusters
                __syncthreads();
                for (int e = tid; e < 2 * 128 * 128; e += nt) {
                    const int h = e >> 14, l = (e >> 7) & 127, j = e & 127;
                    const int s = 3 * k + 1 + h;
                    Ws[e] = (j < d && l <= j) ? a.pv.W[((size_t)s * d + l) * d + j] : 0.f;
                }
                for (int e = tid; e < 256; e += nt) {
                    const int h = e >> 7, j = e & 127;
                    mus[e] = j < d ? a.pv.mu[(size_t)(3 * k + 1 + h) * d + j] : 0.f;
                }
                if (tid < 2) cc[tid] = a.pv.c[3 * k + 1 + tid];
                for (int j = tid; j < 128; j += nt) shf[j] = j < d ? a.shift[(size_t)k * d + j] : 0.f;
                __syncthreads();
                // bh[h][j] = sum_l (mu_h - shift)_l W_h[l][j]: the products below run on the
                // shifted rows x - shift, so y_h = (x - shift) W_h - bh
                for (int e = tid; e < 256; e += nt) {
                    const int h = e >> 7, j = e & 127;
                    const float* Wh = Ws + h * 128 * 128;
                    float b = 0.f;
                    for (int l = 0; l < d; ++l) b = fmaf(mus[h * 128 + l] - shf[l], Wh[l * 128 + j], b);
                    bh[e] = b;
                }
                __syncthreads();
                if (tid == 0) staged = k;
            }
            // the run's rows shifted by the cluster's centre, then 1, then zeros (the
            // statistics read them too)
            for (int e = tid; e < (qe - qs) * dp; e += nt) {
                const int q = qs + e / dp, j = e % dp;
                float* xr = xs + (size_t)q * dp;
                xr[j] = j < d ? xr[j] - shf[j] : (j == d ? 1.f : 0.f);
            }
            if (a.draw) {
                __syncthreads();
                for (int e = tid; e < 128 * WP; e += nt) {
                    const int l = e / WP, p = e % WP;
                    Tt[e] = (l < d && p >= qs && p < qe) ? xs[(size_t)p * dp + l] : 0.f;
                }
                __syncthreads();
                if (tid < 512) {  // warps 0-7: sub-cluster 0, warps 8-15: sub-cluster 1
                    const int h = warp >> 3;
                    const int pg = warp & 7, cg = lane;  // points 8 pg .. 8 pg + 7, columns 4 cg .. 4 cg + 3
                    float y[8][4];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) y[u][v] = 0.f;
                    const float* Wh = Ws + h * 128 * 128;
                    for (int l = 0; l < d; ++l) {
                        const float4 t0 = *(const float4*)(Tt + l * WP + pg * 8);
                        const float4 t1 = *(const float4*)(Tt + l * WP + pg * 8 + 4);
                        const float4 w0 = *(const float4*)(Wh + l * 128 + cg * 4);
                        const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
                        const float wv[4] = {w0.x, w0.y, w0.z, w0.w};
#pragma unroll
                        for (int u = 0; u < 8; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) y[u][v] = fmaf(tv[u], wv[v], y[u][v]);
                    }
                    const float4 b4 = *(const float4*)(bh + h * 128 + cg * 4);
                    const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
                    float qp[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        float s0 = 0.f;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const float t = y[u][v] - bv[v];
                            s0 = fmaf(t, t, s0);
                        }
                        qp[u] = s0;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int u = 0; u < 8; ++u) qp[u] += __shfl_xor_sync(0xffffffffu, qp[u], o);
                    if (cg == 0)
#pragma unroll
                        for (int u = 0; u < 8; ++u) qv[(pg * 8 + u) * 2 + h] = qp[u];
                }
                __syncthreads();
            }
            if (tid >= qs && tid < qe) {
                const int i = a.idx[base + tid];
                int h;
                if (a.draw) {
                    uint32_t w[4];
                    key.block((uint32_t)i, TAG_ZBAR, 0, w);
                    const float vl = cc[0] - 0.5f * qv[tid * 2] + gumbel_of<float>(w[0], w[1]);
                    const float vr = cc[1] - 0.5f * qv[tid * 2 + 1] + gumbel_of<float>(w[2], w[3]);
                    h = vr > vl ? 1 : 0;
                    a.zbar[i] = (uint8_t)h;
                } else {
                    h = a.zbar[i];
                }
                hq[tid] = (unsigned char)h;
            }
        }
        __syncthreads();
        for (int r = 0; r < nr; ++r) {
            const int qs = runs[r], qe = runs[r + 1];
            const int k = kq[qs];
            if (k != cur) {
                if (cur >= 0) flush(cur);
                cur = k;
            }
            if (worker) {
                for (int q = qs; q < qe; ++q) {
                    const float* xr = xs + (size_t)q * dp;
                    const float4 xj = *(const float4*)(xr + jb * 4);
                    const float4 xl = *(const float4*)(xr + lb * 4);
                    const float aj[4] = {xj.x, xj.y, xj.z, xj.w}, al[4] = {xl.x, xl.y, xl.z, xl.w};
                    if (hq[q]) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int w2 = 0; w2 < 4; ++w2) acc1[u * 4 + w2] = fmaf(aj[u], al[w2], acc1[u * 4 + w2]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int w2 = 0; w2 < 4; ++w2) acc0[u * 4 + w2] = fmaf(aj[u], al[w2], acc0[u * 4 + w2]);
                    }
                }
            }
        }
    }
    if (cur >= 0) flush(cur);
}

// Multinomial variant (first-moment statistics only): the point's counts become a
// float row in shared memory (x, then 1, then zeros), each row loaded by one warp in
// 16-byte pieces, four rows in flight per lane; the current run's two sub-cluster log
// theta vectors are staged in shared memory; each sub-cluster score is a d-long dot
// product fed by float4 loads; each worker thread owns the counts of one 4-category
// block for both sub-clusters.  Dynamic shared memory: P x dp rows, P ints (k), P + 2
// ints (runs), P ints (point indices), P bytes (h), then 2 dp + 2 floats (staged
// parameters), then the flush buffer G x nblk x 8 floats.
template <typename XT>
__global__ void __launch_bounds__(256) substats_mult_kernel(SubArgs<float> a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int d = a.d, dp = a.L.dp, P = a.P, G = a.G, nblk = a.L.nblk;
    float* xs = (float*)smraw;
    int* kq = (int*)(xs + (size_t)P * dp);
    int* runs = kq + P;
    int* nruns = runs + P + 1;
    int* iq = nruns + 1;
    unsigned char* hq = (unsigned char*)(iq + P);
    float* lt0 = (float*)(smraw + (((size_t)P * dp * 4 + (3 * P + 2) * sizeof(int) + P + 15) / 16) * 16);
    float* lt1 = lt0 + dp;
    float* cc = lt1 + dp;
    float* red = (float*)(((uintptr_t)(cc + 2) + 15) & ~(uintptr_t)15);
    __shared__ int staged;
    __shared__ int wcnt[32];

    const int tid = threadIdx.x, nt = blockDim.x;
    const int g = blockIdx.x;
    const int64_t p0 = (int64_t)g * a.R, p1 = min(a.N, p0 + a.R);
    Key key{a.seed, a.diter[0], a.diter[1], a.diter[2]};
    const XT* X = (const XT*)a.X;
    const bool worker = tid < nblk * G;
    const int myblk = worker ? tid % nblk : 0, grp = worker ? tid / nblk : 0;
    const int one = d & 3;  // position of the constant 1 inside the last 4-column block
    float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
    int cur = -1;
    if (tid == 0) staged = -1;

    auto flush = [&](int k) {
        __syncthreads();
        if (worker) {
            float* r = red + ((size_t)grp * nblk + myblk) * 8;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                r[u] = acc0[u];
                r[4 + u] = acc1[u];
            }
        }
        __syncthreads();
        double* out = a.rec + (size_t)(g + k) * 2 * a.L.E;
        for (int e = tid; e < nblk * 16; e += nt) {
            const int b = e >> 4, q = e & 15, u = q >> 2, v = q & 3;
            double s0 = 0.0, s1 = 0.0;
            if (v == one)
                for (int gg = 0; gg < G; ++gg) {
                    s0 += (double)red[((size_t)gg * nblk + b) * 8 + u];
                    s1 += (double)red[((size_t)gg * nblk + b) * 8 + 4 + u];
                }
            out[e] = s0;
            out[a.L.E + e] = s1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc0[u] = acc1[u] = 0.f;
    };

    for (int64_t base = p0; base < p1; base += P) {
        const int np = (int)min((int64_t)P, p1 - base);
        __syncthreads();
        int i = 0;
        if (tid < np) {
            i = a.idx[base + tid];
            kq[tid] = a.z[i];
            iq[tid] = i;
        }
        __syncthreads();
        {
            const int lane = tid & 31, nwarp = nt >> 5;
            if constexpr (sizeof(XT) == 2) {  // 16-byte loads: 8 BF16 counts (rows are 16-byte aligned)
                const int nfull = d / 8;      // whole 8-count chunks inside the row's d columns
                for (int q0 = tid >> 5; q0 < np; q0 += 4 * nwarp) {
                    for (int c0 = 0; c0 < nfull; c0 += 32) {
                        const int c8 = c0 + lane;
                        uint4 v[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = q0 + u * nwarp;
                            if (q < np && c8 < nfull) v[u] = ((const uint4*)(X + (int64_t)iq[q] * a.xs))[c8];
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = q0 + u * nwarp;
                            if (q < np && c8 < nfull) {
                                const uint32_t wv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                                float f[8];
#pragma unroll
                                for (int w = 0; w < 4; ++w) {
                                    f[2 * w] = __uint_as_float(wv[w] << 16);
                                    f[2 * w + 1] = __uint_as_float(wv[w] & 0xFFFF0000u);
                                }
                                float* xr = xs + (size_t)q * dp + 8 * c8;
                                *(float4*)xr = make_float4(f[0], f[1], f[2], f[3]);
                                *(float4*)(xr + 4) = make_float4(f[4], f[5], f[6], f[7]);
                            }
                        }
                    }
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + u * nwarp;
                        if (q >= np) break;
                        for (int j = 8 * nfull + lane; j < dp; j += 32)
                            xs[(size_t)q * dp + j] = j < d ? ldx<float, XT>(X + (int64_t)iq[q] * a.xs + j) : (j == d ? 1.f : 0.f);
                    }
                }
            } else {
                for (int q = tid >> 5; q < np; q += nwarp)
                    for (int j = lane; j < dp; j += 32)
                        xs[(size_t)q * dp + j] = j < d ? ldx<float, XT>(X + (int64_t)iq[q] * a.xs + j) : (j == d ? 1.f : 0.f);
            }
        }
        __syncthreads();
        find_runs(kq, np, runs, nruns, wcnt);
        const int nr = *nruns;
        for (int r = 0; r < nr; ++r) {
            const int qs = runs[r], qe = runs[r + 1];
            const int k = kq[qs];
            if (a.draw && k != staged) {  // uniform: stage this cluster's two sub-clusters
                __syncthreads();
                for (int e = tid; e < 2 * dp; e += nt) {
                    const int h = e / dp, j = e % dp;
                    lt0[e] = j < d ? a.pv.lt[(size_t)(3 * k + 1 + h) * d + j] : 0.f;
                }
                if (tid < 2) cc[tid] = a.pv.c[3 * k + 1 + tid];
                __syncthreads();
                if (tid == 0) staged = k;
            }
            if (tid >= qs && tid < qe) {
                int h;
                if (a.draw) {
                    const float4* xr4 = (const float4*)(xs + (size_t)tid * dp);
                    const float4* l04 = (const float4*)lt0;
                    const float4* l14 = (const float4*)lt1;
                    float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;
                    for (int j4 = 0; j4 < dp / 4; ++j4) {
                        const float4 x = xr4[j4], u = l04[j4], w = l14[j4];
                        s0 = fmaf(x.x, u.x, s0);
                        t0 = fmaf(x.y, u.y, t0);
                        s0 = fmaf(x.z, u.z, s0);
                        t0 = fmaf(x.w, u.w, t0);
                        s1 = fmaf(x.x, w.x, s1);
                        t1 = fmaf(x.y, w.y, t1);
                        s1 = fmaf(x.z, w.z, s1);
                        t1 = fmaf(x.w, w.w, t1);
                    }
                    // the padding column d holds 1 and lt[d] = 0: it adds nothing
                    uint32_t wq[4];
                    key.block((uint32_t)i, TAG_ZBAR, 0, wq);
                    const float vl = cc[0] + s0 + t0 + gumbel_of<float>(wq[0], wq[1]);
                    const float vr = cc[1] + s1 + t1 + gumbel_of<float>(wq[2], wq[3]);
                    h = vr > vl ? 1 : 0;
                    a.zbar[i] = (uint8_t)h;
                } else {
                    h = a.zbar[i];
                }
                hq[tid] = (unsigned char)h;
            }
        }
        __syncthreads();
        for (int r = 0; r < nr; ++r) {
            const int qs = runs[r], qe = runs[r + 1];
            const int k = kq[qs];
            if (k != cur) {
                if (cur >= 0) flush(cur);
                cur = k;
            }
            if (worker) {
                for (int q = qs + grp; q < qe; q += G) {
                    const float4 xj = *(const float4*)(xs + (size_t)q * dp + myblk * 4);
                    if (hq[q]) {
                        acc1[0] += xj.x; acc1[1] += xj.y; acc1[2] += xj.z; acc1[3] += xj.w;
                    } else {
                        acc0[0] += xj.x; acc0[1] += xj.y; acc0[2] += xj.z; acc0[3] += xj.w;
                    }
                }
            }
        }
    }
    if (cur >= 0) flush(cur);
}

// Multinomial sub-labels and statistics (first moments only), one warp per range of sorted
// positions, that is, of points in cluster order.  Lane l holds categories 8l .. 8l + 7 (d <= 256)
// of a point's counts and of the two sub-cluster log theta rows of the current cluster; the
// two sub-cluster scores are dot products reduced across the warp; the z-bar draws of 32
// points are made at once, one point per lane; the counts of a cluster's run stay in registers
// and are added at the run's end to the compact table cnt (2 K_max x (d + 1) integers, column
// d: the points) with atomic adds, exact in any order.  No block-wide barrier.
struct MwArgs {
    int64_t N, R;  // points; sorted positions per warp
    int d, xs;
    const void* X;
    const int* idx;     // sorted position -> point
    const int* starts;  // K + 1 cluster offsets in sorted order
    const int* dK;
    const float* lt;    // slots x d log theta (FP32)
    const float* lc;    // slots: log weights
    const uint32_t* diter;
    uint64_t seed;
    const int* gate;
    int draw;
    uint8_t* zbar;
    unsigned* cnt;
};

constexpr int MW_DEPTH = 16;  // rows in flight per warp (a ring in shared memory)
constexpr int MW_ROWB = 512;  // bytes per ring slot: d <= 256 BF16 counts

__device__ __forceinline__ void mw_cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// BF16 counts (rows 16-byte aligned).  Dynamic shared memory: 8 warps x MW_DEPTH x MW_ROWB.
__global__ void __launch_bounds__(256, 3) mult_warp_kernel(MwArgs a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(16) unsigned char mw_sm[];
    const int lane = threadIdx.x & 31;
    unsigned char* ring = mw_sm + (threadIdx.x >> 5) * (MW_DEPTH * MW_ROWB);
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t p0 = w * a.R, p1 = min(a.N, p0 + a.R);
    if (p0 >= p1) return;
    const int K = *a.dK, d = a.d, j0 = 8 * lane, nch = (d + 7) >> 3;
    int k = 0;  // the cluster of position p0: the last k with starts[k] <= p0
    for (int lo = 0, hi = K; hi - lo > 1;) {
        const int mid = (lo + hi) >> 1;
        if (a.starts[mid] <= p0) lo = mid;
        else hi = mid;
        k = lo;
    }
    int64_t kend = a.starts[k + 1];
    float lt0[8], lt1[8], c0 = 0.f, c1 = 0.f;
    auto stage = [&](int kk) {
        const float* r0 = a.lt + (size_t)(3 * kk + 1) * d + j0;
        const float* r1 = r0 + d;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            lt0[u] = j0 + u < d ? r0[u] : 0.f;
            lt1[u] = j0 + u < d ? r1[u] : 0.f;
        }
        c0 = a.lc[3 * kk + 1];
        c1 = a.lc[3 * kk + 2];
    };
    unsigned acc0[8], acc1[8], n0 = 0, n1 = 0;  // integer counts: exact
#pragma unroll
    for (int u = 0; u < 8; ++u) acc0[u] = acc1[u] = 0u;
    auto flush = [&](int kk) {
        unsigned* r0 = a.cnt + (size_t)(2 * kk) * (d + 1);
        unsigned* r1 = r0 + (d + 1);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (j0 + u < d) {
                if (acc0[u]) atomicAdd(r0 + j0 + u, acc0[u]);
                if (acc1[u]) atomicAdd(r1 + j0 + u, acc1[u]);
            }
            acc0[u] = acc1[u] = 0u;
        }
        if (lane == 0) {
            if (n0) atomicAdd(r0 + d, n0);
            if (n1) atomicAdd(r1 + d, n1);
        }
        n0 = n1 = 0;
    };
    if (a.draw) stage(k);
    const Key key{a.seed, a.diter[0], a.diter[1], a.diter[2]};
    // point indices of positions in batches of 32 (lane l: position batch start + l); the
    // next batch's are loaded one batch ahead
    int64_t bstart = p0;
    int cur = p0 + lane < p1 ? a.idx[p0 + lane] : 0;
    int nxt = p0 + 32 + lane < p1 ? a.idx[p0 + 32 + lane] : 0;
    auto pick = [&](int64_t pos) {
        const int r = (int)(pos - bstart);
        const int vc = __shfl_sync(0xffffffffu, cur, r & 31), vn = __shfl_sync(0xffffffffu, nxt, r & 31);
        return r < 32 ? vc : vn;
    };
    auto issue = [&](int slot, int64_t pos) {  // the row of position pos into a ring slot
        if (pos < p1) {
            const int i = pick(pos);
            if (lane < nch)
                mw_cp16(ring + slot * MW_ROWB + lane * 16, (const char*)a.X + (int64_t)i * a.xs * 2 + lane * 16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int t = 0; t < MW_DEPTH; ++t) issue(t, p0 + t);
    float gl = 0.f, gr = 0.f;
    int hz = 0;
    auto draws = [&]() {  // this batch's z-bar Gumbel values (or kept z-bar), one point per lane
        if (bstart + lane < p1) {
            if (a.draw) {
                uint32_t wq[4];
                key.block((uint32_t)cur, TAG_ZBAR, 0, wq);
                gl = gumbel_of<float>(wq[0], wq[1]);
                gr = gumbel_of<float>(wq[2], wq[3]);
            } else {
                hz = a.zbar[cur];
            }
        }
    };
    draws();
    for (int64_t p = p0; p < p1; ++p) {
        if (p - bstart == 32) {  // the next batch
            bstart += 32;
            cur = nxt;
            nxt = bstart + 32 + lane < p1 ? a.idx[bstart + 32 + lane] : 0;
            draws();
        }
        const int slot = (int)((p - p0) % MW_DEPTH);
        asm volatile("cp.async.wait_group %0;" ::"n"(MW_DEPTH - 1) : "memory");
        __syncwarp();
        float x[8];
        if (lane < nch) {
            const uint4 q = *(const uint4*)(ring + slot * MW_ROWB + lane * 16);
            const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[2 * u] = j0 + 2 * u < d ? __uint_as_float(wv[u] << 16) : 0.f;
                x[2 * u + 1] = j0 + 2 * u + 1 < d ? __uint_as_float(wv[u] & 0xFFFF0000u) : 0.f;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = 0.f;
        }
        __syncwarp();  // every lane has read the slot: it may be refilled
        issue(slot, p + MW_DEPTH);
        while (p >= kend) {  // the next cluster's run begins
            flush(k);
            ++k;
            kend = a.starts[k + 1];
            if (a.draw) stage(k);
        }
        const int q = (int)(p - bstart);
        int h;
        if (a.draw) {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                s0 = fmaf(x[u], lt0[u], s0);
                s1 = fmaf(x[u], lt1[u], s1);
            }
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            const float vl = c0 + s0 + __shfl_sync(0xffffffffu, gl, q);
            const float vr = c1 + s1 + __shfl_sync(0xffffffffu, gr, q);
            h = vr > vl ? 1 : 0;
            if (lane == q) a.zbar[cur] = (uint8_t)h;
        } else {
            h = __shfl_sync(0xffffffffu, hz, q);
        }
        if (h) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc1[u] += (unsigned)x[u];
            ++n1;
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc0[u] += (unsigned)x[u];
            ++n0;
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    flush(k);
}

// the compact counts of the 2K sub-clusters: cleared before, copied into the FP64
// statistics table after (grid: y = sub-cluster slot, x strides over the d + 1 columns)
__global__ void mcnt_zero_kernel(const int* dK, const int* gate, int d, unsigned* cnt) {
    if (gate && *gate == 0) return;
    const int s = blockIdx.y;
    if (s >= 2 * *dK) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= d; j += gridDim.x * blockDim.x) cnt[(size_t)s * (d + 1) + j] = 0u;
}

__global__ void mcnt_fill_kernel(const int* dK, const int* gate, StatLayout L, const unsigned* cnt, double* S) {
    if (gate && *gate == 0) return;
    const int s = blockIdx.y, d = L.d;
    if (s >= 2 * *dK) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= d; j += gridDim.x * blockDim.x)
        S[(size_t)s * L.E + L.ent(j, d)] = (double)cnt[(size_t)s * (d + 1) + j];
}

// stats[(2k + h) E + e] = sum over the CTAs g covering cluster k's run of rec[g + k]
__global__ void combine_kernel(const double* rec, const int* starts, const int* dK, int64_t R, int E,
                               const double* shift_new, double* shift_stats, int d, const int* gate,
                               double* stats) {
    if (gate && *gate == 0) return;
    const int K = *dK;
    const int kh = blockIdx.y, k = kh >> 1, h = kh & 1;
    if (k >= K) return;
    const int64_t st = starts[k], cnt = (int64_t)starts[k + 1] - st;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && h == 0)
        for (int j = threadIdx.x; j < d; j += blockDim.x) shift_stats[(size_t)k * d + j] = shift_new[(size_t)k * d + j];
    if (e >= E) return;
    double v = 0.0;
    if (cnt > 0) {  // the ranges' records in order; four loads in flight at a time
        const int64_t g0 = st / R, g1 = (st + cnt - 1) / R;
        for (int64_t g = g0; g <= g1; g += 4) {
            double r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) r[u] = g + u <= g1 ? rec[((size_t)(g + u + k) * 2 + h) * E + e] : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (g + u <= g1) v += r[u];
        }
    }
    stats[(size_t)kh * E + e] = v;
}

// initial labels: K = init_K, z uniform over K, z-bar a fair coin (tag INIT, c1 = 0)
__global__ void init_labels_kernel(int64_t N, int initK, uint64_t seed, const uint32_t* diter, int32_t* z,
                                   uint8_t* zbar) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    Key key{seed, 0, diter[1], diter[2]};
    uint32_t w[4];
    key.block((uint32_t)i, TAG_INIT, 0, w);
    int k = (int)(u01_f64(w[0], w[1]) * initK);
    if (k >= initK) k = initK - 1;
    z[i] = k;
    zbar[i] = u01_f64(w[2], w[3]) < 0.5 ? 0 : 1;
}

// ------------------------------------------------------------------ launchers
template <typename T>
static ParamView<T> pview(dpmm_ctx* c);
template <>
ParamView<double> pview<double>(dpmm_ctx* c) { return {c->p_W, c->p_mu, c->p_c, c->p_logtheta}; }
template <>
ParamView<float> pview<float>(dpmm_ctx* c) { return {c->q_W, c->q_mu, c->q_c, c->q_logtheta}; }

template <typename T, typename XT>
static cudaError_t labels_simt_t(dpmm_ctx* c, uint64_t seed, const int* gate) {
    const int d = c->d;
    const size_t per = c->kind == DPMM_PRIOR_NIW ? (size_t)d * d + d + 1 : (size_t)d + 1;
    size_t budget = 200 * 1024;
    int TB = 256;  // fewer points per CTA when the rows would not leave room for one cluster
    while (TB > 32 && (size_t)TB * (d + 1) * sizeof(T) + per * sizeof(T) > budget / 2) TB /= 2;
    const size_t rows = (size_t)TB * (d + 1) * sizeof(T);
    if (rows + per * sizeof(T) > budget) return cudaErrorInvalidValue;  // d too large for this kernel
    int CB = (int)std::max<size_t>(1, std::min<size_t>(32, (budget - rows) / (per * sizeof(T))));
    size_t sm = CB * per * sizeof(T) + rows;
    auto kern = c->dbg_scores ? labels_simt_kernel<T, XT, true> : labels_simt_kernel<T, XT, false>;
    cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ea != cudaSuccess) return ea;
    // a gated launch usually exits at once: one wave of CTAs (one per SM at this shared
    // memory size) that stride over the tiles
    int64_t tiles = (c->N + TB - 1) / TB;
    int grid = (int)(gate ? std::min<int64_t>(tiles, (int64_t)c->num_sms) : tiles);
    kern<<<grid, TB, sm, c->stream>>>(c->kind, d, c->xs, c->N, (const XT*)c->X, pview<T>(c), c->dK, c->diter, seed,
                                      CB, gate, c->dbg_scores, c->z);
    return cudaGetLastError();
}

cudaError_t launch_labels_simt_gated(dpmm_ctx* c, uint64_t seed, const int* gate) {
    const char* name = gate ? "labels_simt_overflow" : "labels_simt";
    prof_begin(c, name);
    cudaError_t e;
    if (c->prec == DPMM_PREC_FP64_PLAIN) e = labels_simt_t<double, double>(c, seed, gate);
    else if (c->xdt == 2) e = labels_simt_t<float, __nv_bfloat16>(c, seed, gate);
    else e = labels_simt_t<float, float>(c, seed, gate);
    prof_end(c, name);
    c->nlaunch += 1;
    return e;
}

cudaError_t launch_labels_simt(dpmm_ctx* c, uint64_t seed) { return launch_labels_simt_gated(c, seed, nullptr); }

static cudaError_t sort_impl(dpmm_ctx* c, const int* gate) {
    prof_begin(c, "sort");
    hist_kernel<<<c->T_tiles, 256, sizeof(int) * c->K_max, c->stream>>>(c->z, c->N, c->T_tiles, c->K_max, gate,
                                                                         c->hist);
    // tot holds K_max + 1 starts, then the scan's completion counter
    scan_kernel<<<c->K_max, 1024, 0, c->stream>>>(c->hist, c->T_tiles, c->dK, gate, c->tot, c->tot + c->K_max + 1);
    scatter_kernel<<<c->T_tiles, 256, sizeof(int) * 9 * c->K_max, c->stream>>>(c->z, c->N, c->T_tiles, c->hist, c->tot,
                                                                               gate, c->K_max, c->idx);
    prof_end(c, "sort");
    c->nlaunch += 3;
    return cudaGetLastError();
}

struct SubCfg {
    int P, BT, G;
    size_t smem;
};

template <typename T>
static SubCfg sub_cfg(const dpmm_ctx* c) {
    SubCfg q;
    const StatLayout& L = c->st;
    int P = (int)((64 * 1024) / ((size_t)L.dp * sizeof(T)));
    P = std::max(32, std::min(256, P / 32 * 32));
    int BT = std::max(P, L.nblk);
    BT = std::min(1024, std::max(256, (BT + 31) / 32 * 32));
    q.P = P;
    q.BT = BT;
    q.G = std::max(1, BT / L.nblk);
    size_t head = (size_t)P * L.dp * sizeof(T) + (2 * (size_t)P + 2) * sizeof(int) + P;
    head = (head + 15) / 16 * 16;
    q.smem = head + (size_t)q.G * L.nblk * 32 * sizeof(T);
    return q;
}

static SubCfg sub_cfg_f32(const dpmm_ctx* c, int DV) {
    SubCfg q;
    const StatLayout& L = c->st;
    const size_t stage = ((size_t)2 * DV * DV + 2 * DV + 2 + DV + 4) * 4;
    int P = (int)((64 * 1024) / ((size_t)L.dp * 4));
    P = std::max(32, std::min(256, P / 32 * 32));
    q.P = P;
    q.BT = 256;
    q.G = std::max(1, 256 / L.nblk);
    size_t head = (size_t)P * L.dp * 4 + (2 * (size_t)P + 2) * sizeof(int) + P;
    head = (head + 15) / 16 * 16;
    q.smem = head + stage + 16 + (size_t)q.G * L.nblk * 32 * 4;
    return q;
}

size_t substats_smem(const dpmm_ctx* c) {
    return c->prec == DPMM_PREC_FP64_PLAIN ? sub_cfg<double>(c).smem : sub_cfg<float>(c).smem;
}

template <typename T, typename XT>
static cudaError_t substats_t(dpmm_ctx* c, uint64_t seed, int draw, const int* gate) {
    SubCfg q = sub_cfg<T>(c);
    SubArgs<T> a;
    a.kind = c->kind;
    a.d = c->d;
    a.xs = c->xs;
    a.N = c->N;
    a.X = c->X;
    a.pv = pview<T>(c);
    a.shift = (const T*)(sizeof(T) == 8 ? (const void*)c->shift_new : (const void*)c->shift32);
    a.z = c->z;
    a.zbar = c->zbar;
    a.idx = c->idx;
    a.dK = c->dK;
    a.diter = c->diter;
    a.gate = gate;
    a.seed = seed;
    a.draw = draw;
    a.P = q.P;
    a.G = q.G;
    a.R = (c->N + c->Gr - 1) / c->Gr;
    a.L = c->st;
    a.rec = c->records;
    if (q.BT <= 256) {
        cudaError_t ea = cudaFuncSetAttribute(substats_kernel<T, XT, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q.smem);
        if (ea != cudaSuccess) return ea;
        substats_kernel<T, XT, 256><<<c->Gr, q.BT, q.smem, c->stream>>>(a);
    } else {
        cudaError_t ea = cudaFuncSetAttribute(substats_kernel<T, XT, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q.smem);
        if (ea != cudaSuccess) return ea;
        substats_kernel<T, XT, 1024><<<c->Gr, q.BT, q.smem, c->stream>>>(a);
    }
    return cudaGetLastError();
}

static cudaError_t combine_impl(dpmm_ctx* c, const int* gate) {
    dim3 grid((c->st.E + 255) / 256, 2 * c->K_max);
    int64_t R = (c->N + c->Gr - 1) / c->Gr;
    combine_kernel<<<grid, 256, 0, c->stream>>>(c->records, c->tot, c->dK, R, c->st.E, c->shift_new, c->shift_stats,
                                                c->d, gate, c->stats);
    return cudaGetLastError();
}

cudaError_t launch_sort(dpmm_ctx* c) { return sort_impl(c, nullptr); }

template <int DV, typename XT>
static cudaError_t substats_f32_t(dpmm_ctx* c, uint64_t seed, int draw, const int* gate) {
    SubCfg q = sub_cfg_f32(c, DV);
    SubArgs<float> a;
    a.kind = c->kind;
    a.d = c->d;
    a.xs = c->xs;
    a.N = c->N;
    a.X = c->X;
    a.pv = pview<float>(c);
    a.shift = c->shift32;
    a.z = c->z;
    a.zbar = c->zbar;
    a.idx = c->idx;
    a.dK = c->dK;
    a.diter = c->diter;
    a.gate = gate;
    a.seed = seed;
    a.draw = draw;
    a.P = q.P;
    a.G = q.G;
    a.R = (c->N + c->Gr - 1) / c->Gr;
    a.L = c->st;
    a.rec = c->records;
    cudaError_t ea = cudaFuncSetAttribute(substats_f32_kernel<DV, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)q.smem);
    if (ea != cudaSuccess) return ea;
    substats_f32_kernel<DV, XT><<<c->Gr, q.BT, q.smem, c->stream>>>(a);
    return cudaGetLastError();
}

template <typename XT>
static cudaError_t substats_mult_t(dpmm_ctx* c, uint64_t seed, int draw, const int* gate) {
    const StatLayout& L = c->st;
    // tiles of about 40 KB of rows: four CTAs per SM
    int P = (int)((40 * 1024) / ((size_t)L.dp * 4));
    P = std::max(32, std::min(256, P / 16 * 16));
    const int G = std::max(1, 256 / L.nblk);
    size_t head = (size_t)P * L.dp * 4 + (3 * (size_t)P + 2) * sizeof(int) + P;
    head = (head + 15) / 16 * 16;
    const size_t smem = head + ((size_t)2 * L.dp + 2) * 4 + 16 + (size_t)G * L.nblk * 8 * 4;
    SubArgs<float> a;
    a.kind = c->kind;
    a.d = c->d;
    a.xs = c->xs;
    a.N = c->N;
    a.X = c->X;
    a.pv = pview<float>(c);
    a.shift = c->shift32;
    a.z = c->z;
    a.zbar = c->zbar;
    a.idx = c->idx;
    a.dK = c->dK;
    a.diter = c->diter;
    a.gate = gate;
    a.seed = seed;
    a.draw = draw;
    a.P = P;
    a.G = G;
    a.R = (c->N + c->Gr - 1) / c->Gr;
    a.L = L;
    a.rec = c->records;
    cudaError_t ea = cudaFuncSetAttribute(substats_mult_kernel<XT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return ea;
    substats_mult_kernel<XT><<<c->Gr, 256, smem, c->stream>>>(a);
    return cudaGetLastError();
}

static size_t wide_smem(const dpmm_ctx* c) {
    return ((size_t)2 * 128 * 128 + 128 * WP + (size_t)WP * c->st.dp + 2 * WP + 256 + 256 + 128 + 4) * 4 +
           ((size_t)2 * WP + 2) * sizeof(int) + WP + 16;
}

template <typename XT>
static cudaError_t substats_wide_t(dpmm_ctx* c, uint64_t seed, int draw, const int* gate) {
    SubArgs<float> a;
    a.kind = c->kind;
    a.d = c->d;
    a.xs = c->xs;
    a.N = c->N;
    a.X = c->X;
    a.pv = pview<float>(c);
    a.shift = c->shift32;
    a.z = c->z;
    a.zbar = c->zbar;
    a.idx = c->idx;
    a.dK = c->dK;
    a.diter = c->diter;
    a.gate = gate;
    a.seed = seed;
    a.draw = draw;
    a.P = WP;
    a.G = 1;
    a.R = (c->N + c->Gr - 1) / c->Gr;
    a.L = c->st;
    a.rec = c->records;
    const size_t smem = wide_smem(c);
    cudaError_t ea = cudaFuncSetAttribute(substats_wide_kernel<XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (ea != cudaSuccess) return ea;
    substats_wide_kernel<XT><<<c->Gr, WIDE_T, smem, c->stream>>>(a);
    return cudaGetLastError();
}

// dense multinomial data on the reduced-precision paths: mult_warp_kernel and its compact counts
bool mult_direct(const dpmm_ctx* c) {
    return c->kind == DPMM_PRIOR_DIRICHLET && !c->sparse && c->prec != DPMM_PREC_FP64_PLAIN && c->d <= 256 && c->mcnt &&
           c->xdt == 2 && (c->xs & 7) == 0;
}

static cudaError_t mult_direct_t(dpmm_ctx* c, uint64_t seed, int draw, const int* gate) {
    const dim3 sg((unsigned)std::min(8, (c->d + 1 + 255) / 256), (unsigned)(2 * c->K_max));
    mcnt_zero_kernel<<<sg, 256, 0, c->stream>>>(c->dK, gate, c->d, c->mcnt);
    MwArgs a;
    a.N = c->N;
    a.d = c->d;
    a.xs = c->xs;
    a.X = c->X;
    a.idx = c->idx;
    a.starts = c->tot;
    a.dK = c->dK;
    a.lt = c->q_logtheta;
    a.lc = c->q_c;
    a.diter = c->diter;
    a.seed = seed;
    a.gate = gate;
    a.draw = draw;
    a.zbar = c->zbar;
    a.cnt = c->mcnt;
    const int64_t warps = 24 * (int64_t)c->num_sms;  // three 256-thread blocks per SM
    a.R = std::max<int64_t>(1, (c->N + warps - 1) / warps);
    const unsigned grid = (unsigned)((((c->N + a.R - 1) / a.R) + 7) / 8);
    const int smem = 8 * MW_DEPTH * MW_ROWB;
    cudaError_t e = cudaFuncSetAttribute(mult_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    mult_warp_kernel<<<grid, 256, smem, c->stream>>>(a);
    mcnt_fill_kernel<<<sg, 256, 0, c->stream>>>(c->dK, gate, c->st, c->mcnt, c->stats);
    return cudaGetLastError();
}

static cudaError_t substats_dispatch(dpmm_ctx* c, uint64_t seed, int draw, const int* gate) {
    prof_begin(c, draw ? "substats" : "restats");
    cudaError_t e;
    if (mult_direct(c)) {
        e = mult_direct_t(c, seed, draw, gate);
        prof_end(c, draw ? "substats" : "restats");
        c->nlaunch += 3;
        return e;
    }
    const bool mult_fast = c->prec != DPMM_PREC_FP64_PLAIN && c->kind == DPMM_PRIOR_DIRICHLET && c->st.nblk <= 256;
    if (mult_fast) {
        e = c->xdt == 2 ? substats_mult_t<__nv_bfloat16>(c, seed, draw, gate) : substats_mult_t<float>(c, seed, draw, gate);
        prof_end(c, draw ? "substats" : "restats");
        c->nlaunch += 1;
        return e;
    }
    const bool fast = c->prec != DPMM_PREC_FP64_PLAIN && c->kind == DPMM_PRIOR_NIW && c->d <= 64 && c->st.nblk <= 256;
    if (substats_tc_supported(c)) e = launch_substats_tc(c, seed, draw, gate);
    else if (fast && c->d <= 32) e = c->xdt == 2 ? substats_f32_t<32, __nv_bfloat16>(c, seed, draw, gate)
                                             : substats_f32_t<32, float>(c, seed, draw, gate);
    else if (fast) e = c->xdt == 2 ? substats_f32_t<64, __nv_bfloat16>(c, seed, draw, gate)
                                   : substats_f32_t<64, float>(c, seed, draw, gate);
    else if (c->prec != DPMM_PREC_FP64_PLAIN && c->kind == DPMM_PRIOR_NIW && c->d <= 128 && c->st.nblk <= WIDE_T)
        e = c->xdt == 2 ? substats_wide_t<__nv_bfloat16>(c, seed, draw, gate) : substats_wide_t<float>(c, seed, draw, gate);
    else if (c->prec == DPMM_PREC_FP64_PLAIN) e = substats_t<double, double>(c, seed, draw, gate);
    else if (c->xdt == 2) e = substats_t<float, __nv_bfloat16>(c, seed, draw, gate);
    else e = substats_t<float, float>(c, seed, draw, gate);
    prof_end(c, draw ? "substats" : "restats");
    c->nlaunch += 1;
    return e;
}

cudaError_t launch_substats(dpmm_ctx* c, uint64_t seed, int draw_zbar) {
    return substats_dispatch(c, seed, draw_zbar, nullptr);
}

cudaError_t launch_combine(dpmm_ctx* c) {
    if (mult_direct(c)) return cudaSuccess;  // the counts went straight to the table
    prof_begin(c, "combine");
    cudaError_t e = combine_impl(c, nullptr);
    prof_end(c, "combine");
    c->nlaunch += 1;
    return e;
}

// statistics recomputed from the labels, only when the split/merge step changed them
cudaError_t launch_restats_gated(dpmm_ctx* c, const int* gate) {
    if (c->sparse) return launch_sparse(c, 0, 2, gate);
    cudaError_t e = sort_impl(c, gate);
    if (e == cudaSuccess) e = substats_dispatch(c, 0, 0, gate);
    if (e == cudaSuccess && !mult_direct(c)) {
        prof_begin(c, "combine");
        e = combine_impl(c, gate);
        prof_end(c, "combine");
        c->nlaunch += 1;
    }
    return e;
}

cudaError_t launch_init_labels(dpmm_ctx* c, uint64_t seed) {
    c->nlaunch += 1;
    init_labels_kernel<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(c->N, c->init_K, seed, c->diter, c->z,
                                                                                c->zbar);
    return cudaGetLastError();
}

}  // namespace dpmm
