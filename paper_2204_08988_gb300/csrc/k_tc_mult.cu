// k_tc_mult.cu -- the multinomial cluster label step (Sec. 4.1 step (e) with
// multinomial components and a Dirichlet prior) on the tensor cores.
//
// log f(x_i; theta_k) = sum_j x_ij log theta_kj (the multinomial coefficient is the
// same for every k and is dropped), so the scores of all points under all clusters
// are the contraction X (N x d, counts, exact in BF16) times [log theta_1 ...
// log theta_K] (d x K).  log theta is split as hi + lo (two BF16 values, about 16
// significant bits together) and both halves accumulate into the same FP32 tensor
// memory columns: D = X hi + X lo.  The epilogue adds log pi_k and draws z_i by
// exact Gumbel-max (no draw when one cluster is out of reach of all others, as in the
// Gaussian kernel).  The data are read
// once from HBM; the kernel is bandwidth-bound by design.
//
// CTA roles (192 threads, persistent): warp 0 TMA producer (X tiles of 128 rows as up to
// four 128-byte K atoms, each atom its own stage of an 8-slot ring, so that up to
// 128 KB of X are in flight per SM), warp 1 TMEM owner and MMA issuer (per atom: the
// hi and the lo products, then the atom's slot is released), warps 2-5 epilogue (one
// per TMEM lane quarter).  All waits are bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "dpmm_internal.cuh"
#include "tc_ptx.cuh"

namespace dpmm {
namespace tcm {

using namespace tc;

constexpr int XS = 8;              // X atom slots
constexpr int ATOM = BM * 128;    // one K atom of an X tile: 128 rows x 128 B (64 BF16)
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 256;  // two 128-column accumulators
constexpr float WINDOW = 20.5f;

struct Args {
    int64_t N;
    int d, NA;        // dimension, K atoms (64 categories each)
    int cap_rows;     // cluster rows that fit (multiple of 16, <= 128)
    int Kmax;
    const int* dK;
    const uint32_t* diter;
    uint64_t seed;
    const void* img;  // [hi, lo][atom][cap_rows][128 B], swizzled
    const float* qc;  // log pi_k at slot 3k
    int32_t* z;
    int* overflow;
    int* derr;
    double* scores;
};

// one Gumbel-max draw (kept out of line: the unrolled epilogue must stay small)
__device__ __noinline__ void gumbel_update(uint64_t seed, uint32_t iter, uint32_t prob, uint32_t i, int k, float sc,
                                           float* best,
                                           int* zb) {
    Key key{seed, iter, prob, 0};  // i is the point's index in the whole data set
    uint32_t w[4];
    key.block(i, TAG_Z, (uint32_t)(k >> 1), w);
    const float u = u01_f32((k & 1) ? w[2] : w[0]);
    const float v = sc - __logf(-logf(u));
    if (v > *best || (v == *best && k < *zb)) {
        *best = v;
        *zb = k;
    }
}

template <bool SCORES>
__global__ void __launch_bounds__(NTHREADS, 1) labels_mult_kernel(const __grid_constant__ CUtensorMap xmap, Args a) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* xs = base;                                              // XS x ATOM
    unsigned char* bs = xs + (size_t)XS * ATOM;                            // 2 x NA x cap_rows x 128
    float* ct = (float*)(bs + (size_t)2 * a.NA * a.cap_rows * 128);        // Kmax
    uint64_t* bars = (uint64_t*)(((uintptr_t)(ct + a.Kmax) + 7) & ~(uintptr_t)7);
    uint64_t* full = bars;
    uint64_t* empty = full + XS;
    uint64_t* tfull = empty + XS;
    uint64_t* tempty = tfull + 2;
    uint64_t* bload = tempty + 2;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = *a.dK;
    const int NB = (K + 15) / 16 * 16;
    if (NB > a.cap_rows) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *a.overflow = 1;
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.overflow = 0;
    const int64_t ntiles = (a.N + BM - 1) / BM;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < XS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4 * 32);
        }
        mbar_init(bload, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) ct[k] = a.qc[3 * k];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    volatile int* abort = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {
            // log theta halves: NB rows of each (half, atom) block
            const uint32_t rb = (uint32_t)NB * 128u;
            mbar_expect_tx(bload, rb * 2u * (uint32_t)a.NA);
            for (int q = 0; q < 2 * a.NA; ++q)
                bulk_load(bs + (size_t)q * a.cap_rows * 128, (const unsigned char*)a.img + (size_t)q * a.cap_rows * 128,
                          rb, bload);
            uint32_t ac = 0;  // atoms issued
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int at = 0; at < a.NA; ++at, ++ac) {
                    const int s = (int)(ac % XS);
                    if (!mbar_wait(&empty[s], ((ac / XS) & 1u) ^ 1u, abort)) { ok = false; break; }
                    mbar_expect_tx(&full[s], (uint32_t)ATOM);
                    tma_load_2d(xs + (size_t)s * ATOM, &xmap, 64 * at, (int)(t * BM), &full[s]);
                }
            }
            if (!ok) {
                atomicExch(a.derr, (int)DPMM_ETIMEOUT);
                *abort = 1;
            }
            mbar_wait(bload, 0, abort);
            for (uint32_t j = (ac > (uint32_t)XS ? ac - XS : 0); j < ac; ++j)
                mbar_wait(&full[j % XS], (j / XS) & 1u, abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(bload, 0, abort);
            int64_t it = 0;
            uint32_t ac = 0;  // atoms consumed
            const uint32_t id = idesc(NB, 1);  // BF16 x BF16 -> FP32
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
                const int b = (int)(it & 1);
                if (!mbar_wait(&tempty[b], (uint32_t)(((it >> 1) & 1) ^ 1), abort)) { ok = false; break; }
                uint32_t acc = 0;
                for (int at = 0; at < a.NA; ++at, ++ac) {
                    const int s = (int)(ac % XS);
                    if (!mbar_wait(&full[s], (ac / XS) & 1u, abort)) { ok = false; break; }
                    fence_after();
                    const uint32_t xa = saddr(xs + (size_t)s * ATOM);
                    for (int half = 0; half < 2; ++half) {
                        const uint32_t ba = saddr(bs + ((size_t)half * a.NA + at) * a.cap_rows * 128);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            mma<1>(tmem + (uint32_t)(b * 128), sdesc(xa + kk * 32), sdesc(ba + kk * 32), id, acc);
                            acc = 1;
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[b]);
            }
            if (!ok) {
                atomicExch(a.derr, (int)DPMM_ETIMEOUT);
                *abort = 1;
            }
        }
        __syncwarp();
    } else {
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        int64_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
            const int64_t i = t * BM + r;
            const int b = (int)(it & 1);
            if (!mbar_wait(&tfull[b], (uint32_t)((it >> 1) & 1), abort)) { ok = false; break; }
            fence_after();
            // Exact Gumbel-max.  Pass 1 scores every cluster and keeps the two best; a
            // cluster can win only within WINDOW of the best, so when the second best is
            // outside it the best cluster is the label whatever the Gumbel values, and no
            // draw is made.  Otherwise the accumulators (still held) are read again and every
            // cluster within the window gets its draw.
            // four independent best/second-best trackers (cluster k in tracker k % 4), merged
            // at the end: a quarter of the dependent chain of one running maximum
            float t1[4], t2[4];
            int tk[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                t1[c] = t2[c] = -INFINITY;
                tk[c] = c;
            }
            const uint32_t iter = a.diter[0], prob = a.diter[1], poff = a.diter[2];  // poff: point offset (shards)
            const uint32_t tb = tmem + lane_off + (uint32_t)(b * 128);
            for (int k0 = 0; k0 < NB; k0 += 32) {
                float y[32];
                tmem_ld32(tb + (uint32_t)k0, y);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int k = k0 + j, c = j & 3;
                    const float sc = k < K ? ct[k] + y[j] : -INFINITY;
                    if constexpr (SCORES) {
                        if (k < K && i < a.N) a.scores[i * K + k] = (double)sc;
                    }
                    const bool gt = sc > t1[c];
                    t2[c] = gt ? t1[c] : fmaxf(t2[c], sc);
                    tk[c] = gt ? k : tk[c];
                    t1[c] = gt ? sc : t1[c];
                }
            }
            float m1 = t1[0], m2 = t2[0];
            int k1 = tk[0];
#pragma unroll
            for (int c = 1; c < 4; ++c) {  // ties keep the lower cluster index
                if (t1[c] > m1 || (t1[c] == m1 && tk[c] < k1)) {
                    m2 = fmaxf(m1, t2[c]);
                    m1 = t1[c];
                    k1 = tk[c];
                } else {
                    m2 = fmaxf(m2, t1[c]);
                }
            }
            const float lim = m1 - WINDOW;
            const bool need = !(m2 <= lim);
            int zb = k1;
            if (__any_sync(0xffffffffu, need)) {
                float best = -INFINITY;
                int zd = 0;
                for (int k0 = 0; k0 < NB; k0 += 32) {
                    float y[32];
                    tmem_ld32(tb + (uint32_t)k0, y);
                    if (need) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int k = k0 + j;
                            const float sc = k < K ? ct[k] + y[j] : -INFINITY;
                            if (sc > lim) gumbel_update(a.seed, iter, prob, (uint32_t)i + poff, k, sc, &best, &zd);
                        }
                    }
                }
                if (need) zb = zd;
            }
            fence_before();
            mbar_arrive(&tempty[b]);
            if (i < a.N) a.z[i] = zb;
        }
        if (!ok) {
            atomicExch(a.derr, (int)DPMM_ETIMEOUT);
            *abort = 1;
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (*abort && warp == 1) __nanosleep(1000000);
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                                 : "memory");
}

// log theta image: [half][atom][row n = cluster][64 BF16], 128-byte swizzle (16-byte
// chunk c of row n at chunk c ^ (n & 7)); hi = bf16(log theta), lo = bf16(log theta - hi)
__global__ void mult_image_kernel(const int* dK, int Kmax, int d, int NA, int cap_rows, const double* lt,
                                  __nv_bfloat16* img) {
    const int K = *dK;
    const int64_t total = (int64_t)2 * NA * cap_rows * 64;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % 64);
        const int n = (int)((e / 64) % cap_rows);
        const int at = (int)((e / 64 / cap_rows) % NA);
        const int half = (int)(e / 64 / cap_rows / NA);
        const int j = at * 64 + l;
        float v = 0.f;
        if (n < K && n < Kmax && j < d) {
            const double x = lt[(size_t)3 * n * d + j];
            const __nv_bfloat16 hi = __double2bfloat16(x);
            v = half == 0 ? __bfloat162float(hi) : __bfloat162float(__double2bfloat16(x - (double)__bfloat162float(hi)));
        }
        const size_t row = ((size_t)(half * NA + at) * cap_rows + n) * 64;
        img[row + (size_t)(((l >> 3) ^ (n & 7)) * 8 + (l & 7))] = __float2bfloat16_rn(v);
    }
}

}  // namespace tcm

// -------------------------------------------------------------------------- host
struct MultCfg {
    int NA, cap_rows;
    size_t smem;
};

static MultCfg mult_cfg(const dpmm_ctx* c) {
    MultCfg q;
    q.NA = (c->d + 63) / 64;
    const size_t fixed = 1024 + (size_t)tcm::XS * tcm::ATOM + (size_t)c->K_max * 4 + (2 * tcm::XS + 5) * 8 + 64;
    const size_t limit = 227 * 1024 - 4096;
    const size_t per_row = (size_t)2 * q.NA * 128;
    int cap = (int)((limit - fixed) / per_row);
    cap = std::min(cap, 128);
    cap = std::min(cap, (c->K_max + 15) / 16 * 16);
    q.cap_rows = cap / 16 * 16;
    q.smem = fixed + (size_t)q.cap_rows * per_row;
    if (q.smem < 120 * 1024) q.smem = 120 * 1024;  // one CTA per SM
    return q;
}

bool mult_supported(const dpmm_ctx* c) {
    return c->kind == DPMM_PRIOR_DIRICHLET && c->prec == DPMM_PREC_BF16 && c->d >= 1 && c->d <= 256;
}

cudaError_t mult_prepare(dpmm_ctx* c) {
    MultCfg q = mult_cfg(c);
    const size_t bytes = (size_t)2 * q.NA * q.cap_rows * 128;
    if (!c->tc_img || c->tc_img_bytes < bytes) {
        if (c->tc_img) cudaFree(c->tc_img);
        c->tc_img = nullptr;
        cudaError_t e = cudaMalloc(&c->tc_img, bytes);
        if (e != cudaSuccess) return e;
        c->tc_img_bytes = bytes;
    }
    tcm::mult_image_kernel<<<256, 256, 0, c->stream>>>(c->dK, c->K_max, c->d, q.NA, q.cap_rows, c->p_logtheta,
                                                      (__nv_bfloat16*)c->tc_img);
    c->nlaunch += 1;
    return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn();
cudaError_t launch_labels_simt_gated(dpmm_ctx* c, uint64_t seed, const int* gate);

cudaError_t launch_labels_mult(dpmm_ctx* c, uint64_t seed) {
    MultCfg q = mult_cfg(c);
    PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encode_fn();
    if (!enc || !c->tc_img) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)c->xs, (cuuint64_t)c->N};
    const cuuint64_t gstride[1] = {(cuuint64_t)c->xs * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)tc::BM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, c->X, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    if (!c->tc_flag) {
        cudaError_t e = cudaMalloc(&c->tc_flag, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(c->tc_flag, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) return e;
    }
    tcm::Args a;
    a.N = c->N;
    a.d = c->d;
    a.NA = q.NA;
    a.cap_rows = q.cap_rows;
    a.Kmax = c->K_max;
    a.dK = c->dK;
    a.diter = c->diter;
    a.seed = seed;
    a.img = c->tc_img;
    a.qc = c->q_c;
    a.z = c->z;
    a.overflow = c->tc_flag;
    a.derr = c->derr;
    a.scores = c->dbg_scores;
    auto kern = a.scores ? tcm::labels_mult_kernel<true> : tcm::labels_mult_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q.smem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (c->N + tc::BM - 1) / tc::BM;
    const int grid = (int)std::min<int64_t>(c->num_sms, ntiles);
    prof_begin(c, "labels_tc_mult");
    kern<<<grid, tcm::NTHREADS, q.smem, c->stream>>>(map, a);
    prof_end(c, "labels_tc_mult");
    c->nlaunch += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_labels_simt_gated(c, seed, c->tc_flag);
}

}  // namespace dpmm
