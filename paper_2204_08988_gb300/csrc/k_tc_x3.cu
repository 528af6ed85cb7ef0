// k_tc_x3.cu -- the cluster label step (Sec. 4.1 step (e), Eq. sample_labels) for
// Gaussian data of dimension up to 128 on the 5th-generation tensor cores, with split
// BF16 operands (precision DPMM_PREC_BF16X3).
//
// As in the TF32 kernel, s_ik = c_k - 1/2 ||x_i W_k - b_k||^2 (Lambda_k = W_k W_k^T,
// b_k = mu_k^T W_k) comes from the stacked contraction X [W_1 .. W_K] - 1 [b_1 .. b_K].
// At d > 32 a single TF32 product is too coarse: y = x W and b nearly cancel when
// Lambda_k's spectrum is wide, and the error grows with d.  So each operand is split
// into two BF16 values, x = x_h + x_l and W = W_h + W_l, and the contraction runs as
// the three products x_h W_h + x_l W_h + x_h W_l (x_l W_l is below the FP32 rounding of
// the result), FP32 accumulation in tensor memory; -b enters through one more K step,
// a tile of ones times the three BF16 parts of -b.  d is padded to dp = 64 or 128
// (zero features and zero factor rows and columns change nothing).
//
// Tiling (one persistent CTA per SM): a pass holds MT = 2 point tiles of 128 rows
// (x_h and x_l, SWIZZLE_128B K-major, 16 KB per 64 features) and streams every
// cluster's factor through a ring of shared-memory stages: stage A = W_h (dp rows x dp,
// the B operand) plus the -b block, stage B = W_l.  MMA shape M = 128, N = dp, K = 16.
// Each cluster's accumulators (MT x dp columns) alternate between TMEM buffers, so the
// epilogue of cluster k overlaps the MMAs of cluster k + 1.
//
// The epilogue thread owns one point: it sums the squares of the dp accumulator
// columns, forms s_ik, and keeps the Gumbel-max running over k with exact lazy draws:
// cluster k's Gumbel is drawn (Philox, tag Z, block k/2, word 0 or 2) only if s_ik plus
// the largest value an FP32 Gumbel can take reaches the best perturbed score so far, so
// skipped clusters could not have won and the argmax is that of every draw.
//
// CTA roles (320 threads):
//   warp 0    : producer (bulk copies of the pre-swizzled point tiles and factor stages)
//   warp 1    : TMEM allocation (512 columns) and the single-thread MMA issue
//   warps 2-9 : epilogue, warp w reads TMEM lane quarter w % 4 of tile (w - 2) / 4
// Every mbarrier wait is bounded; on timeout the kernel records DPMM_ETIMEOUT, drains
// its own copies (bounded), frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "dpmm_internal.cuh"
#include "tc_ptx.cuh"

namespace dpmm {
namespace x3 {

using namespace tc;
constexpr int MT = 2;              // point tiles per pass
constexpr int NEPI = 4 * MT;       // epilogue warps
constexpr int NTHREADS = 32 * (2 + NEPI);
constexpr uint32_t TMEM_COLS = 512;
constexpr int XBLK = BM * 128;     // one 64-feature block of a point tile (128 rows x 128 B)
constexpr int FSTMAX = 8;
// largest FP32 Gumbel value -log(-log(1 - 2^-24)) = 16.64, plus margin for the fast
// logarithm and the rounding of s + G
constexpr float GSKIP = 17.0f;

struct Geo {
    int dp, KB;       // padded dimension, 64-feature blocks
    int fst, nbuf;    // factor stages, TMEM buffers
    uint32_t wbytes;  // one factor half: KB x (dp rows x 128 B)
    uint32_t sbytes;  // one stage: wbytes + dp x 32 B (-b block)
    uint32_t cbytes;  // one cluster in the factor image: 2 wbytes + dp x 32
    uint32_t xtile;   // one point tile: 2 KB x XBLK (x_h blocks, then x_l blocks)
};

struct Args {
    int64_t N;
    Geo g;
    int Kmax;
    const int* dK;
    const uint32_t* diter;
    uint64_t seed;
    const unsigned char* ximg;  // point tiles, pre-swizzled; npass * MT tiles
    const unsigned char* fimg;  // factor image, K_max clusters of g.cbytes
    const float* qc;            // c_k at slot 3k
    int32_t* z;
    int* derr;
    double* scores;             // optional N x K scores (test hook), else null
};

__device__ __noinline__ void gumbel_draw(uint64_t seed, uint32_t iter, uint32_t prob, uint32_t i, int k, float sc,
                                         float* best,
                                         int* zb) {
    Key key{seed, iter, prob, 0};  // i is the point's index in the whole data set
    uint32_t w[4];
    key.block(i, TAG_Z, (uint32_t)(k >> 1), w);
    const float u = u01_f32((k & 1) ? w[2] : w[0]);
    const float v = sc - __logf(-logf(u));
    if (v > *best) {  // clusters arrive in increasing k: a tie keeps the lower index
        *best = v;
        *zb = k;
    }
}

// shared memory: [point tiles (MT x xtile) | factor stages (fst x sbytes) | ones | c table | barriers]
template <bool SCORES>
__global__ void __launch_bounds__(NTHREADS, 1) labels_x3_kernel(Args a) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const Geo g = a.g;
    unsigned char* xs = base;                                   // MT x xtile
    unsigned char* fs = xs + (size_t)MT * g.xtile;              // fst x sbytes
    __nv_bfloat16* ones = (__nv_bfloat16*)(fs + (size_t)g.fst * g.sbytes);  // BM rows x 16, no swizzle
    float* ct = (float*)(ones + BM * 16);                       // Kmax
    uint64_t* bars = (uint64_t*)(((uintptr_t)(ct + a.Kmax) + 7) & ~(uintptr_t)7);
    uint64_t* xfull = bars;            // 1
    uint64_t* xempty = xfull + 1;      // 1
    uint64_t* ffull = xempty + 1;      // fst
    uint64_t* fempty = ffull + FSTMAX; // fst
    uint64_t* tfull = fempty + FSTMAX; // nbuf
    uint64_t* tempty = tfull + 4;      // nbuf
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = *a.dK;
    const int64_t ntiles = (a.N + BM - 1) / BM;
    const int64_t npass = (ntiles + MT - 1) / MT;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(xfull, 1);
        mbar_init(xempty, 1);
        for (int s = 0; s < g.fst; ++s) {
            mbar_init(&ffull[s], 1);
            mbar_init(&fempty[s], 1);
        }
        for (int b = 0; b < g.nbuf; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], NEPI * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // A operand of the -b step: every row (1, 1, 1, 0, ..., 0); element (m, kk) of the
    // no-swizzle layout at byte (m / 8) * 256 + (kk / 8) * 128 + (m % 8) * 16 + (kk % 8) * 2
    for (int e = threadIdx.x; e < BM * 16; e += blockDim.x) {
        const int m = e >> 4, kk = e & 15;
        ones[(m >> 3) * 128 + (kk >> 3) * 64 + (m & 7) * 8 + (kk & 7)] = __float2bfloat16_rn(kk < 3 ? 1.f : 0.f);
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) ct[k] = a.qc[3 * k];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // ones: generic writes, async-proxy reads
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    volatile int* abort = &abort_flag;
    const uint32_t ncols = (uint32_t)(MT * g.dp);  // one TMEM buffer

    if (warp == 0) {
        if (lane == 0) {
            int64_t it = 0;
            uint32_t pc = 0;  // factor stages issued
            bool ok = true;
            for (int64_t t = blockIdx.x; t < npass && ok; t += gridDim.x, ++it) {
                if (!tc::mbar_wait(xempty, (uint32_t)((it & 1) ^ 1), abort)) { ok = false; break; }
                const uint32_t xb = (uint32_t)MT * g.xtile;
                tc::mbar_expect_tx(xfull, xb);
                const unsigned char* src = a.ximg + (size_t)t * xb;
                for (uint32_t off = 0; off < xb; off += 32768u)
                    tc::bulk_load(xs + off, src + off, min(32768u, xb - off), xfull);
                for (int k = 0; k < K && ok; ++k) {
                    for (int h = 0; h < 2; ++h, ++pc) {  // stage A: W_h and -b; stage B: W_l
                        const int s = (int)(pc % (uint32_t)g.fst);
                        if (!tc::mbar_wait(&fempty[s], ((pc / (uint32_t)g.fst) & 1u) ^ 1u, abort)) { ok = false; break; }
                        const uint32_t n = h == 0 ? g.sbytes : g.wbytes;
                        const unsigned char* fsrc = a.fimg + (size_t)k * g.cbytes + (h == 0 ? 0 : g.sbytes);
                        unsigned char* dst = fs + (size_t)s * g.sbytes;
                        tc::mbar_expect_tx(&ffull[s], n);
                        for (uint32_t off = 0; off < n; off += 32768u)
                            tc::bulk_load(dst + off, fsrc + off, min(32768u, n - off), &ffull[s]);
                    }
                }
            }
            if (!ok) {
                atomicExch(a.derr, (int)DPMM_ETIMEOUT);
                *abort = 1;
            }
            // own copies must land before the CTA may exit
            if (it > 0) tc::mbar_wait(xfull, (uint32_t)((it - 1) & 1), abort);
            const uint32_t f = (uint32_t)g.fst;
            for (uint32_t j = (pc > f ? pc - f : 0); j < pc; ++j) tc::mbar_wait(&ffull[j % f], (j / f) & 1u, abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = tc::idesc(g.dp, 1);
            int64_t it = 0;
            uint32_t pc = 0, cc = 0;  // factor stages consumed, clusters (TMEM buffer uses)
            bool ok = true;
            for (int64_t t = blockIdx.x; t < npass && ok; t += gridDim.x, ++it) {
                if (!tc::mbar_wait(xfull, (uint32_t)(it & 1), abort)) { ok = false; break; }
                tc::fence_after();
                const uint32_t xa = tc::saddr(xs);
                for (int k = 0; k < K && ok; ++k, ++cc) {
                    const int b = (int)(cc % (uint32_t)g.nbuf);
                    if (!tc::mbar_wait(&tempty[b], ((cc / (uint32_t)g.nbuf) & 1u) ^ 1u, abort)) { ok = false; break; }
                    for (int h = 0; h < 2; ++h, ++pc) {
                        const int s = (int)(pc % (uint32_t)g.fst);
                        if (!tc::mbar_wait(&ffull[s], (pc / (uint32_t)g.fst) & 1u, abort)) { ok = false; break; }
                        tc::fence_after();
                        const uint32_t fa = tc::saddr(fs + (size_t)s * g.sbytes);
                        for (int mt = 0; mt < MT; ++mt) {
                            const uint32_t dt = tmem + (uint32_t)b * ncols + (uint32_t)(mt * g.dp);
                            const uint32_t xt = xa + (uint32_t)mt * g.xtile;
                            // stage A: x_h W_h + x_l W_h, then -b; stage B: x_h W_l
                            const int nprod = h == 0 ? 2 : 1;
                            for (int pr = 0; pr < nprod; ++pr) {
                                const uint32_t xh = xt + (uint32_t)(pr * g.KB) * XBLK;
                                for (int kb = 0; kb < g.KB; ++kb)
#pragma unroll
                                    for (int kk = 0; kk < 4; ++kk)
                                        tc::mma<1>(dt, tc::sdesc(xh + kb * XBLK + kk * 32),
                                                   tc::sdesc(fa + (uint32_t)kb * (uint32_t)(g.dp * 128) + kk * 32), id,
                                                   (h | pr | kb | kk) != 0);
                            }
                            if (h == 0)
                                tc::mma<1>(dt, tc::sdesc_ns(tc::saddr(ones)), tc::sdesc_ns(fa + g.wbytes), id, 1u);
                        }
                        tc::mma_commit(&fempty[s]);
                    }
                    if (!ok) break;
                    tc::mma_commit(&tfull[b]);
                }
                if (!ok) break;
                tc::mma_commit(xempty);
            }
            if (!ok) {
                atomicExch(a.derr, (int)DPMM_ETIMEOUT);
                *abort = 1;
            }
        }
        __syncwarp();
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3, mt = ew >> 2;
        const int r = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const uint32_t iter = a.diter[0], prob = a.diter[1], poff = a.diter[2];  // poff: point offset (shards)
        uint32_t cc = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < npass && ok; t += gridDim.x) {
            const int64_t i = (t * MT + mt) * BM + r;
            float best = -INFINITY;
            int zb = 0;
            for (int k = 0; k < K; ++k, ++cc) {
                const int b = (int)(cc % (uint32_t)g.nbuf);
                if (!tc::mbar_wait(&tfull[b], (cc / (uint32_t)g.nbuf) & 1u, abort)) { ok = false; break; }
                tc::fence_after();
                const uint32_t ta = tmem + lane_off + (uint32_t)b * ncols + (uint32_t)(mt * g.dp);
                float q = 0.f;
                for (int c0 = 0; c0 < g.dp; c0 += 64) {
                    float ya[32], yb[32];
                    tc::tmem_ld32x2(ta + (uint32_t)c0, ta + (uint32_t)(c0 + 32), ya, yb);
                    q += tc::sqsum32(ya) + tc::sqsum32(yb);
                }
                tc::fence_before();
                tc::mbar_arrive(&tempty[b]);
                const float sc = ct[k] - 0.5f * q;
                if constexpr (SCORES) {  // test hook only: no FP64 in the production kernel
                    if (i < a.N) a.scores[i * K + k] = (double)sc;
                }
                if (sc + GSKIP > best) gumbel_draw(a.seed, iter, prob, (uint32_t)i + poff, k, sc, &best, &zb);
            }
            if (ok && i < a.N) a.z[i] = zb;
        }
        if (!ok) {
            atomicExch(a.derr, (int)DPMM_ETIMEOUT);
            *abort = 1;
        }
    }
    // teardown: MMAs must be complete before TMEM is released.  On the normal path the
    // epilogue has consumed every commit; after an abort, give in-flight MMAs time.
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (*abort && warp == 1) __nanosleep(1000000);
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Point tiles: tile T, half h (0: x_h, 1: x_l), 64-feature block kb, row r, feature
// j = kb * 64 + e at byte T * xtile + (h * KB + kb) * XBLK + r * 128 + ((e / 8) ^ (r % 8)) * 16
// + (e % 8) * 2 (the 128-byte swizzle pattern); rows beyond N and features beyond d are 0.
__global__ void x3_points_kernel(const float* X, int64_t N, int d, int xs, Geo g, int64_t ntile_pad,
                                 unsigned char* img) {
    const int64_t per_tile = (int64_t)2 * g.KB * BM * 64;
    const int64_t total = ntile_pad * per_tile;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t T = e / per_tile;
        const int rem = (int)(e % per_tile);
        const int hb = rem / (BM * 64), r = (rem / 64) % BM, el = rem % 64;
        const int h = hb / g.KB, kb = hb % g.KB;
        const int64_t row = T * BM + r;
        const int j = kb * 64 + el;
        const float x = (row < N && j < d) ? X[row * xs + j] : 0.f;
        const __nv_bfloat16 xh = __float2bfloat16_rn(x);
        const __nv_bfloat16 v = h == 0 ? xh : __float2bfloat16_rn(x - __bfloat162float(xh));
        const size_t off = (size_t)T * g.xtile + (size_t)hb * XBLK + (size_t)r * 128 + (((el >> 3) ^ (r & 7)) << 4) +
                           (el & 7) * 2;
        *(__nv_bfloat16*)(img + off) = v;
    }
}

// Factor image, cluster k at k * cbytes: [W_h | -b | W_l].  A half holds KB blocks of dp
// rows (output column j) x 128 B (K index l = kb * 64 + e, swizzled as above with the
// row n = j); entry W_k[l][j] (zero beyond d).  The -b block (no swizzle, 32 B per row,
// element (j, kk) at (j / 8) * 256 + (kk / 8) * 128 + (j % 8) * 16 + (kk % 8) * 2) holds the
// three BF16 parts of -b_j, b_j = sum_m mu_m (W_h + W_l)[m][j] formed in FP64 with the
// factor as the tensor cores see it.
__global__ void x3_factor_kernel(const int* dK, int Kmax, int d, Geo g, const double* pW, const double* pmu,
                                 unsigned char* img) {
    const int K = min(*dK, Kmax);
    const int64_t per_k = (int64_t)2 * g.KB * g.dp * 64 + g.dp;
    const int64_t total = (int64_t)K * per_k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / per_k);
        const int rem = (int)(e % per_k);
        const double* W = pW + (size_t)3 * k * d * d;
        unsigned char* ck = img + (size_t)k * g.cbytes;
        if (rem < 2 * g.KB * g.dp * 64) {
            const int hb = rem / (g.dp * 64), n = (rem / 64) % g.dp, el = rem % 64;
            const int h = hb / g.KB, kb = hb % g.KB;
            const int l = kb * 64 + el;
            const double w = (l < d && n < d) ? W[(size_t)l * d + n] : 0.0;
            const __nv_bfloat16 wh = __float2bfloat16_rn((float)w);
            const __nv_bfloat16 v = h == 0 ? wh : __float2bfloat16_rn((float)(w - (double)__bfloat162float(wh)));
            const size_t off = (h == 0 ? 0 : (size_t)g.sbytes) + (size_t)kb * g.dp * 128 + (size_t)n * 128 +
                               (((el >> 3) ^ (n & 7)) << 4) + (el & 7) * 2;
            *(__nv_bfloat16*)(ck + off) = v;
        } else {
            const int j = rem - 2 * g.KB * g.dp * 64;
            double b = 0.0;
            if (j < d) {
                const double* mu = pmu + (size_t)3 * k * d;
                for (int m = 0; m < d; ++m) {
                    const double w = W[(size_t)m * d + j];
                    const float wh = __bfloat162float(__float2bfloat16_rn((float)w));
                    const float wl = __bfloat162float(__float2bfloat16_rn((float)(w - (double)wh)));
                    b += mu[m] * ((double)wh + (double)wl);
                }
            }
            const __nv_bfloat16 b0 = __float2bfloat16_rn((float)b);
            const double r1 = b - (double)__bfloat162float(b0);
            const __nv_bfloat16 b1 = __float2bfloat16_rn((float)r1);
            const __nv_bfloat16 b2 = __float2bfloat16_rn((float)(r1 - (double)__bfloat162float(b1)));
            __nv_bfloat16* nb = (__nv_bfloat16*)(ck + g.wbytes);
            for (int kk = 0; kk < 16; ++kk) {
                const __nv_bfloat16 v = kk == 0 ? __hneg(b0) : kk == 1 ? __hneg(b1) : kk == 2 ? __hneg(b2)
                                                                                     : __float2bfloat16_rn(0.f);
                nb[(j >> 3) * 128 + (kk >> 3) * 64 + (j & 7) * 8 + (kk & 7)] = v;
            }
        }
    }
}

}  // namespace x3

// -------------------------------------------------------------------------- host
static x3::Geo x3_geo(const dpmm_ctx* c, size_t* smem) {
    x3::Geo g;
    g.dp = c->d <= 64 ? 64 : 128;
    g.KB = g.dp / 64;
    g.wbytes = (uint32_t)g.KB * (uint32_t)g.dp * 128u;
    g.sbytes = g.wbytes + (uint32_t)g.dp * 32u;
    g.cbytes = 2 * g.wbytes + (uint32_t)g.dp * 32u;
    g.xtile = (uint32_t)(2 * g.KB * x3::XBLK);
    g.nbuf = (int)(x3::TMEM_COLS / (uint32_t)(x3::MT * g.dp));
    if (g.nbuf > 4) g.nbuf = 4;
    const size_t fixed = 1024 + (size_t)x3::MT * g.xtile + (size_t)tc::BM * 16 * 2 + (size_t)c->K_max * 4 + 8 +
                         (size_t)(2 + 2 * x3::FSTMAX + 8) * 8;
    const size_t limit = 227 * 1024 - 2048;  // room for the static shared memory (1 KB with its alignment)
    g.fst = (int)std::min<size_t>(x3::FSTMAX, (limit - fixed) / g.sbytes);
    if (smem) *smem = fixed + (size_t)g.fst * g.sbytes;
    return g;
}

bool x3_supported(const dpmm_ctx* c) {
    return c->kind == DPMM_PRIOR_NIW && c->prec == DPMM_PREC_BF16X3 && c->d >= 1 && c->d <= 128;
}

static int64_t x3_ntile_pad(const dpmm_ctx* c) {
    const int64_t ntiles = (c->N + 127) / 128;
    return (ntiles + x3::MT - 1) / x3::MT * x3::MT;
}

// after the data are stored (centred FP32): allocate the point and factor images and
// split the points into their BF16 parts
cudaError_t x3_prepare_data(dpmm_ctx* c) {
    if (!x3_supported(c)) return cudaSuccess;
    const x3::Geo g = x3_geo(c, nullptr);
    const int64_t nt = x3_ntile_pad(c);
    const size_t xbytes = (size_t)nt * g.xtile;
    if (!c->x3_ximg) {
        cudaError_t e = cudaMalloc(&c->x3_ximg, xbytes);
        if (e != cudaSuccess) return e;
    }
    if (!c->x3_fimg) {
        cudaError_t e = cudaMalloc(&c->x3_fimg, (size_t)c->K_max * g.cbytes);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c->x3_fimg, 0, (size_t)c->K_max * g.cbytes, c->stream);
        if (e != cudaSuccess) return e;
    }
    x3::x3_points_kernel<<<4 * c->num_sms, 256, 0, c->stream>>>((const float*)c->X, c->N, c->d, c->xs, g, nt,
                                                                (unsigned char*)c->x3_ximg);
    return cudaGetLastError();
}

// per sweep, after the parameters are drawn: the factor image
cudaError_t x3_prepare(dpmm_ctx* c) {
    if (!c->x3_fimg) return cudaErrorNotSupported;
    const x3::Geo g = x3_geo(c, nullptr);
    x3::x3_factor_kernel<<<2 * c->num_sms, 256, 0, c->stream>>>(c->dK, c->K_max, c->d, g, c->p_W, c->p_mu,
                                                                (unsigned char*)c->x3_fimg);
    c->nlaunch += 1;
    return cudaGetLastError();
}

cudaError_t launch_labels_x3(dpmm_ctx* c, uint64_t seed) {
    if (!c->x3_ximg || !c->x3_fimg) return cudaErrorNotSupported;
    size_t smem = 0;
    const x3::Geo g = x3_geo(c, &smem);
    if (g.fst < 2) return cudaErrorNotSupported;
    x3::Args a;
    a.N = c->N;
    a.g = g;
    a.Kmax = c->K_max;
    a.dK = c->dK;
    a.diter = c->diter;
    a.seed = seed;
    a.ximg = (const unsigned char*)c->x3_ximg;
    a.fimg = (const unsigned char*)c->x3_fimg;
    a.qc = c->q_c;
    a.z = c->z;
    a.derr = c->derr;
    a.scores = c->dbg_scores;
    auto kern = a.scores ? x3::labels_x3_kernel<true> : x3::labels_x3_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t npass = x3_ntile_pad(c) / x3::MT;
    const int grid = (int)std::min<int64_t>(c->num_sms, npass);
    prof_begin(c, "labels_x3");
    kern<<<grid, x3::NTHREADS, smem, c->stream>>>(a);
    prof_end(c, "labels_x3");
    c->nlaunch += 1;
    return cudaGetLastError();
}

}  // namespace dpmm
