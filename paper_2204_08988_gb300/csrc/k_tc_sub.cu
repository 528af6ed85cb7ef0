// k_tc_sub.cu -- the sub-cluster label step (Sec. 4.1 step (f), Eq. sample_sub_labels)
// and the sufficient statistics of every cluster and sub-cluster that the next
// parameter draws and the split/merge step read (Sec. 4.1), on the 5th-generation
// tensor cores: Gaussian model, d <= 32, TF32 mode.
//
// Points are visited in cluster order (the permutation of the counting sort).  The
// sorted positions are cut into G ranges of R points (range g: [g R, (g + 1) R)); a
// CTA takes ranges blockIdx.x, blockIdx.x + gridDim.x, ... and cuts each into tiles
// of at most 128 points that never straddle a cluster boundary, so a tile has one
// cluster k and one pair of sub-cluster parameters.
//   score : Y - B = X [W_k1 W_k2] - 1 [b_k1 b_k2] (M = 128 points, N = 64) exactly as
//           in the cluster label step (TF32 operands, -b split in two TF32 parts and
//           multiplied by a tile of ones); the score warps draw z-bar_i by Gumbel-max
//           over the two sub-cluster scores (Philox tag ZBAR, words 0 and 2).
//   stats : x~ = x - shift_k is split as hi + lo (two TF32 values).  With the points
//           as the MMA's K dimension, D = A B^T where A's rows are (hi, lo, 1) and B's
//           rows are (hi m_1, m_1, hi m_2, m_2) (m_h: sub-cluster masks), so D holds,
//           per sub-cluster, sum hi hi^T, sum lo hi^T, the first moments and the count;
//           S_h = HH + LH + LH^T leaves out only sum lo lo^T (relative 2^-22).  The
//           tensor cores' FP32 accumulation is not rounded to nearest, so D spans at
//           most GT tiles; the epilogue adds it into FP32 accumulators in shared memory
//           and, after the range's last tile of the cluster, writes record g + k in
//           FP64 (the 4 x 4 block layout the combine step sums).
// CTA roles (512 threads, one CTA per SM, persistent):
//   warps 0, 15 : gather of each tile's 128 rows by cp.async (16-byte pieces, written in
//                 the 128-byte swizzle pattern the MMA reads; completion on an mbarrier),
//                 64 rows each; warp 0 also bulk-copies each new cluster's sub-cluster
//                 factor image
//   warp 1      : TMEM allocation (512 columns) and the single-thread score MMA issue
//   warps 2-5   : score warps, one thread per point (TMEM lane): z-bar
//   warps 6-13  : operand warps, lane j = feature j: the transposed hi / lo operands of
//                 each half tile (64 points, double-buffered), then the accumulators
//                 and the records
//   warp 14     : the single-thread statistics MMA issue (a thread of its own, so that
//                 waiting for operands never holds back a score)
// Every mbarrier wait is bounded; on timeout the kernel records DPMM_ETIMEOUT, gives
// its copies and MMAs time to land, frees TMEM and returns.
#include <algorithm>

#include "dpmm_internal.cuh"
#include "tc_ptx.cuh"

namespace dpmm {

namespace tcs {

using namespace tc;

constexpr int XST = 4;                         // gathered X tiles in flight
constexpr int XBYTES = BM * 128;               // 128 points x 32 TF32
constexpr int IMG_BYTES = 64 * 128 + 64 * 32;  // factor image (SW128) + -b image (no swizzle)
constexpr int PIM_STRIDE = 11 * 1024;          // one staged image, 1024-aligned
constexpr int HP = 64;                         // points per half tile (stats MMA K per buffer)
constexpr int SA_ROWS = 128;                   // A: hi (0..31), lo (32..63), 1 (64), zero rows
constexpr int SB_ROWS = 80;                    // B: hi m1 (0..31), m1 (32), hi m2 (40..71), m2 (72)
constexpr int SA_BUF = (HP / 32) * SA_ROWS * 128;  // two 32-point K chunks
constexpr int SB_BUF = (HP / 32) * SB_ROWS * 128;
constexpr int FR = 65, FS = 81;                // accumulator rows (D rows 0..64), row stride
constexpr int GT = 4;                          // tiles per tensor-memory accumulation group
constexpr int NS = 4, NB = 8;                  // score warps, operand warps
constexpr int W_B = 2 + NS;                    // first operand warp (the score warps are 2 .. 1 + NS)
constexpr int W_T = W_B + NB;                  // statistics MMA warp
constexpr int W_P = W_T + 1;                   // second producer warp
constexpr int NTHREADS = 32 * (4 + NS + NB);
constexpr uint32_t TMEM_COLS = 512;            // score 2 x 64; statistics 2 x 80 at 128, 256
constexpr uint32_t SCORE_COL = 0, STAT_COL = 128;

constexpr size_t SMEM_BYTES = 1024 + (size_t)XST * XBYTES + 2 * (size_t)PIM_STRIDE + (size_t)BM * 8 * 4 +
                              2 * (size_t)SA_BUF + 2 * (size_t)SB_BUF + (size_t)FR * FS * 4 + 2 * BM;

struct Args {
    int64_t N, R;  // points; sorted positions per range
    int G;         // ranges (records g + k, g < G)
    int d;
    const int* dK;
    const int* starts;  // K + 1 cluster offsets in sorted order
    const int* idx;     // sorted position -> point
    const float* X;     // N x 32 (TF32 values)
    const uint32_t* diter;
    uint64_t seed;
    const unsigned char* img;  // K_max x IMG_BYTES sub-cluster factor images
    const float* qc;           // c_s
    const float* shift;        // K_max x d cluster shifts
    uint8_t* zbar;
    double* rec;  // (G + K_max) x 2 x E
    StatLayout L;
    const int* gate;
    int* derr;
};

// The tile sequence of one CTA; every role walks it identically.  A run is the range's
// tiles of one cluster; grp_end marks the last tile of an accumulation group.
struct Tiles {
    const int* st;
    int64_t N, R, pos, end;
    int G, K, g, k, pk, pg, tir;
    __device__ void init(const int* s, int K_, int64_t n, int64_t r, int G_) {
        st = s;
        K = K_;
        N = n;
        R = r;
        G = G_;
        g = K_ >= 1 ? (int)blockIdx.x - (int)gridDim.x : G_;  // no cluster: no tile
        pos = end = 0;
        k = 0;
        pk = pg = -1;
        tir = 0;
    }
    __device__ bool next(int64_t& p0, int& cnt, int& kk, int& gg, bool& newrun, bool& last, bool& grp_first,
                         bool& grp_end) {
        while (pos >= end) {
            g += (int)gridDim.x;
            if (g >= G) return false;
            pos = (int64_t)g * R;
            end = min(N, pos + R);
            k = 0;
        }
        while (k + 1 < K && (int64_t)st[k + 1] <= pos) ++k;
        const int64_t lim = min(end, (int64_t)st[k + 1]);
        if (lim <= pos) {  // the starts do not cover the points (never for consistent state)
            g = G;
            pos = end = 0;
            return false;
        }
        cnt = (int)min((int64_t)BM, lim - pos);
        p0 = pos;
        kk = k;
        gg = g;
        newrun = k != pk || g != pg;
        pk = k;
        pg = g;
        tir = newrun ? 0 : tir + 1;
        pos += cnt;
        last = pos >= lim;
        grp_first = tir % GT == 0;
        grp_end = last || tir % GT == GT - 1;
        return true;
    }
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
// the mbarrier receives one arrival when all of this thread's earlier cp.async are done
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr(bar)) : "memory");
}
// FP32 -> TF32, round to nearest (ties away from zero), for the finite values the operands
// hold: half a TF32 unit added to the magnitude bits, the 13 low bits cleared (a carry
// into the exponent is the correct rounding).  Two integer operations.
__device__ __forceinline__ float tf32_rna(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

template <bool DRAW>
__global__ void __launch_bounds__(NTHREADS, 1) substats_tc_kernel(Args a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* xs = base;                             // XST x XBYTES
    unsigned char* pim = xs + XST * XBYTES;               // 2 x PIM_STRIDE
    float* ones = (float*)(pim + 2 * PIM_STRIDE);         // BM x 8, no swizzle
    unsigned char* SA = (unsigned char*)(ones + BM * 8);  // 2 x SA_BUF
    unsigned char* SB = SA + 2 * SA_BUF;                  // 2 x SB_BUF
    float* F = (float*)(SB + 2 * SB_BUF);                 // FR x FS accumulators (row = D row)
    uint8_t* hq = (uint8_t*)(F + FR * FS);                // 2 x BM sub-labels (2: padding row)
    __shared__ uint64_t bars[2 * XST + 17];
    uint64_t* xfull = bars;           // XST (64 cp.async arrivals: two producer warps)
    uint64_t* xempty = bars + XST;    // XST (operand threads)
    uint64_t* pfull = bars + 2 * XST; // 2
    uint64_t* pempty = pfull + 2;     // 2 (MMA commit)
    uint64_t* sfull = pfull + 4;      // 2 (MMA commit)
    uint64_t* sempty = pfull + 6;     // 2 (score threads)
    uint64_t* hfull = pfull + 8;      // 2 (score threads)
    uint64_t* hempty = pfull + 10;    // 2 (operand threads)
    uint64_t* opfull = pfull + 12;    // 2, one per half-tile buffer (operand threads)
    uint64_t* opempty = pfull + 14;   // 2 (MMA commit)
    uint64_t* ebar = pfull + 16;      // 1 (operand threads)
    __shared__ int st[257];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = *a.dK;
    for (int k = threadIdx.x; k <= K; k += blockDim.x) st[k] = a.starts[k];
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int b = 0; b < XST; ++b) {
            mbar_init(&xfull[b], 64);
            mbar_init(&xempty[b], NB * 32);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&pfull[b], 1);
            mbar_init(&pempty[b], 1);
            mbar_init(&sfull[b], 1);
            mbar_init(&sempty[b], NS * 32);
            mbar_init(&hfull[b], NS * 32);
            mbar_init(&hempty[b], NB * 32);
            mbar_init(&opfull[b], NB * 32);
            mbar_init(&opempty[b], 1);
        }
        mbar_init(ebar, NB * 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // constant operand parts: the ones tile of the -b step (row m = (1, 1, 0, ..., 0),
    // no-swizzle element (m, kk) at (m / 8) * 256 + (kk / 4) * 128 + (m % 8) * 16 +
    // (kk % 4) * 4); A row 64 = 1 and rows 65.. = 0; B rows 33..39 and 73..79 = 0
    for (int e = threadIdx.x; e < BM * 8; e += blockDim.x) {
        const int m = e >> 3, kk = e & 7;
        ones[(m >> 3) * 64 + (kk >> 2) * 32 + (m & 7) * 4 + (kk & 3)] = kk < 2 ? 1.f : 0.f;
    }
    for (int e = threadIdx.x; e < 2 * (HP / 32) * (SA_ROWS - 64) * 32; e += blockDim.x) {
        const int c = e / ((SA_ROWS - 64) * 32), rem = e % ((SA_ROWS - 64) * 32);
        ((float*)(SA + c * (SA_ROWS * 128) + 64 * 128))[rem] = rem < 32 ? 1.f : 0.f;
    }
    for (int e = threadIdx.x; e < 2 * (HP / 32) * 14 * 32; e += blockDim.x) {
        const int c = e / (14 * 32), rem = e % (14 * 32), row = rem / 32;
        ((float*)(SB + c * (SB_ROWS * 128) + (row < 7 ? 33 + row : 66 + row) * 128))[rem % 32] = 0.f;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    volatile int* abort = &abort_flag;
    Tiles tl;
    tl.init(st, K, a.N, a.R, a.G);
    int64_t p0;
    int cnt, k, g;
    bool newrun, last, gfirst, gend;

    if (warp == 0 || warp == W_P) {
        // ------------------------------------------------------------ producers
        // Two warps gather 64 rows each; the point indices of the next tile are loaded
        // while the current one is issued.  Warp 0 also stages the factor images.
        const int pw = warp == 0 ? 0 : 1;
        bool ok = true;
        int it = 0, cidx = -1;
        Tiles tn = tl;  // one tile ahead: its indices are loaded early
        int64_t np0;
        int ncnt, nk, ng;
        bool nnew, nlast, ngf, nge;
        bool have = tn.next(np0, ncnt, nk, ng, nnew, nlast, ngf, nge);
        int pn0 = 0, pn1 = 0;  // rows 64 pw + lane and 64 pw + 32 + lane of the next tile
        auto load_idx = [&]() {
            const int r0 = 64 * pw + lane, r1 = r0 + 32;
            pn0 = a.idx[np0 + (r0 < ncnt ? r0 : 0)];
            pn1 = a.idx[np0 + (r1 < ncnt ? r1 : 0)];
        };
        if (have) load_idx();
        while (ok && tl.next(p0, cnt, k, g, newrun, last, gfirst, gend)) {
            const int pt0 = pn0, pt1 = pn1;
            have = tn.next(np0, ncnt, nk, ng, nnew, nlast, ngf, nge);
            if (have) load_idx();
            if (newrun) {
                ++cidx;
                if (DRAW && pw == 0) {
                    const int pb = cidx & 1;
                    if (lane == 0) {
                        ok = mbar_wait(&pempty[pb], (uint32_t)(((cidx >> 1) & 1) ^ 1), abort);
                        if (ok) {
                            mbar_expect_tx(&pfull[pb], IMG_BYTES);
                            bulk_load(pim + pb * PIM_STRIDE, a.img + (size_t)k * IMG_BYTES, IMG_BYTES, &pfull[pb]);
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) break;
                }
            }
            const int s = it % XST;
            if (lane == 0) ok = mbar_wait(&xempty[s], (uint32_t)(((it / XST) & 1) ^ 1), abort);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            // step t copies rows 64 pw + 4t .. + 3, eight lanes (16-byte chunks) per row
            // (padding rows repeat the first point and are masked later)
            unsigned char* xt = xs + (size_t)s * XBYTES;
            const int c = lane & 7;
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int rr = 4 * t + (lane >> 3);  // row within this warp's 64
                const int pr = __shfl_sync(0xffffffffu, t < 8 ? pt0 : pt1, rr & 31);
                const int r = 64 * pw + rr;
                cp_async16(xt + r * 128 + ((c ^ (r & 7)) << 4), a.X + (size_t)pr * 32 + c * 4);
            }
            cp_async_arrive(&xfull[s]);
            ++it;
        }
        if (!ok && lane == 0) {
            atomicExch(a.derr, (int)DPMM_ETIMEOUT);
            *abort = 1;
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ score MMA issue
        if (DRAW && lane == 0) {
            bool ok = true;
            const uint32_t idS = idesc(64, 2);
            int it = 0, cidx = -1;
            while (ok && tl.next(p0, cnt, k, g, newrun, last, gfirst, gend)) {
                if (newrun) {
                    ++cidx;
                    if (!mbar_wait(&pfull[cidx & 1], (uint32_t)((cidx >> 1) & 1), abort)) { ok = false; break; }
                }
                const int pb = cidx & 1, s = it % XST, sb = it & 1;
                if (!mbar_wait(&xfull[s], (uint32_t)((it / XST) & 1), abort)) { ok = false; break; }
                if (!mbar_wait(&sempty[sb], (uint32_t)(((it >> 1) & 1) ^ 1), abort)) { ok = false; break; }
                fence_after();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // cp.async data -> MMA
                const uint32_t xa = saddr(xs + (size_t)s * XBYTES), ba = saddr(pim + pb * PIM_STRIDE);
                const uint32_t dt = tmem + SCORE_COL + (uint32_t)(sb * 64);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) mma<2>(dt, sdesc(xa + kk * 32), sdesc(ba + kk * 32), idS, kk > 0);
                mma<2>(dt, sdesc_ns(saddr(ones)), sdesc_ns(ba + 64 * 128), idS, 1);  // - b
                mma_commit(&sfull[sb]);
                if (last) mma_commit(&pempty[pb]);  // the image may be replaced
                ++it;
            }
            if (!ok) {
                atomicExch(a.derr, (int)DPMM_ETIMEOUT);
                *abort = 1;
            }
        }
        __syncwarp();
    } else if (warp == W_T) {
        // ------------------------------------------------------------ statistics MMA issue
        if (lane == 0) {
            bool ok = true;
            const uint32_t idT = idesc(SB_ROWS, 2);
            int it = 0, grp = -1;
            while (ok && tl.next(p0, cnt, k, g, newrun, last, gfirst, gend)) {
                if (gfirst) ++grp;
                // the two half tiles into D[grp & 1]; the operand warps read that buffer's
                // previous group before they arrived on opfull for this one
                const uint32_t dt = tmem + STAT_COL + (uint32_t)((grp & 1) * 128);
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    if (!mbar_wait(&opfull[hf], (uint32_t)(it & 1), abort)) { ok = false; break; }
                    fence_after();
                    const uint32_t sa = saddr(SA + hf * SA_BUF), sbb = saddr(SB + hf * SB_BUF);
#pragma unroll
                    for (int c = 0; c < HP / 32; ++c)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma<2>(dt, sdesc(sa + c * SA_ROWS * 128 + kk * 32), sdesc(sbb + c * SB_ROWS * 128 + kk * 32),
                                   idT, !(gfirst && hf == 0 && c == 0 && kk == 0));
                    mma_commit(&opempty[hf]);
                }
                if (!ok) break;
                ++it;
            }
            if (!ok) {
                atomicExch(a.derr, (int)DPMM_ETIMEOUT);
                *abort = 1;
            }
        }
        __syncwarp();
    } else if (warp < W_B) {
        // ------------------------------------------------------------ score warps
        const int q = warp & 3, r = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        Key key{a.seed, a.diter[0], a.diter[1], a.diter[2]};
        float c0 = 0.f, c1 = 0.f;
        bool ok = true;
        int it = 0;
        while (ok && tl.next(p0, cnt, k, g, newrun, last, gfirst, gend)) {
            if (DRAW && newrun) {
                c0 = a.qc[3 * k + 1];
                c1 = a.qc[3 * k + 2];
            }
            const bool valid = r < cnt;
            const int i = a.idx[p0 + (valid ? r : 0)];
            const int b = it & 1;
            int h = 2;  // padding row: neither sub-cluster
            if (DRAW) {
                if (!mbar_wait(&sfull[b], (uint32_t)((it >> 1) & 1), abort)) { ok = false; break; }
                fence_after();
                float y0[32], y1[32];
                const uint32_t ta = tmem + lane_off + SCORE_COL + (uint32_t)(b * 64);
                tmem_ld32x2(ta, ta + 32, y0, y1);
                fence_before();
                mbar_arrive(&sempty[b]);
                const float s0 = c0 - 0.5f * sqsum32(y0), s1 = c1 - 0.5f * sqsum32(y1);
                if (valid) {
                    uint32_t w[4];
                    key.block((uint32_t)i, TAG_ZBAR, 0, w);
                    const float vl = s0 - __logf(-logf(u01_f32(w[0])));
                    const float vr = s1 - __logf(-logf(u01_f32(w[2])));
                    h = vr > vl ? 1 : 0;
                    a.zbar[i] = (uint8_t)h;
                }
            } else if (valid) {
                h = a.zbar[i];
            }
            if (!mbar_wait(&hempty[b], (uint32_t)(((it >> 1) & 1) ^ 1), abort)) { ok = false; break; }
            hq[b * BM + r] = (uint8_t)h;
            mbar_arrive(&hfull[b]);
            ++it;
        }
        if (!ok) {
            atomicExch(a.derr, (int)DPMM_ETIMEOUT);
            *abort = 1;
        }
    } else {
        // ------------------------------------------------------------ operand warps
        const int wb = warp - W_B;  // 0..7
        const int j = lane;         // feature
        const int d = a.d;
        const int q = warp & 3;     // TMEM lane quarter of the accumulator reads
        const int cpart = wb >> 2;  // columns [40 cpart, 40 cpart + 40) of D
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        float sj = 0.f;
        // Point quad wb + 8u of a half tile holds points 4 wb + e of K chunk u: their rows
        // of the X tile sit at (4 wb + e) * 128 within the chunk's 32 rows, feature j in
        // 16-byte chunk (j / 4) ^ ((4 wb + e) & 7).  In the operands, feature row j (and
        // 32 + j, 40 + j: the same row phase) takes the quad in 16-byte chunk wb ^ (j & 7).
        uint32_t xo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int pr = 4 * wb + e;
            xo[e] = (uint32_t)(pr * 128 + ((((j >> 2) ^ (pr & 7))) << 4) + (j & 3) * 4);
        }
        const uint32_t ao = (uint32_t)(j * 128 + ((wb ^ (j & 7)) << 4));
        bool ok = true, pending = false, ffirst = true;
        int it = 0, grp = -1, fc = 0;
        // add D of group gr (complete) into the accumulators: lanes of quarters 0..2
        // (D rows 0..95, of which 0..64 are used), 40 columns per warp pair
        auto consume = [&](int gr) {
            if (q == 3) return;
            fence_after();
            float dv[32], de[8];
            const uint32_t ta = tmem + lane_off + STAT_COL + (uint32_t)((gr & 1) * 128) + (uint32_t)(cpart * 40);
            tmem_ld32(ta, dv);
            tmem_ld8(ta + 32, de);
            fence_before();
            const int m = q * 32 + lane;
            if (m < FR) {
                float* Fr = F + m * FS + cpart * 40;
                if (ffirst) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) Fr[c] = dv[c];
#pragma unroll
                    for (int c = 0; c < 8; ++c) Fr[32 + c] = de[c];
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) Fr[c] += dv[c];
#pragma unroll
                    for (int c = 0; c < 8; ++c) Fr[32 + c] += de[c];
                }
            }
        };
        while (ok && tl.next(p0, cnt, k, g, newrun, last, gfirst, gend)) {
            if (newrun) sj = j < d ? a.shift[(size_t)k * d + j] : 0.f;
            if (gfirst) ++grp;
            const int s = it % XST, b = it & 1;
            if (!mbar_wait(&hfull[b], (uint32_t)((it >> 1) & 1), abort)) { ok = false; break; }
            if (!mbar_wait(&xfull[s], (uint32_t)((it / XST) & 1), abort)) { ok = false; break; }
            const unsigned char* xt = xs + (size_t)s * XBYTES;
            const uint8_t* hb = hq + b * BM;
            // one half tile: this warp's point quads wb and wb + 8 (K chunks 0 and 1)
            auto build = [&](const int hf) -> bool {
                if (!mbar_wait(&opempty[hf], (uint32_t)((it & 1) ^ 1), abort)) return false;
                if (hf == 1 && pending) {  // the previous group is complete: add it up
                    consume(grp - 1);
                    pending = false;
                    ffirst = false;
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const uint32_t hw = *(const uint32_t*)(hb + hf * HP + 4 * (wb + 8 * u));
                    const unsigned char* xr = xt + hf * (HP * 128) + u * (32 * 128);
                    float hi[4], lo[4], b0[4], b1[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float xt1 = *(const float*)(xr + xo[e]) - sj;
                        hi[e] = tf32_rna(xt1);
                        lo[e] = tf32_rna(xt1 - hi[e]);
                        const uint32_t he = (hw >> (8 * e)) & 0xFFu;
                        b0[e] = he == 0 ? hi[e] : 0.f;
                        b1[e] = he == 1 ? hi[e] : 0.f;
                    }
                    unsigned char* Ac = SA + hf * SA_BUF + u * (SA_ROWS * 128) + ao;
                    unsigned char* Bc = SB + hf * SB_BUF + u * (SB_ROWS * 128) + ao;
                    *(float4*)Ac = make_float4(hi[0], hi[1], hi[2], hi[3]);
                    *(float4*)(Ac + 32 * 128) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                    *(float4*)Bc = make_float4(b0[0], b0[1], b0[2], b0[3]);
                    *(float4*)(Bc + 40 * 128) = make_float4(b1[0], b1[1], b1[2], b1[3]);
                    {  // the mask rows (m_1 at row 32, m_2 at row 72) of the quad: lanes 0-7, one value each
                        const uint32_t he = (hw >> (8 * (j & 3))) & 0xFFu;
                        const float mv = he == (uint32_t)((j >> 2) & 1) ? 1.f : 0.f;
                        if (j < 8)
                            *(float*)(SB + hf * SB_BUF + u * (SB_ROWS * 128) + ((j >> 2) ? 72 : 32) * 128 + (wb << 4) +
                                      (j & 3) * 4) = mv;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&opfull[hf]);
                return true;
            };
            if (!build(0) || !build(1)) { ok = false; break; }
            if (!ok) break;
            mbar_arrive(&xempty[s]);
            mbar_arrive(&hempty[b]);
            ++it;
            if (gend) pending = true;
            if (!last) continue;
            // ---- the range's last tile of cluster k: write record g + k.  Every thread
            // has arrived on opfull for a later tile before any accumulator of the next
            // run is written, so the reads below finish first.
            if (!mbar_wait(&opempty[1], (uint32_t)((it - 1) & 1), abort)) { ok = false; break; }
            consume(grp);
            pending = false;
            mbar_arrive(ebar);
            if (!mbar_wait(ebar, (uint32_t)(fc & 1), abort)) { ok = false; break; }
            ++fc;
            ffirst = true;
            const int E = a.L.E;
            double* out = a.rec + (size_t)(g + k) * 2 * E;
            for (int e = wb * 32 + lane; e < 2 * E; e += NB * 32) {
                const int hh = e / E, ee = e % E;
                int jb, lb;
                a.L.blk_coords(ee >> 4, jb, lb);
                int j1 = jb * 4 + ((ee >> 2) & 3), l1 = lb * 4 + (ee & 3);
                if (j1 > l1) {
                    const int t = j1;
                    j1 = l1;
                    l1 = t;
                }
                const int cb = 40 * hh;
                double v = 0.0;
                if (l1 < d) {
                    v = (double)F[j1 * FS + cb + l1] + (double)F[(32 + j1) * FS + cb + l1] +
                        (double)F[(32 + l1) * FS + cb + j1];
                } else if (l1 == d && j1 < d) {
                    v = (double)F[j1 * FS + cb + 32] + (double)F[(32 + j1) * FS + cb + 32];
                } else if (l1 == d && j1 == d) {
                    v = (double)F[64 * FS + cb + 32];
                }
                out[e] = v;
            }
        }
        if (!ok) {
            atomicExch(a.derr, (int)DPMM_ETIMEOUT);
            *abort = 1;
        }
    }
    // teardown: every MMA and copy has been consumed on the normal path; after an
    // abort, give those in flight time to land before TMEM and shared memory go
    fence_before();
    __syncthreads();
    fence_after();
    if (*abort) __nanosleep(1000000);
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                                 : "memory");
}

// Sub-cluster factor images, one per cluster k (IMG_BYTES apart): row n = h * 32 + j
// holds W_s[l][j] (s = 3k + 1 + h, l = 0..31, zero beyond d) in the 128-byte swizzle
// pattern (16-byte chunk c of row n at chunk c ^ (n & 7)); then the -b image (no
// swizzle, 32 B per row, element (n, l) at (n / 8) * 256 + (l / 4) * 128 + (n % 8) *
// 16 + (l % 4) * 4) with row n = (-b_hi, -b_lo, 0, ...), b = sum_m mu_s[m] W_s[m][j]
// in FP64 with the factor as the tensor cores see it.
__global__ void image_kernel(const int* dK, int d, const double* pW, const double* pb, unsigned char* img) {
    const int K = *dK;
    const int64_t total = (int64_t)K * 64 * 32;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / 2048), n = (int)((e / 32) % 64), l = (int)(e % 32);
        const int h = n >> 5, j = n & 31, s = 3 * k + 1 + h;
        float* fb = (float*)(img + (size_t)k * IMG_BYTES);
        const double* W = pW + (size_t)s * d * d;
        float v = 0.f;
        if (j < d && l < d) v = round_tf32((float)W[(size_t)l * d + j]);
        fb[n * 32 + (((l >> 2) ^ (n & 7)) << 2) + (l & 3)] = v;
        if (l < 8) {
            float bv = 0.f;
            if (j < d && l < 2) {
                const double bj = pb[(size_t)s * d + j];  // formed once per sweep by derive_kernel
                const float hi = round_tf32((float)bj);
                bv = l == 0 ? -hi : -round_tf32((float)(bj - (double)hi));
            }
            float* nb = fb + 64 * 32;
            nb[(n >> 3) * 64 + (l >> 2) * 32 + (n & 7) * 4 + (l & 3)] = bv;
        }
    }
}

}  // namespace tcs

bool substats_tc_supported(const dpmm_ctx* c) {
    return c->kind == DPMM_PRIOR_NIW && c->prec == DPMM_PREC_TF32 && c->d >= 1 && c->d <= 32 && c->xs == 32 &&
           c->K_max <= 256;
}

cudaError_t substats_tc_prepare(dpmm_ctx* c) {
    const size_t bytes = (size_t)c->K_max * tcs::IMG_BYTES;
    if (!c->tcs_img) {
        cudaError_t e = cudaMalloc(&c->tcs_img, bytes);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c->tcs_img, 0, bytes, c->stream);
        if (e != cudaSuccess) return e;
    }
    tcs::image_kernel<<<256, 256, 0, c->stream>>>(c->dK, c->d, c->p_W, c->p_b, (unsigned char*)c->tcs_img);
    c->nlaunch += 1;
    return cudaGetLastError();
}

cudaError_t launch_substats_tc(dpmm_ctx* c, uint64_t seed, int draw, const int* gate) {
    if (draw && !c->tcs_img) return cudaErrorNotSupported;
    tcs::Args a;
    a.N = c->N;
    a.G = c->Gr;
    a.R = (c->N + c->Gr - 1) / c->Gr;
    a.d = c->d;
    a.dK = c->dK;
    a.starts = c->tot;
    a.idx = c->idx;
    a.X = (const float*)c->X;
    a.diter = c->diter;
    a.seed = seed;
    a.img = (const unsigned char*)c->tcs_img;
    a.qc = c->q_c;
    a.shift = c->shift32;
    a.zbar = c->zbar;
    a.rec = c->records;
    a.L = c->st;
    a.gate = gate;
    a.derr = c->derr;
    auto kern = draw ? tcs::substats_tc_kernel<true> : tcs::substats_tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcs::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = std::min(c->num_sms, c->Gr);
    kern<<<grid, tcs::NTHREADS, tcs::SMEM_BYTES, c->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace dpmm
