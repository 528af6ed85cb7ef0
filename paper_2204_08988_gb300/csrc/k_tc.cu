// k_tc.cu -- the cluster label step (Sec. 4.1 step (e), Eq. sample_labels) on the
// 5th-generation tensor cores.
//
// The Gaussian log-likelihood of every point under every cluster is one stacked
// contraction: with Lambda_k = W_k W_k^T (W_k upper-triangular), y_k = x W_k and
// b_k = mu_k^T W_k, log N(x; mu_k, Lambda_k^-1) = c'_k - 1/2 ||y_k - b_k||^2.  So
// Y - B = X [W_1 ... W_K] - 1 [b_1 ... b_K] runs as tcgen05.mma (TF32 operands, FP32
// accumulation in tensor memory): four K steps over X and one more step that
// multiplies a constant tile of ones by -b (split as two exact TF32 values, so the
// subtraction keeps FP32 precision).  The epilogue adds log pi_k and the
// log-determinant (c_k), takes the squared norm of each d-wide block, and draws
// z_i = argmax_k (s_ik + G_ik) by Gumbel-max with Philox (tag Z, block k/2, word
// 0 or 2).  Gumbels are drawn only for clusters that can still win: a cluster whose
// score plus the largest possible FP32 Gumbel is below the best perturbed score seen
// so far is skipped, which leaves the argmax unchanged.
//
// Cluster groups: the factors of the clusters being scored are held in shared memory (up
// to capc clusters: 26 at d = 32).  More clusters are scored in groups of capc: each CTA
// passes over its tiles once per group, reloading the factor slice in between.  Between groups each point carries its best and
// second-best scores so far (and the cluster of the best), and the best perturbed score
// among the clusters drawn so far (and its cluster).  A group draws for its clusters within
// the window of the running best whenever two or more clusters are in that window, and
// also for the carried best cluster, whose draw was deferred while it stood alone; a
// cluster skipped in an earlier group was outside an earlier (lower) best's window and so
// is outside the final one.  The result is the same argmax as one pass over all clusters.
//
// CTA roles (608 threads, one CTA per SM, persistent over 128-point tiles):
//   warp 0     : TMA producer (X tiles, 128 rows x 128 B, SWIZZLE_128B, 3 stages)
//   warp 1     : TMEM allocation (512 columns) and the single-thread MMA issue
//   warps 2-17 : epilogue, four warps (parts) per TMEM lane quarter, part p taking
//                clusters p, p + 4, ... of a chunk; per tile each part publishes its two
//                best scores and every score in one of two slots and moves on
//   warp 18    : merge: per tile and point, the best over the parts, the Gumbel draws
//                when needed, and the label (or the carried state).
// The factor image of all clusters is copied once into shared memory (pre-swizzled
// by tc_prepare).  Accumulators are double-buffered in TMEM (NBUF = 2 buffers of 256
// columns; four buffers of 128 columns were slower: the cost per chunk is mostly fixed).
// Every mbarrier wait is bounded; on timeout the kernel records DPMM_ETIMEOUT,
// drains its own copies and MMAs (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "dpmm_internal.cuh"
#include "tc_ptx.cuh"

namespace dpmm {

namespace tc {

constexpr int XST = 3;           // X stages
constexpr int XBYTES = BM * 128; // one X tile: 128 rows x 128 B
constexpr int NPART = 4;         // epilogue warps per TMEM lane quarter
constexpr int EPI0 = 2;          // first epilogue warp
constexpr int NEPI = 4 * NPART;  // epilogue warps
constexpr int MRG = EPI0 + NEPI; // the merge warp
constexpr int NTHREADS = 32 * (MRG + 1);
// A cluster can win the Gumbel-max only if its score is within G_MAX - G_MIN of the
// best score (FP32 uniforms: 16.64 + 2.82), plus one nat for rounding.
constexpr float WINDOW = 20.5f;
constexpr uint32_t TMEM_COLS = 512;
constexpr int NBUF = 2;                        // TMEM accumulator buffers
constexpr int BUFCOLS = (int)TMEM_COLS / NBUF; // columns per buffer (the chunk width)

// per-point state carried from one cluster group to the next
struct Carry {
    float* g1;  // best score so far
    float* g2;  // second-best score so far
    float* v;   // best perturbed score among the clusters drawn so far (-inf: none)
    int* k1;    // cluster of the best score
    int* zv;    // cluster of the best perturbed score
};

struct Args {
    int64_t N;
    int d, dn;        // dimension and per-cluster column block (round_up(d, 8))
    int NC;           // clusters per MMA chunk (NC * dn <= BUFCOLS, multiple of 16)
    int cap_rows;     // factor rows that fit in shared memory
    int capc;         // clusters per group (cap_rows / dn)
    int gmax;         // most cluster groups (more clusters: the CUDA-core kernel)
    int img_rows;     // rows of the factor image in global memory (all K_max clusters)
    Carry carry;
    int Kmax;
    const int* dK;
    const uint32_t* diter;
    uint64_t seed;
    const void* img;  // factor image: rows (k * dn + j) x 128 B, swizzled; at img_rows * 128 B
                      // the -b image: rows x 32 B, no swizzle (8-row groups of 256 B)
    const float* qc;  // c_k, slot 3k
    int32_t* z;
    int* overflow;    // set to 1 when K does not fit (the CUDA-core kernel then runs)
    int* derr;
    double* scores;   // optional N x K scores (test hook), else null
};

// shared memory: [X stages | factor image | -b image | ones tile | scores | c table | barriers]
template <int FMT, bool SCORES>
__global__ void __launch_bounds__(NTHREADS, 1) labels_tc_kernel(const __grid_constant__ CUtensorMap xmap, Args a) {
    static_assert(FMT == 2, "the ones tile and the -b image hold TF32 values");
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* xs = base;                                   // XST x XBYTES
    unsigned char* bs = xs + XST * XBYTES;                      // cap_rows x 128
    unsigned char* bb = bs + (size_t)a.cap_rows * 128;          // cap_rows x 32
    float* ones = (float*)(bb + (size_t)a.cap_rows * 32);       // BM rows x 8, no swizzle
    float* sbuf = ones + BM * 8;                                // 2 slots x capc clusters x BM
    float* ct = sbuf + (size_t)2 * a.capc * BM;                  // 2 x Kmax: c_k of a group, by group parity
    uint64_t* bars = (uint64_t*)(((uintptr_t)(ct + 2 * a.Kmax) + 7) & ~(uintptr_t)7);
    uint64_t* full = bars;            // XST
    uint64_t* empty = full + XST;     // XST
    uint64_t* tfull = empty + XST;    // NBUF
    uint64_t* tempty = tfull + NBUF;  // NBUF
    uint64_t* bload = tempty + NBUF;  // 1: the group's factor image has landed (phase g & 1)
    uint64_t* facfree = bload + 1;    // 1: the group's last MMAs are complete (phase g & 1)
    uint64_t* sfull = facfree + 1;    // 2 (slot): every part has published its tile
    uint64_t* sfree = sfull + 2;      // 2 (slot): the merge warp has read it
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ float xm1[2][NPART][BM], xm2[2][NPART][BM];  // per part: best and second score
    __shared__ int xk1[2][NPART][BM];                         // per part: cluster of the best

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = *a.dK;
    const int ngroups = (K + a.capc - 1) / a.capc;
    if (ngroups > a.gmax) {  // too many groups: the CUDA-core kernel does the step
        if (blockIdx.x == 0 && threadIdx.x == 0) *a.overflow = 1;
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.overflow = 0;
    // the clusters of group g: [g capc, g capc + Kg(g))
    auto group_size = [&](int g) { return min(a.capc, K - g * a.capc); };
    const int64_t ntiles = (a.N + BM - 1) / BM;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < XST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], NEPI * 32);
        }
        mbar_init(bload, 1);
        mbar_init(facfree, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sfull[b], NEPI * 32);
            mbar_init(&sfree[b], 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // A operand of the fifth K step: every row (1, 1, 0, ..., 0); element (m, kk) of
    // the no-swizzle layout at (m / 8) * 256 + (kk / 4) * 128 + (m % 8) * 16 + (kk % 4) * 4
    for (int e = threadIdx.x; e < BM * 8; e += blockDim.x) {
        const int m = e >> 3, kk = e & 7;
        ones[(m >> 3) * 64 + (kk >> 2) * 32 + (m & 7) * 4 + (kk & 3)] = kk < 2 ? 1.f : 0.f;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    volatile int* abort = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {
            int64_t it = 0;  // X tiles loaded, over all groups
            bool ok = true;
            for (int g = 0; g < ngroups && ok; ++g) {
                // the group's slice of the factor image (its first row g capc dn is a multiple
                // of 8, so the swizzle phase and the 8-row groups of the -b image line up),
                // once the previous group's MMAs no longer read the old one
                if (g > 0 && !mbar_wait(facfree, (uint32_t)((g - 1) & 1), abort)) { ok = false; break; }
                const int kb = g * a.capc, rows_pad = (group_size(g) * a.dn + 15) / 16 * 16;
                const uint32_t bbytes = (uint32_t)rows_pad * 128u, nbytes = (uint32_t)rows_pad * 32u;
                // the group's c_k, published by this thread's arrival below (the epilogue of
                // group g - 2, the last reader of this half, has finished: the factors of
                // group g - 1 are no longer read)
                float* ctg = ct + (g & 1) * a.capc;
                for (int kk = 0; kk < group_size(g); ++kk) ctg[kk] = a.qc[3 * (kb + kk)];
                mbar_expect_tx(bload, bbytes + nbytes);
                const unsigned char* fsrc = (const unsigned char*)a.img + (size_t)kb * a.dn * 128;
                for (uint32_t off = 0; off < bbytes; off += 32768u) {
                    uint32_t n = min(32768u, bbytes - off);
                    bulk_load(bs + off, fsrc + off, n, bload);
                }
                const unsigned char* nsrc =
                    (const unsigned char*)a.img + (size_t)a.img_rows * 128 + (size_t)kb * a.dn * 32;
                for (uint32_t off = 0; off < nbytes; off += 32768u) {
                    uint32_t n = min(32768u, nbytes - off);
                    bulk_load(bb + off, nsrc + off, n, bload);
                }
                for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
                    const int s = (int)(it % XST);
                    const uint32_t ph = (uint32_t)((it / XST) & 1);
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort)) { ok = false; break; }
                    mbar_expect_tx(&full[s], XBYTES);
                    tma_load_2d(xs + (size_t)s * XBYTES, &xmap, 0, (int)(t * BM), &full[s]);
                }
                // own copies must land before the next group's factors are loaded over them
                if (ok && !mbar_wait(bload, (uint32_t)(g & 1), abort)) ok = false;
            }
            if (!ok) {
                atomicExch(a.derr, (int)DPMM_ETIMEOUT);
                *abort = 1;
            }
            // own copies must land before the CTA may exit
            for (int64_t j = (it > XST ? it - XST : 0); j < it; ++j)
                mbar_wait(&full[(int)(j % XST)], (uint32_t)((j / XST) & 1), abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            int64_t it = 0, ch = 0;
            for (int g = 0; g < ngroups && ok; ++g) {
                if (!mbar_wait(bload, (uint32_t)(g & 1), abort)) { ok = false; break; }
                const int Kg = group_size(g), nch = (Kg + a.NC - 1) / a.NC;
                for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
                    const int s = (int)(it % XST);
                    if (!mbar_wait(&full[s], (uint32_t)((it / XST) & 1), abort)) { ok = false; break; }
                    fence_after();
                    const uint32_t xa = saddr(xs + (size_t)s * XBYTES);
                    for (int c = 0; c < nch; ++c, ++ch) {
                        const int b = (int)(ch % NBUF);
                        if (!mbar_wait(&tempty[b], (uint32_t)(((ch / NBUF) & 1) ^ 1), abort)) { ok = false; break; }
                        fence_after();
                        const int nclus = min(a.NC, Kg - c * a.NC);
                        const int n = (nclus * a.dn + 15) / 16 * 16;
                        const uint32_t ba = saddr(bs + (size_t)c * a.NC * a.dn * 128);
                        const uint32_t nb = saddr(bb + (size_t)c * a.NC * a.dn * 32);
                        const uint32_t id = idesc(n, FMT);
                        const int ksteps = 4;  // 128-byte rows in 32-byte MMA steps
#pragma unroll
                        for (int kk = 0; kk < ksteps; ++kk)
                            mma<FMT>(tmem + (uint32_t)(b * BUFCOLS), sdesc(xa + kk * 32), sdesc(ba + kk * 32), id,
                                     kk > 0);
                        mma<FMT>(tmem + (uint32_t)(b * BUFCOLS), sdesc_ns(saddr(ones)), sdesc_ns(nb), id, true);  // - b
                        mma_commit(&tfull[b]);
                    }
                    if (!ok) break;
                    mma_commit(&empty[s]);
                }
                // the factor image may be replaced once this group's MMAs are complete
                if (ok) mma_commit(facfree);
            }
            if (!ok) {
                atomicExch(a.derr, (int)DPMM_ETIMEOUT);
                *abort = 1;
            }
        }
        __syncwarp();
    } else if (warp < MRG) {
        // parts: thread <-> TMEM lane (point row); NPART warps per lane quarter, part p
        // takes clusters cc = p, p + NPART, ... of every chunk.  Per tile a part publishes
        // its two best scores (and every score, for the rare draws) in slot it & 1 and goes
        // on to the next tile; the merge warp reads the slot.
        const int ew = warp - EPI0;
        const int quarter = warp & 3, part = ew >> 2;
        const int r = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        int64_t ch = 0, it = 0;
        bool ok = true;
        for (int g = 0; g < ngroups && ok; ++g) {
        const int kb = g * a.capc, Kg = group_size(g), nch = (Kg + a.NC - 1) / a.NC;
        // the group's c_k table (written before the factor copies' arrival)
        if (!mbar_wait(bload, (uint32_t)(g & 1), abort)) { ok = false; break; }
        const float* ctg = ct + (g & 1) * a.capc;
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
            const int64_t i = t * BM + r;
            const int sl = (int)(it & 1);
            // slot sl was last used two tiles ago: wait until the merge warp has read it
            if (it >= 2 && !mbar_wait(&sfree[sl], (uint32_t)(((it >> 1) - 1) & 1), abort)) { ok = false; break; }
            float m1 = -INFINITY, m2 = -INFINITY;
            int k1 = 0;
            float* sr = sbuf + (size_t)sl * a.capc * BM + r;  // score of the group's cluster kk at sr[kk * BM]
            auto score = [&](int kk, float q) {
                const float sc = ctg[kk] - 0.5f * q;
                if constexpr (SCORES) {  // test hook only: no FP64 in the production kernel
                    if (i < a.N) a.scores[i * K + kb + kk] = (double)sc;
                }
                sr[kk * BM] = sc;
                const bool gt = sc > m1;
                m2 = gt ? m1 : fmaxf(m2, sc);
                k1 = gt ? kb + kk : k1;
                m1 = gt ? sc : m1;
            };
            for (int c = 0; c < nch; ++c, ++ch) {
                const int b = (int)(ch % NBUF);
                if (!mbar_wait(&tfull[b], (uint32_t)((ch / NBUF) & 1), abort)) { ok = false; break; }
                fence_after();
                const int nclus = min(a.NC, Kg - c * a.NC);
                const uint32_t cbase = tmem + lane_off + (uint32_t)(b * BUFCOLS);
                if (a.dn == 32) {  // 32-column loads never pass the block's own columns
                    for (int cc = part; cc < nclus; cc += NPART) {
                        float y[32];
                        tmem_ld32(cbase + (uint32_t)(cc * 32), y);
                        score(c * a.NC + cc, sqsum32(y));
                    }
                } else {
                    for (int cc = part; cc < nclus; cc += NPART) {
                        float q0 = 0.f, q1 = 0.f;
                        for (int j0 = 0; j0 < a.dn; j0 += 8) {
                            float y[8];
                            tmem_ld8(cbase + (uint32_t)(cc * a.dn + j0), y);
#pragma unroll
                            for (int j = 0; j < 8; j += 2) {
                                q0 = fmaf(y[j], y[j], q0);
                                q1 = fmaf(y[j + 1], y[j + 1], q1);
                            }
                        }
                        score(c * a.NC + cc, q0 + q1);
                    }
                }
                // the warp's loads are complete (wait::ld); one lane arrives for the warp
                fence_before();
                mbar_arrive(&tempty[b]);
            }
            if (!ok) break;
            xm1[sl][part][r] = m1;
            xm2[sl][part][r] = m2;
            xk1[sl][part][r] = k1;
            mbar_arrive(&sfull[sl]);
        }
        }
        if (!ok) {
            atomicExch(a.derr, (int)DPMM_ETIMEOUT);
            *abort = 1;
        }
    } else {
        // merge warp: per tile and row (lane + 32 q), the best and second-best score over the
        // four parts and the earlier groups; Gumbel draws only when another cluster is
        // within the window (the best one wins whatever the Gumbel values otherwise); then
        // the label, or the state carried to the next group
        const uint32_t iter = *a.diter;
        Key key{a.seed, iter, a.diter[1], a.diter[2]};
        int64_t it = 0;
        bool ok = true;
        for (int g = 0; g < ngroups && ok; ++g) {
        const int kb = g * a.capc, Kg = group_size(g);
        const bool first = g == 0, final = g == ngroups - 1;
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
            const int sl = (int)(it & 1);
            if (!mbar_wait(&sfull[sl], (uint32_t)((it >> 1) & 1), abort)) { ok = false; break; }
            const float* sb = sbuf + (size_t)sl * a.capc * BM;
            for (int qr = 0; qr < 4; ++qr) {
                const int r = qr * 32 + lane;
                const int64_t i = t * BM + r;
                float g1 = xm1[sl][0][r], g2 = xm2[sl][0][r];
                int gk = xk1[sl][0][r];
#pragma unroll
                for (int p2 = 1; p2 < NPART; ++p2) {
                    const float o1 = xm1[sl][p2][r], o2 = xm2[sl][p2][r];
                    const int ok1 = xk1[sl][p2][r];
                    if (o1 > g1 || (o1 == g1 && ok1 < gk)) {
                        g2 = fmaxf(g1, o2);
                        g1 = o1;
                        gk = ok1;
                    } else {
                        g2 = fmaxf(g2, o1);
                    }
                }
                // the state carried from the earlier groups (their clusters have lower ids)
                float cg1 = -INFINITY, cg2 = -INFINITY, cv = -INFINITY;
                int ck1 = 0, cz = 0;
                if (!first && i < a.N) {
                    cg1 = a.carry.g1[i];
                    cg2 = a.carry.g2[i];
                    cv = a.carry.v[i];
                    ck1 = a.carry.k1[i];
                    cz = a.carry.zv[i];
                }
                if (!first) {
                    if (cg1 >= g1) {
                        g2 = fmaxf(g1, cg2);
                        g1 = cg1;
                        gk = ck1;
                    } else {
                        g2 = fmaxf(g2, cg1);
                    }
                }
                const float lim = g1 - WINDOW;
                const bool need = !(g2 <= lim);  // another cluster might win: draw
                float vbest = cv;  // best perturbed score among all clusters drawn so far
                int zbest = cz;
                if (need) {
                    float best = -INFINITY;
                    int zb = 0;
                    auto draw = [&](int k, float sc) {
                        uint32_t w[4];
                        key.block((uint32_t)i, TAG_Z, (uint32_t)(k >> 1), w);
                        const float u = u01_f32((k & 1) ? w[2] : w[0]);
                        const float v = sc - __logf(-logf(u));
                        if (v > best || (v == best && k < zb)) {
                            best = v;
                            zb = k;
                        }
                    };
                    for (int kk = 0; kk < Kg; ++kk) {
                        const float sc = sb[(size_t)kk * BM + r];
                        if (sc > lim) draw(kb + kk, sc);
                    }
                    // the carried best cluster: its draw was deferred until a rival appeared
                    // (drawing it again later gives the same value)
                    if (!first && cg1 > lim) draw(ck1, cg1);
                    if (cv > best || (cv == best && cz < zb)) {
                        best = cv;
                        zb = cz;
                    }
                    vbest = best;
                    zbest = zb;
                }
                if (i < a.N) {
                    if (final) {
                        a.z[i] = need ? zbest : gk;
                    } else {
                        // read back by this lane in the next group
                        a.carry.g1[i] = g1;
                        a.carry.g2[i] = g2;
                        a.carry.v[i] = vbest;
                        a.carry.k1[i] = gk;
                        a.carry.zv[i] = zbest;
                    }
                }
            }
            mbar_arrive(&sfree[sl]);
        }
        }
        if (!ok) {
            atomicExch(a.derr, (int)DPMM_ETIMEOUT);
            *abort = 1;
        }
    }
    // teardown: MMAs must be complete before TMEM is released.  On the normal path the
    // epilogue has consumed every commit; after an abort, give in-flight MMAs time.
    fence_before();
    __syncthreads();
    fence_after();
    if (*abort && warp == 1) __nanosleep(1000000);
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                                 : "memory");
}

// factor image: row n = k * dn + j holds W_k[l][j], l = 0..31 (zero beyond d), in the
// 128-byte swizzle pattern: 16-byte chunk c of row n sits at chunk c ^ (n & 7).  At
// byte offset img_rows * 128 (every cluster up to K_max) follows the -b image (no swizzle, 32 B per row, element
// (n, l) at (n / 8) * 256 + (l / 4) * 128 + (n % 8) * 16 + (l % 4) * 4): row n holds
// (-b_hi, -b_lo, 0, ..., 0), where b = sum_m mu_m W_k[m][j] is formed in FP64 with
// the factor as the tensor cores see it (by derive_kernel, once per sweep for every
// slot), b_hi = tf32(b) and b_lo = tf32(b - b_hi).
__global__ void tc_image_kernel(const int* dK, int Kmax, int d, int dn, const double* pW, const double* pb,
                                int img_rows, float* img) {
    const int K = *dK;
    const int rows = (K * dn + 15) / 16 * 16;
    const int64_t total = (int64_t)min(rows, img_rows) * 32;
    float* nb = img + (size_t)img_rows * 32;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(e / 32), l = (int)(e % 32);
        const int k = n / dn, j = n % dn;
        const bool live = k < K && k < Kmax && j < d;
        const double* W = pW + (size_t)3 * k * d * d;
        float v = 0.f;
        if (live && l < d) v = round_tf32((float)W[(size_t)l * d + j]);
        const int chunk = (l >> 2) ^ (n & 7);
        img[(size_t)n * 32 + chunk * 4 + (l & 3)] = v;
        if (l < 8) {
            float bv = 0.f;
            if (live && l < 2) {
                const double bj = pb[(size_t)3 * k * d + j];  // formed once per sweep by derive_kernel
                const float hi = round_tf32((float)bj);
                bv = l == 0 ? -hi : -round_tf32((float)(bj - (double)hi));
            }
            nb[(size_t)(n >> 3) * 64 + (l >> 2) * 32 + (n & 7) * 4 + (l & 3)] = bv;
        }
    }
}

}  // namespace tc

// -------------------------------------------------------------------------- host
PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn();
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() { return tc_encode_fn(); }

PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

struct TcCfg {
    int dn, NC, cap_rows, capc, gmax, img_rows;
    size_t smem;
};

// cluster groups per label step at most; K beyond gmax * capc goes to the CUDA-core kernel
constexpr int TC_GMAX = 4;

static TcCfg tc_cfg(const dpmm_ctx* c) {
    TcCfg q;
    q.dn = (c->d + 7) / 8 * 8;
    q.NC = tc::BUFCOLS / q.dn;
    while ((q.NC * q.dn) % 16) --q.NC;
    const size_t fixed = 1024 + tc::XST * tc::XBYTES + (size_t)tc::BM * 8 * 4 + (size_t)c->K_max * 8 + 32 * 8 + 64;
    const size_t limit = 227 * 1024 - 16384;  // leave room for the kernel's static shared memory (13 KB)
    // factor row, -b row, and each cluster's two slots of 128 scores spread over its dn rows
    const size_t per_row = 128 + 32 + (2 * tc::BM * 4 + q.dn - 1) / q.dn;
    size_t want = (size_t)((c->K_max * q.dn + 15) / 16 * 16) * per_row;
    size_t cap = std::min(want, limit - fixed);
    q.cap_rows = (int)(cap / per_row / 16 * 16);
    q.capc = q.cap_rows / q.dn;
    q.gmax = std::max(1, std::min(TC_GMAX, (c->K_max + q.capc - 1) / q.capc));
    // a group's slice starts at row kb * dn (a multiple of 8: the swizzle phase and the -b
    // image's 8-row groups line up) and is read padded to 16 rows, which can pass the last
    // cluster's rows by 8: 16 zero rows of slack
    q.img_rows = (c->K_max * q.dn + 15) / 16 * 16 + 16;
    q.smem = fixed + (size_t)q.cap_rows * (128 + 32) + (size_t)2 * (q.cap_rows / q.dn) * tc::BM * 4;
    if (q.smem < 120 * 1024) q.smem = 120 * 1024;  // one CTA per SM: it owns all 512 TMEM columns
    return q;
}

bool mult_supported(const dpmm_ctx* c);
cudaError_t mult_prepare(dpmm_ctx* c);
cudaError_t launch_labels_mult(dpmm_ctx* c, uint64_t seed);

bool tc_supported(const dpmm_ctx* c) {
    if (get_encode() == nullptr) return false;
    // Gaussian: TF32, one 128-byte swizzle atom in the contraction dimension;
    // multinomial: BF16 counts, up to four atoms
    return (c->kind == DPMM_PRIOR_NIW && c->prec == DPMM_PREC_TF32 && c->d >= 1 && c->d <= 32) || mult_supported(c);
}

cudaError_t tc_prepare(dpmm_ctx* c) {
    if (c->kind == DPMM_PRIOR_DIRICHLET) return mult_supported(c) ? mult_prepare(c) : cudaSuccess;
    if (c->prec != DPMM_PREC_TF32) return cudaSuccess;
    TcCfg q = tc_cfg(c);
    const size_t bytes = (size_t)q.img_rows * (128 + 32);
    if (!c->tc_img || c->tc_img_bytes < bytes) {
        if (c->tc_img) cudaFree(c->tc_img);
        c->tc_img = nullptr;
        cudaError_t e = cudaMalloc(&c->tc_img, bytes);
        if (e != cudaSuccess) return e;
        c->tc_img_bytes = bytes;
        // on the context's stream: a memset on the legacy stream is not ordered with the
        // image kernel below when the context's stream does not block on it
        e = cudaMemsetAsync(c->tc_img, 0, bytes, c->stream);
        if (e != cudaSuccess) return e;
    }
    tc::tc_image_kernel<<<256, 256, 0, c->stream>>>(c->dK, c->K_max, c->d, q.dn, c->p_W, c->p_b, q.img_rows,
                                                    (float*)c->tc_img);
    c->nlaunch += 1;
    return cudaGetLastError();
}

cudaError_t launch_labels_simt_gated(dpmm_ctx* c, uint64_t seed, const int* gate);

cudaError_t launch_labels_tc(dpmm_ctx* c, uint64_t seed) {
    if (c->kind == DPMM_PRIOR_DIRICHLET) return launch_labels_mult(c, seed);
    TcCfg q = tc_cfg(c);
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc || !c->tc_img) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)c->xs, (cuuint64_t)c->N};
    const cuuint64_t gstride[1] = {(cuuint64_t)c->xs * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)tc::BM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->X, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    if (!c->tc_flag) {
        cudaError_t e = cudaMalloc(&c->tc_flag, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(c->tc_flag, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) return e;
    }
    if (q.gmax > 1 && !c->tc_carry) return cudaErrorNotSupported;  // allocated with the data
    tc::Args a;
    a.N = c->N;
    a.d = c->d;
    a.dn = q.dn;
    a.NC = q.NC;
    a.cap_rows = q.cap_rows;
    a.capc = q.capc;
    a.gmax = q.gmax;
    a.img_rows = q.img_rows;
    {
        float* f = (float*)c->tc_carry;
        const size_t n = (size_t)c->N;
        a.carry = tc::Carry{f, f + n, f + 2 * n, (int*)(f + 3 * n), (int*)(f + 4 * n)};
    }
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
    auto kern = a.scores ? tc::labels_tc_kernel<2, true> : tc::labels_tc_kernel<2, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q.smem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (c->N + tc::BM - 1) / tc::BM;
    const int grid = (int)std::min<int64_t>(c->num_sms, ntiles);
    prof_begin(c, "labels_tc");
    kern<<<grid, tc::NTHREADS, q.smem, c->stream>>>(map, a);
    c->nlaunch += 1;
    prof_end(c, "labels_tc");
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // K beyond the groups' capacity: the CUDA-core kernel does the step (launched only
    // when K_max can exceed it)
    if ((int64_t)q.gmax * q.capc >= c->K_max) return cudaSuccess;
    return launch_labels_simt_gated(c, seed, c->tc_flag);
}

}  // namespace dpmm

namespace dpmm {
// bytes of the per-point state carried between cluster groups of the TF32 label step
// (0 when one group holds every cluster up to K_max)
size_t tc_carry_bytes(const dpmm_ctx* c) {
    if (c->kind != DPMM_PRIOR_NIW || c->prec != DPMM_PREC_TF32 || !tc_supported(c)) return 0;
    return tc_cfg(c).gmax > 1 ? (size_t)c->N * 20 : 0;
}
}  // namespace dpmm
