// dpmm_internal.cuh -- device helpers and the context layout of the sweep library.
//
// Random streams (same written specification as the public header):
//   Philox4x32-10 (Salmon et al., SC'11); key = (seed lo, seed hi); counter =
//   (c0 entity, c1 sweep index, c2 = tag << 24 | block, c3 problem).
//   FP64 uniform from words (a, b): ((((a >> 6) << 26) | (b >> 6)) * 2 + 1) * 2^-53.
//   FP32 uniform from word a: ((a >> 9) * 2 + 1) * 2^-24.
//   Normal q of a stream at base block B: Box-Muller on block B + q/2 (u1 = words
//   0,1; u2 = words 2,3), cos for even q, sin for odd q.
//   Gamma(a): Marsaglia-Tsang (2000) in log space, attempt r uses blocks B + 2r
//   (normal, cos branch) and B + 2r + 1 (uniform, words 0,1), <= 31 attempts;
//   a < 1 boosted by U^(1/a), U from block B + 63.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/dpmm.h"

namespace dpmm {

enum : uint32_t {
    TAG_INIT = 1, TAG_WEIGHT = 2, TAG_SUBW = 3, TAG_PARAM = 4, TAG_Z = 5,
    TAG_ZBAR = 6, TAG_SPLIT = 7, TAG_MERGE = 8, TAG_RESUB = 9
};

// Largest Gumbel value a uniform of each precision can produce, rounded up:
// FP64 u in [2^-53, 1 - 2^-53] gives G = -log(-log u) in [-3.61, 36.74];
// FP32 u in [2^-24, 1 - 2^-24] gives G in [-2.82, 16.64].  A cluster whose score
// plus G_MAX is below the best perturbed score so far cannot win the argmax.
constexpr double GUMBEL_MAX_F64 = 37.5;
constexpr float GUMBEL_MAX_F32 = 17.5f;

// multinomial data with more categories than this are held as compressed rows
constexpr int SPARSE_MIN_D = 256;
constexpr int DIRICHLET_MAX_D = 65536;
constexpr int SP_LGT = 1 << 16;  // entries of the lgamma-difference table (counts below it)
constexpr int SORT_TILE = 1024;  // points per tile of the counting sort (four rounds of 256 threads)

__host__ __device__ inline void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                       uint32_t k1, uint32_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
        uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// The entity word c0 of the point-keyed streams (tags INIT, Z, ZBAR, RESUB) is the point's
// index in the whole data set: poff + its index in this context's data (poff = 0 unless the
// data are one shard of a larger set, dpmm_set_shard).
__host__ __device__ inline bool point_tag(uint32_t tag) {
    return tag == TAG_INIT || tag == TAG_Z || tag == TAG_ZBAR || tag == TAG_RESUB;
}

struct Key {
    uint64_t seed;
    uint32_t iter;
    uint32_t problem;
    uint32_t poff;  // point offset of this context's data in the whole data set
    __host__ __device__ void block(uint32_t c0, uint32_t tag, uint32_t blk, uint32_t w[4]) const {
        if (point_tag(tag)) c0 += poff;
        philox(c0, iter, (tag << 24) | (blk & 0xFFFFFFu), problem, (uint32_t)seed, (uint32_t)(seed >> 32), w);
    }
};

__host__ __device__ inline double u01_f64(uint32_t a, uint32_t b) {
    uint64_t m = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    return (double)(2 * m + 1) * 1.1102230246251565e-16;  // 2^-53
}
__host__ __device__ inline float u01_f32(uint32_t a) {
    return (float)(2u * (a >> 9) + 1u) * 5.9604644775390625e-08f;  // 2^-24
}

__device__ inline double d_uniform(const Key& k, uint32_t c0, uint32_t tag, uint32_t blk) {
    uint32_t w[4];
    k.block(c0, tag, blk, w);
    return u01_f64(w[0], w[1]);
}

__device__ inline double d_normal(const Key& k, uint32_t c0, uint32_t tag, uint32_t base, uint32_t q) {
    uint32_t w[4];
    k.block(c0, tag, base + q / 2, w);
    double u1 = u01_f64(w[0], w[1]), u2 = u01_f64(w[2], w[3]);
    double r = sqrt(-2.0 * log(u1));
    // sin / cos of 2 pi u2 as sinpi / cospi of 2 u2: no argument reduction by pi
    return (q & 1) ? r * sinpi(2.0 * u2) : r * cospi(2.0 * u2);
}

__device__ inline float f_normal(const Key& k, uint32_t c0, uint32_t tag, uint32_t base, uint32_t q) {
    uint32_t w[4];
    k.block(c0, tag, base + q / 2, w);
    const float u1 = u01_f32(w[0]), u2 = u01_f32(w[2]);
    const float r = sqrtf(-2.f * logf(u1));
    return (q & 1) ? r * sinpif(2.f * u2) : r * cospif(2.f * u2);
}

// The FP32 form of d_log_gamma below (same Philox blocks, FP32 uniforms from the leading
// bits of the same words), for the reduced-precision path of high-dimensional
// multinomial data, whose FP64 draws would cost milliseconds per sweep on GB300's narrow
// FP64 pipes.  An accept/reject decision within FP32 rounding of its bound can differ
// from the FP64 one; the variate is then another draw from the same distribution.
__device__ inline float f_log_gamma(const Key& k, uint32_t c0, uint32_t tag, uint32_t base, float a) {
    float boost = 0.f;
    if (a < 1.f) {
        uint32_t w[4];
        k.block(c0, tag, base + 63, w);
        boost = logf(u01_f32(w[0])) / a;
        a += 1.f;
    }
    const float dd = a - 1.f / 3.f, c = rsqrtf(9.f * dd);
    for (uint32_t r = 0; r < 31; ++r) {
        const float x = f_normal(k, c0, tag, base + 2 * r, 0);
        float v = 1.f + c * x;
        if (v <= 0.f) continue;
        v = v * v * v;
        uint32_t w[4];
        k.block(c0, tag, base + 2 * r + 1, w);
        const float u = u01_f32(w[0]);
        if (logf(u) < 0.5f * x * x + dd - dd * v + dd * logf(v)) return logf(dd) + logf(v) + boost;
    }
    return logf(dd) + boost;
}

// log of a Gamma(a, 1) variate (Marsaglia & Tsang, ACM TOMS 2000), log space.
__device__ inline double d_log_gamma(const Key& k, uint32_t c0, uint32_t tag, uint32_t base, double a) {
    double boost = 0.0;
    if (a < 1.0) {
        boost = log(d_uniform(k, c0, tag, base + 63)) / a;
        a += 1.0;
    }
    double dd = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * dd);
    for (uint32_t r = 0; r < 31; ++r) {
        double x = d_normal(k, c0, tag, base + 2 * r, 0);
        double v = 1.0 + c * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        double u = d_uniform(k, c0, tag, base + 2 * r + 1);
        if (log(u) < 0.5 * x * x + dd - dd * v + dd * log(v)) return log(dd) + log(v) + boost;
    }
    return log(dd) + boost;
}

// Round an FP32 value to the nearest TF32 value (10 explicit mantissa bits, ties away
// from zero).  The tensor cores would otherwise truncate FP32 operands, which scales
// every product by up to 1 - 2^-10 in the same direction.
__host__ __device__ inline float round_tf32(float x) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, 4);
#endif
    if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float y;
    memcpy(&y, &u, 4);
    return y;
#endif
}

// ---------------------------------------------------------------- statistics
// The statistics of one sub-cluster are the upper triangle of M = sum_i xt xt^T
// with xt = [x - shift_k, 1, 0 ...] padded to dp = round_up(d + 1, 4): M[d][d] is
// the count, M[j][d] the first moment, M[j][l] (j <= l < d) the second moment.
// M is stored as 4x4 blocks: FULL mode keeps every block (jb <= lb), FIRST mode
// (multinomial) only the last block column lb = nb - 1.  E = 16 * blocks.
enum StatMode { STAT_FULL = 0, STAT_FIRST = 1 };

struct StatLayout {
    int d, dp, nb, mode, nblk, E;
    __host__ __device__ void init(int d_, int mode_) {
        d = d_;
        dp = (d_ + 1 + 3) / 4 * 4;
        nb = dp / 4;
        mode = mode_;
        nblk = mode_ == STAT_FULL ? nb * (nb + 1) / 2 : nb;
        E = 16 * nblk;
    }
    // block index of (jb, lb), jb <= lb
    __host__ __device__ int blk(int jb, int lb) const {
        return mode == STAT_FULL ? jb * nb - jb * (jb - 1) / 2 + (lb - jb) : jb;
    }
    __host__ __device__ void blk_coords(int b, int& jb, int& lb) const {
        if (mode == STAT_FIRST) { jb = b; lb = nb - 1; return; }
        int j = 0, rem = b;
        while (rem >= nb - j) { rem -= nb - j; ++j; }
        jb = j; lb = j + rem;
    }
    // entry of M[j][l] (j <= l)
    __host__ __device__ int ent(int j, int l) const { return blk(j >> 2, l >> 2) * 16 + (j & 3) * 4 + (l & 3); }
};

// ---------------------------------------------------------------- context
struct Profile {
    std::string name;
    std::vector<cudaEvent_t> ev;  // pairs (start, stop)
    int launches = 0;
    double ms = 0.0;
};

}  // namespace dpmm

struct dpmm_ctx {
    // configuration
    int kind = 0, d = 0, K_max = 0;
    double alpha = 1.0, kappa0 = 1.0, nu0 = 1.0, logdet_psi0 = 0.0;
    std::vector<double> m0, psi0, beta;
    int prec = DPMM_PREC_FP64_PLAIN, init_K = 1, burn_out = 15;
    unsigned step_mask = 7;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 148;
    std::string err;

    // data
    int64_t N = 0;
    int xdt = 0;           // storage: 0 fp64, 1 fp32, 2 bf16
    int xs = 0;            // row stride of X in elements
    void* X = nullptr;     // device
    double* center = nullptr;  // device, d: data were stored as x - center
    std::vector<double> h_center;
    dpmm_dtype in_dt = DPMM_F64;
    // staged input (dpmm_stage_data): the next sweep's values, copied on a copy stream of
    // their own while the current sweep runs, converted at the start of the next sweep
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_copied = nullptr, ev_free = nullptr;
    bool staged = false;

    // chain state
    int32_t* z = nullptr;
    uint8_t* zbar = nullptr;
    int* dK = nullptr;        // device: current K
    uint32_t* diter = nullptr;// device: [sweep counter, problem id, point offset] (Philox words c1, c3; c0 offset)
    int* age = nullptr;       // device, K_max
    int* counters = nullptr;  // device, 8
    int* derr = nullptr;      // device error word
    bool initialized = false;
    uint32_t h_iter = 0;      // host mirror of the sweep counter at last sync
    uint64_t seed = 0;

    // statistics
    dpmm::StatLayout st;
    double* stats = nullptr;       // 2 K_max x E
    double* shift_new = nullptr;   // K_max x d (storage coordinates)
    double* shift_stats = nullptr; // K_max x d: shift the statistics table was accumulated with
    float* shift32 = nullptr;      // K_max x d (fp32 copy of shift_new)

    // parameters, slots s = 3k + {0,1,2}
    double *p_logw = nullptr, *p_mu = nullptr, *p_W = nullptr, *p_logdetW = nullptr, *p_c = nullptr,
           *p_logtheta = nullptr;
    float *q_mu = nullptr, *q_W = nullptr, *q_c = nullptr, *q_b = nullptr, *q_logtheta = nullptr;
    double* p_b = nullptr;   // b = mu^T W per slot (FP64, TF32-rounded W on the TF32 path)
    void* tc_img = nullptr;  // tensor-core operand image of the cluster parameters
    size_t tc_img_bytes = 0;
    void* tcs_img = nullptr;  // tensor-core sub-cluster factor images (K_max x 10 KB)
    void* x3_ximg = nullptr;  // split-BF16 point tiles (BF16X3), pre-swizzled
    void* x3_fimg = nullptr;  // split-BF16 factor image (BF16X3), K_max clusters
    double* cweights = nullptr;  // K_max: pi_k of the last sweep (linear)
    double* eps = nullptr;       // 3 K_max x d: normals of the drawn means
    double* bart = nullptr;      // 3 K_max x d: Bartlett diagonal (chi-square roots)
    double* lgs = nullptr;       // 3 K_max + 1: log-Gamma draws of the weights
    int* retry = nullptr;        // 3 K_max: slots whose FP32 parameter draw is redone in FP64

    // sort / reduction scratch
    int T_tiles = 0;         // sort tiles of SORT_TILE points
    int* hist = nullptr;     // K_max x T_tiles
    int* tot = nullptr;      // K_max + 1: totals, then starts
    int* idx = nullptr;      // N: points sorted by cluster
    int G2 = 0;              // most ranges of the sub-label/statistics step (records capacity)
    int Gr = 1;              // ranges used for the current data: about one per 512 points, at most G2
    double* records = nullptr;  // (G2 + K_max) x 2 x E
    size_t records_bytes = 0;

    // split/merge scratch
    double* Ltab = nullptr;  // 3 K_max + K_max (K_max - 1)/2 log marginals, 1 spare, then per slot
                             // lgamma(n_s) and lgamma(alpha/2 + n_s) (6 K_max), then per merge
                             // pair lgamma(n) and lgamma(alpha + n) (K_max (K_max - 1))
    int* relabel = nullptr;  // 4 K_max
    int* acc = nullptr;      // K_max + K_max (K_max - 1)/2 accept flags of the split/merge proposals
    double* canon = nullptr; // canonical (n, xbar, C) per cluster and sub-cluster: 3 K_max x (1 + d + d d)

    // tensor-core path
    int* tc_flag = nullptr;        // device: 1 when K did not fit the tensor-core kernel
    void* tc_carry = nullptr;      // device: per-point state between cluster groups (TF32), N x 20 B

    // multinomial data of more than SPARSE_MIN_D categories: compressed rows
    bool sparse = false;
    int64_t nnz = 0;
    int64_t* csr_ptr = nullptr;    // N + 1
    int* csr_idx = nullptr;        // nnz categories, increasing within a row
    int* csr_val = nullptr;        // nnz counts
    void* sp_ltT = nullptr;        // d x round_up(K_max, 32) cluster log theta (FP64 or FP32)
    void* sp_ct = nullptr;         // K_max cluster log weights (FP64 or FP32)
    float* sp_cc = nullptr;        // 2 K_max x d compact sub-cluster counts
    unsigned* mcnt = nullptr;      // dense multinomial data: 2 K_max x (d + 1) sub-cluster counts
    double* sp_lgt = nullptr;      // lgamma(beta + c) - lgamma(beta), c < SP_LGT (uniform beta)
    double* sp_lgb = nullptr;      // lgamma(beta_j)
    void* sp_part = nullptr;       // 3 K_max x ceil(d / 2048) (max, sum exp) of the FP32 theta draws

    // point-sharded chains: this context's first point in the whole data set
    int64_t poff = 0;
    void* shard_scratch = nullptr; // the summed statistics of a sharded sweep (shard 0)
    double* dbg_scores = nullptr;  // device N x K scores when the score hook is active

    // one sweep captured as a CUDA graph (kernels read K and the sweep index from
    // device memory, so the graph is reused until the seed, mask or data change)
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_seed = 0;
    unsigned graph_mask = 0;
    bool use_graph = true;
    int64_t graph_kernels = 0;  // kernel nodes of the captured sweep

    // label-step kernel choice (Sec. 4.2): requested choice (dpmm_kernel), kernel in
    // force (0 tensor cores where the precision has them, 1 CUDA cores), a timing
    // pending for the next eager sweep, and the timed ms (tensor, CUDA cores; -1: none)
    int kchoice = 0, kuse = 0;
    bool ktune = false;
    float kms[2] = {-1.f, -1.f};

    // profiling: 0 off, 1 every kernel, 2 only the label kernel
    int profiling = 0;
    int64_t nlaunch = 0;  // kernels launched since the last dpmm_profile call
    std::vector<dpmm::Profile> prof;
};

namespace dpmm {
// Sub-cluster count sources of the multinomial model (slot 2k + h, category j): the FP32
// compact table of compressed-row data, or the FP64 statistics table of dense data (the one
// table a point-sharded chain exchanges).
struct CountsF32 {  // integer counts below 2^24: sums of a few stay exact in FP32
    const float* cc;
    int d;
    __device__ float operator()(int slot, int j) const { return cc[(size_t)slot * d + j]; }
};
struct CountsStats {
    const double* S;
    StatLayout L;
    __device__ double operator()(int slot, int j) const { return S[(size_t)slot * L.E + L.ent(j, L.d)]; }
};

// kernel launchers, one per .cu file group; each returns cudaGetLastError().
cudaError_t launch_weights(dpmm_ctx* c, uint64_t seed);
cudaError_t launch_params(dpmm_ctx* c, uint64_t seed);
cudaError_t launch_derive(dpmm_ctx* c);
cudaError_t launch_labels_simt(dpmm_ctx* c, uint64_t seed);
cudaError_t launch_labels_tc(dpmm_ctx* c, uint64_t seed);
cudaError_t launch_sort(dpmm_ctx* c);
cudaError_t launch_substats(dpmm_ctx* c, uint64_t seed, int draw_zbar);
cudaError_t launch_combine(dpmm_ctx* c);
bool mult_direct(const dpmm_ctx* c);
cudaError_t launch_init_labels(dpmm_ctx* c, uint64_t seed);
cudaError_t launch_splitmerge(dpmm_ctx* c, uint64_t seed, int labels_ran, int sm_enabled);
cudaError_t launch_relabel(dpmm_ctx* c, uint64_t seed);
cudaError_t launch_advance(dpmm_ctx* c);
bool tc_supported(const dpmm_ctx* c);
size_t tc_carry_bytes(const dpmm_ctx* c);
cudaError_t tc_prepare(dpmm_ctx* c);
bool substats_tc_supported(const dpmm_ctx* c);
cudaError_t substats_tc_prepare(dpmm_ctx* c);
cudaError_t launch_substats_tc(dpmm_ctx* c, uint64_t seed, int draw, const int* gate);
bool x3_supported(const dpmm_ctx* c);
cudaError_t x3_prepare_data(dpmm_ctx* c);
cudaError_t x3_prepare(dpmm_ctx* c);
cudaError_t launch_labels_x3(dpmm_ctx* c, uint64_t seed);
cudaError_t launch_wait_selftest(dpmm_ctx* c);
bool sparse_path(const dpmm_ctx* c);
cudaError_t sparse_build_dense(dpmm_ctx* c, const void* X, dpmm_dtype dt, int* bad);
cudaError_t sparse_prepare(dpmm_ctx* c);
cudaError_t launch_sparse(dpmm_ctx* c, uint64_t seed, int mode, const int* gate);
cudaError_t shard_exchange(dpmm_ctx* const* sh, int G, const int* gate);

// profiling helpers (no-ops unless enabled)
void prof_begin(dpmm_ctx* c, const char* name);
void prof_end(dpmm_ctx* c, const char* name);
}  // namespace dpmm
