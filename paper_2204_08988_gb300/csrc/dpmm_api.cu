// dpmm_api.cu -- the C ABI (include/dpmm.h): context, data upload, the sweep
// (Sec. 4.1) as a sequence of stream-ordered kernels, getters and test hooks.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dpmm_internal.cuh"

using namespace dpmm;

namespace dpmm {
cudaError_t launch_restats_gated(dpmm_ctx* c, const int* gate);

static bool prof_on(const dpmm_ctx* c, const char* name) {
    return c->profiling == 1 || (c->profiling == 2 && strncmp(name, "labels", 6) == 0);
}

// Every kernel group is also an NVTX range (named after the step) on the host thread that
// enqueues it, for timeline and ncu --nvtx filtering; ranges are recorded when the sweep is
// enqueued eagerly or captured, not when a captured graph is replayed.
void prof_begin(dpmm_ctx* c, const char* name) {
    nvtxRangePushA(name);
    if (!prof_on(c, name)) return;
    Profile* p = nullptr;
    for (auto& q : c->prof)
        if (q.name == name) p = &q;
    if (!p) {
        c->prof.push_back(Profile());
        p = &c->prof.back();
        p->name = name;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, c->stream);
    p->ev.push_back(e);
}

void prof_end(dpmm_ctx* c, const char* name) {
    nvtxRangePop();
    if (!prof_on(c, name)) return;
    for (auto& q : c->prof)
        if (q.name == name) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            cudaEventRecord(e, c->stream);
            q.ev.push_back(e);
            q.launches += 1;
            return;
        }
}
}  // namespace dpmm

// ------------------------------------------------------------------ helpers
static dpmm_status fail(dpmm_ctx* c, dpmm_status s, const std::string& m) {
    if (c) c->err = m;
    return s;
}

#define CK(c, x)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess) return fail((c), DPMM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename P>
static cudaError_t dalloc(P** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    // every buffer starts zeroed: no kernel result may depend on what the allocator
    // returned (the caller synchronises the device before the buffers are used)
    if (e == cudaSuccess) e = cudaMemset((void*)*p, 0, bytes);
    return e;
}

static void dfree(void* p) {
    if (p) cudaFree(p);
}

// host Cholesky, returns false when A is not positive definite; *logdet = log det A
static bool host_logdet_spd(const double* A, int d, double* logdet) {
    std::vector<double> L((size_t)d * d, 0.0);
    double s2 = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * d + j];
            for (int m = 0; m < j; ++m) s -= L[i * d + m] * L[j * d + m];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * d + i] = sqrt(s);
                s2 += log(L[i * d + i]);
            } else {
                L[i * d + j] = s / L[j * d + j];
            }
        }
    *logdet = 2.0 * s2;
    return true;
}

// ------------------------------------------------------------------ data kernels
template <typename IN>
__device__ inline double to_d(IN v) { return (double)v; }
template <>
__device__ inline double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <typename IN>
__global__ void colsum_kernel(const IN* X, int64_t N, int d, int64_t R, double* part) {
    const int g = blockIdx.x;
    const int64_t a = (int64_t)g * R, b = min(N, a + R);
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int64_t i = a; i < b; ++i) s += to_d(X[i * d + j]);
        part[(size_t)g * d + j] = s;
    }
}

__global__ void colmean_kernel(const double* part, int G, int d, int64_t N, double* center) {
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += part[(size_t)g * d + j];
        center[j] = s / (double)N;
    }
}

template <typename OUT>
__device__ inline OUT from_d(double v) { return (OUT)v; }
template <>
__device__ inline __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

template <typename IN, typename OUT>
__global__ void convert_kernel(const IN* X, int64_t N, int d, int xs, const double* center, int tf32, OUT* Y) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = N * xs;
    if (q >= total) return;
    const int64_t i = q / xs;
    const int j = (int)(q % xs);
    double v = 0.0;
    if (j < d) v = to_d(X[i * d + j]) - center[j];
    Y[q] = from_d<OUT>(v);
    if constexpr (sizeof(OUT) == 4) {
        if (tf32) Y[q] = round_tf32((float)Y[q]);  // the tensor-core operand, stored exactly
    }
}

template <typename IN>
static cudaError_t convert_any(dpmm_ctx* c, const IN* src, bool compute_center) {
    const int d = c->d;
    if (compute_center) {
        const int G = 256;
        int64_t R = (c->N + G - 1) / G;
        double* part = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&part, sizeof(double) * G * d, c->stream);
        if (e != cudaSuccess) return e;
        colsum_kernel<IN><<<G, 256, 0, c->stream>>>(src, c->N, d, R, part);
        colmean_kernel<<<1, 256, 0, c->stream>>>(part, G, d, c->N, c->center);
        cudaFreeAsync(part, c->stream);
    }
    int64_t total = c->N * c->xs;
    unsigned grid = (unsigned)((total + 255) / 256);
    const int tf32 = c->prec == DPMM_PREC_TF32;
    if (c->xdt == 0) convert_kernel<IN, double><<<grid, 256, 0, c->stream>>>(src, c->N, d, c->xs, c->center, 0, (double*)c->X);
    else if (c->xdt == 1) convert_kernel<IN, float><<<grid, 256, 0, c->stream>>>(src, c->N, d, c->xs, c->center, tf32, (float*)c->X);
    else convert_kernel<IN, __nv_bfloat16><<<grid, 256, 0, c->stream>>>(src, c->N, d, c->xs, c->center, 0, (__nv_bfloat16*)c->X);
    return cudaGetLastError();
}

static size_t dt_size(dpmm_dtype t) { return t == DPMM_F64 ? 8 : (t == DPMM_BF16 ? 2 : 4); }

// upload (host or device) input of type dt and convert it into the storage buffer
static dpmm_status upload(dpmm_ctx* c, const void* X, dpmm_dtype dt, int on_device, bool compute_center) {
    const size_t bytes = (size_t)c->N * c->d * dt_size(dt);
    const void* src = X;
    void* tmp = nullptr;
    if (!on_device) {
        // page-locked host memory is read by the conversion kernels in place (one pass over
        // the interconnect, no staging copy); pageable memory is staged in device memory
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, X) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
            src = at.devicePointer;
        } else {
            cudaGetLastError();
            CK(c, cudaMallocAsync(&tmp, bytes, c->stream));
            CK(c, cudaMemcpyAsync(tmp, X, bytes, cudaMemcpyHostToDevice, c->stream));
            src = tmp;
        }
    }
    cudaError_t e;
    switch (dt) {
        case DPMM_F64: e = convert_any(c, (const double*)src, compute_center); break;
        case DPMM_F32: e = convert_any(c, (const float*)src, compute_center); break;
        case DPMM_BF16: e = convert_any(c, (const __nv_bfloat16*)src, compute_center); break;
        default: e = convert_any(c, (const int32_t*)src, compute_center); break;
    }
    if (tmp) cudaFreeAsync(tmp, c->stream);
    CK(c, e);
    CK(c, x3_prepare_data(c));  // split-BF16 point tiles (BF16X3 only)
    return DPMM_OK;
}

static dpmm_status check_derr(dpmm_ctx* c) {
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (h != 0) {
        // cleared on the context's stream, so that the clear is ordered before any later
        // kernel of this chain (which may set the word again)
        cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream);
        cudaStreamSynchronize(c->stream);
        return fail(c, (dpmm_status)h, h == DPMM_ENUMERIC ? "non-positive-definite scale matrix or NaN seen on the device"
                                                         : "device error");
    }
    return DPMM_OK;
}

static void free_data(dpmm_ctx* c) {
    dfree(c->X); dfree(c->z); dfree(c->zbar); dfree(c->idx); dfree(c->hist); dfree(c->x3_ximg); dfree(c->tc_carry);
    dfree(c->csr_ptr); dfree(c->csr_idx); dfree(c->csr_val);
    c->X = nullptr; c->z = nullptr; c->zbar = nullptr; c->idx = nullptr; c->hist = nullptr; c->x3_ximg = nullptr;
    c->tc_carry = nullptr; c->csr_ptr = nullptr; c->csr_idx = nullptr; c->csr_val = nullptr; c->nnz = 0;
}

static void drop_graph(dpmm_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
}

// new data: an automatic label-kernel choice is made again for the new size
static void rearm_kernel_choice(dpmm_ctx* c) {
    if (c->kchoice != DPMM_KERNEL_AUTO) return;
    c->ktune = true;
    c->kuse = 0;
    c->kms[0] = c->kms[1] = -1.f;
}

// ------------------------------------------------------------------ compressed rows
// what every data set of the compressed-row path has in common: labels, the row
// pointer, the prior in storage coordinates (beta), the sweep counter reset
static dpmm_status sparse_alloc(dpmm_ctx* c, int64_t N) {
    free_data(c);
    c->N = N;
    rearm_kernel_choice(c);
    c->T_tiles = (int)((N + SORT_TILE - 1) / SORT_TILE);
    c->Gr = 1;
    bool ok = true;
    auto A = [&](auto** p, size_t bytes) { ok = ok && dalloc(p, bytes) == cudaSuccess; };
    A(&c->X, 16);  // no dense copy: a marker that data are set
    A(&c->z, sizeof(int32_t) * N);
    A(&c->zbar, N);
    A(&c->csr_ptr, sizeof(int64_t) * (N + 1));
    if (!ok) {
        cudaGetLastError();
        free_data(c);
        return fail(c, DPMM_ENOMEM, "device allocation for the data failed");
    }
    CK(c, cudaDeviceSynchronize());  // the zeroing memsets ran on the legacy stream
    return DPMM_OK;
}

static dpmm_status sparse_finish(dpmm_ctx* c) {
    const int d = c->d;
    std::vector<double> cen((size_t)2 * d + (size_t)d * d, 0.0);
    for (int j = 0; j < d; ++j) cen[d + j] = c->beta[j];
    c->h_center.assign(d, 0.0);
    CK(c, cudaMemcpyAsync(c->center, cen.data(), sizeof(double) * cen.size(), cudaMemcpyHostToDevice, c->stream));
    uint32_t zero = 0;
    CK(c, cudaMemcpyAsync(c->diter, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->initialized = false;
    c->h_iter = 0;
    return DPMM_OK;
}

// dense counts (host or device) -> compressed rows on the device
static dpmm_status sparse_upload(dpmm_ctx* c, const void* X, dpmm_dtype dt, int on_device) {
    const size_t bytes = (size_t)c->N * c->d * dt_size(dt);
    const void* src = X;
    void* tmp = nullptr;
    if (!on_device) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, X) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
            src = at.devicePointer;
        } else {
            cudaGetLastError();
            CK(c, cudaMallocAsync(&tmp, bytes, c->stream));
            CK(c, cudaMemcpyAsync(tmp, X, bytes, cudaMemcpyHostToDevice, c->stream));
            src = tmp;
        }
    }
    int* bad = nullptr;
    CK(c, cudaMallocAsync((void**)&bad, sizeof(int), c->stream));
    CK(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    cudaError_t e = sparse_build_dense(c, src, dt, bad);
    int hb = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (tmp) cudaFreeAsync(tmp, c->stream);
    cudaFreeAsync(bad, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    CK(c, e);
    if (hb) return fail(c, DPMM_EINVAL, "multinomial data must be non-negative integer counts below 2^24");
    return DPMM_OK;
}

static dpmm_status set_data_sparse(dpmm_ctx* c, const void* X, int64_t N, dpmm_dtype dt, int on_device) {
    dpmm_status s = sparse_alloc(c, N);
    if (s != DPMM_OK) return s;
    c->in_dt = dt;
    s = sparse_upload(c, X, dt, on_device);
    if (s != DPMM_OK) {
        free_data(c);
        return s;
    }
    return sparse_finish(c);
}

// ------------------------------------------------------------------ ABI
extern "C" {

const char* dpmm_last_error(const dpmm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dpmm_status dpmm_create(const dpmm_prior* prior, double alpha, int d, int K_max, dpmm_ctx** out) {
    if (!out) return DPMM_EINVAL;
    *out = nullptr;
    if (!prior || d < 1 || K_max < 1 || K_max > 1000 || !(alpha > 0.0)) return DPMM_EINVAL;
    double ld0 = 0.0;
    if (prior->kind == DPMM_PRIOR_NIW) {
        // d <= 160: the factorisations of the parameter and split/merge steps hold a d x d
        // FP64 matrix in one CTA's shared memory
        if (!prior->m0 || !prior->psi0 || !(prior->kappa0 > 0.0) || !(prior->nu0 > d - 1.0) || d > 160)
            return DPMM_EINVAL;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j)
                if (prior->psi0[i * d + j] != prior->psi0[j * d + i]) return DPMM_EINVAL;
        if (!host_logdet_spd(prior->psi0, d, &ld0)) return DPMM_EINVAL;
    } else if (prior->kind == DPMM_PRIOR_DIRICHLET) {
        if (!prior->beta || d > DIRICHLET_MAX_D) return DPMM_EINVAL;
        for (int j = 0; j < d; ++j)
            if (!(prior->beta[j] > 0.0)) return DPMM_EINVAL;
    } else {
        return DPMM_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return DPMM_ECUDA;
    dpmm_ctx* c = new dpmm_ctx();
    cudaGetDevice(&c->device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess || prop.major != 10 || prop.minor != 3) {
        delete c;
        return DPMM_ECUDA;  // built for sm_103a only
    }
    c->num_sms = prop.multiProcessorCount;
    c->kind = prior->kind;
    c->d = d;
    c->K_max = K_max;
    c->alpha = alpha;
    c->logdet_psi0 = ld0;
    if (c->kind == DPMM_PRIOR_NIW) {
        c->kappa0 = prior->kappa0;
        c->nu0 = prior->nu0;
        c->m0.assign(prior->m0, prior->m0 + d);
        c->psi0.assign(prior->psi0, prior->psi0 + (size_t)d * d);
    } else {
        c->beta.assign(prior->beta, prior->beta + d);
    }
    c->st.init(d, c->kind == DPMM_PRIOR_NIW ? STAT_FULL : STAT_FIRST);
    c->sparse = sparse_path(c);
    // the dense statistics kernels' limit; the compressed-row label kernel scores up to
    // 256 clusters (eight per lane)
    if ((!c->sparse && c->st.nblk > 1024) || (c->sparse && K_max > 256)) {
        delete c;
        return DPMM_EINVAL;
    }
    // multinomial statistics are first moments only (small records): four ranges per SM,
    // so that four CTAs per SM hide the latency of the gathered rows
    c->G2 = (c->kind == DPMM_PRIOR_DIRICHLET ? 4 : 2) * c->num_sms;
    const size_t S = 3 * (size_t)K_max;
    bool ok = true;
    auto A = [&](auto** p, size_t bytes) { ok = ok && dalloc(p, bytes) == cudaSuccess; };
    A(&c->dK, sizeof(int));
    A(&c->diter, 3 * sizeof(uint32_t));  // [sweep index, problem id, point offset]
    A(&c->age, sizeof(int) * K_max);
    A(&c->counters, sizeof(int) * 8);
    A(&c->derr, sizeof(int));
    A(&c->stats, sizeof(double) * 2 * K_max * c->st.E);
    A(&c->shift_new, sizeof(double) * K_max * d);
    A(&c->shift_stats, sizeof(double) * K_max * d);
    A(&c->shift32, sizeof(float) * K_max * d);
    A(&c->p_logw, sizeof(double) * S);
    A(&c->p_mu, sizeof(double) * S * d);
    if (c->kind == DPMM_PRIOR_NIW) A(&c->p_W, sizeof(double) * S * d * d);
    A(&c->p_logdetW, sizeof(double) * S);
    A(&c->p_c, sizeof(double) * S);
    A(&c->p_logtheta, sizeof(double) * S * d);
    A(&c->q_mu, sizeof(float) * S * d);
    if (c->kind == DPMM_PRIOR_NIW) A(&c->q_W, sizeof(float) * S * d * d);
    A(&c->q_c, sizeof(float) * S);
    A(&c->q_b, sizeof(float) * S * d);
    if (c->kind == DPMM_PRIOR_NIW) A(&c->p_b, sizeof(double) * S * d);
    A(&c->q_logtheta, sizeof(float) * S * d);
    A(&c->cweights, sizeof(double) * K_max);
    A(&c->eps, sizeof(double) * S * d);
    A(&c->bart, sizeof(double) * S * d);
    A(&c->lgs, sizeof(double) * (S + 1));
    A(&c->retry, sizeof(int) * S);
    A(&c->tot, sizeof(int) * (K_max + 2));  // starts, then the sort's completion counter
    // range records of the dense statistics kernels (the compressed-row path adds its
    // counts straight into the table)
    c->records_bytes = c->sparse ? 0 : sizeof(double) * (size_t)(c->G2 + K_max) * 2 * c->st.E;
    A(&c->records, c->records_bytes);
    if (c->kind == DPMM_PRIOR_DIRICHLET && !c->sparse) A(&c->mcnt, sizeof(unsigned) * 2 * (size_t)K_max * (d + 1));
    if (c->sparse) {
        const size_t ks = (size_t)(K_max + 31) / 32 * 32;
        A(&c->sp_cc, sizeof(float) * 2 * (size_t)K_max * d);
        A(&c->sp_ltT, sizeof(double) * ks * d);
        A(&c->sp_ct, sizeof(double) * K_max);
    }
    if (c->kind == DPMM_PRIOR_DIRICHLET) {  // FP32 theta draws; the marginals' lgamma tables
        A(&c->sp_part, sizeof(float) * 2 * S * ((d + 2047) / 2048));
        A(&c->sp_lgb, sizeof(double) * d);
        bool uniform = true;
        for (int j = 1; j < d; ++j) uniform = uniform && prior->beta[j] == prior->beta[0];
        if (uniform) A(&c->sp_lgt, sizeof(double) * SP_LGT);
        if (ok) {  // lgamma terms of the Dirichlet-multinomial marginal, from the host's libm
            std::vector<double> lgb(d);
            for (int j = 0; j < d; ++j) lgb[j] = std::lgamma(prior->beta[j]);
            ok = cudaMemcpy(c->sp_lgb, lgb.data(), sizeof(double) * d, cudaMemcpyHostToDevice) == cudaSuccess;
            if (ok && uniform) {
                std::vector<double> t(SP_LGT);
                const double b = prior->beta[0];
                for (int q = 0; q < SP_LGT; ++q) t[q] = std::lgamma(b + q) - std::lgamma(b);
                ok = cudaMemcpy(c->sp_lgt, t.data(), sizeof(double) * SP_LGT, cudaMemcpyHostToDevice) == cudaSuccess;
            }
            // a copy from pageable memory may return before its transfer lands, and the
            // context's stream (set later) need not be ordered after the legacy stream
            ok = ok && cudaDeviceSynchronize() == cudaSuccess;
        }
    }
    A(&c->Ltab, sizeof(double) * (3 * (size_t)K_max + 3 * ((size_t)K_max * (K_max - 1) / 2) + 1 + 6 * (size_t)K_max));
    A(&c->relabel, sizeof(int) * 4 * K_max);
    A(&c->acc, sizeof(int) * ((size_t)K_max + (size_t)K_max * (K_max - 1) / 2 + 1));
    A(&c->center, sizeof(double) * (2 * (size_t)d + (size_t)d * d));
    if (!ok) {
        cudaGetLastError();  // the failed allocation's error is not left for a later call to report
        dpmm_destroy(c);
        return DPMM_ENOMEM;
    }
    cudaMemset(c->derr, 0, sizeof(int));
    cudaMemset(c->diter, 0, 3 * sizeof(uint32_t));
    cudaMemset(c->retry, 0, sizeof(int) * S);
    cudaMemset(c->counters, 0, sizeof(int) * 8);
    cudaMemset(c->p_logw, 0, sizeof(double) * S);
    cudaMemset(c->dK, 0, sizeof(int));
    cudaMemset(c->center, 0, sizeof(double) * (2 * (size_t)d + (size_t)d * d));
    // the memsets above run on the legacy stream; the context's stream may not wait for it
    if (cudaDeviceSynchronize() != cudaSuccess) {
        dpmm_destroy(c);
        return DPMM_ECUDA;
    }
    *out = c;
    return DPMM_OK;
}

void dpmm_destroy(dpmm_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_data(c);
    void* ps[] = {c->dK, c->diter, c->age, c->counters, c->derr, c->stats, c->shift_new, c->shift_stats,
                  c->shift32, c->p_logw, c->p_mu, c->p_W, c->p_logdetW, c->p_c, c->p_logtheta, c->q_mu,
                  c->q_W, c->q_c, c->q_b, c->q_logtheta, c->cweights, c->tot, c->records, c->Ltab,
                  c->relabel, c->acc, c->center, c->tc_img, c->tcs_img, c->tc_flag, c->dbg_scores, c->eps, c->bart, c->lgs, c->retry, c->x3_fimg,
                  c->sp_cc, c->sp_ltT, c->sp_ct, c->sp_lgt, c->sp_lgb, c->sp_part, c->shard_scratch, c->p_b, c->mcnt,
                  c->stage};
    if (c->cstream) cudaStreamSynchronize(c->cstream);
    for (void* p : ps) dfree(p);
    if (c->ev_copied) cudaEventDestroy(c->ev_copied);
    if (c->ev_free) cudaEventDestroy(c->ev_free);
    if (c->cstream) cudaStreamDestroy(c->cstream);
    for (auto& p : c->prof)
        for (auto e : p.ev) cudaEventDestroy(e);
    drop_graph(c);
    delete c;
}

dpmm_status dpmm_set_options(dpmm_ctx* c, dpmm_prec prec, int init_K, int burn_out, void* stream) {
    if (!c) return DPMM_EINVAL;
    drop_graph(c);
    if (prec < DPMM_PREC_FP64_PLAIN || prec > DPMM_PREC_BF16X3) return fail(c, DPMM_EINVAL, "unknown precision");
    if (init_K < 1 || init_K > c->K_max) return fail(c, DPMM_EINVAL, "init_K must be in [1, K_max]");
    if (burn_out < 0) return fail(c, DPMM_EINVAL, "burn_out must be >= 0");
    if (c->X && prec != c->prec) return fail(c, DPMM_ESTATE, "set the precision before dpmm_set_data");
    int old = c->prec;
    c->prec = prec;
    if (((prec == DPMM_PREC_TF32 || prec == DPMM_PREC_BF16) && !tc_supported(c)) ||
        (prec == DPMM_PREC_BF16X3 && !x3_supported(c))) {
        c->prec = old;
        return fail(c, DPMM_EINVAL, "tensor-core precision not available for this prior/dimension");
    }
    c->init_K = init_K;
    c->burn_out = burn_out;
    c->stream = (cudaStream_t)stream;
    return DPMM_OK;
}

dpmm_status dpmm_set_data(dpmm_ctx* c, const void* X, int64_t N, dpmm_dtype dt, int on_device) {
    if (!c) return DPMM_EINVAL;
    c->staged = false;
    drop_graph(c);
    if (!X || N < 1 || N > 0x7FFFFFFFLL) return fail(c, DPMM_EINVAL, "need 1 <= N < 2^31 and a non-NULL X");
    if (dt < DPMM_F64 || dt > DPMM_I32) return fail(c, DPMM_EINVAL, "unknown dtype");
    if (c->kind == DPMM_PRIOR_NIW && dt == DPMM_I32) return fail(c, DPMM_EINVAL, "Gaussian data must be floating point");
    CK(c, cudaStreamSynchronize(c->stream));
    free_data(c);
    c->N = N;
    rearm_kernel_choice(c);
    c->in_dt = dt;
    const int d = c->d;
    if (c->prec == DPMM_PREC_FP64_PLAIN) {
        c->xdt = 0;
        c->xs = d;
    } else if (c->prec == DPMM_PREC_BF16) {
        c->xdt = 2;
        c->xs = (d + 7) / 8 * 8;
        if (c->xs < 64) c->xs = 64;  // one 128-byte TMA box per row
    } else {
        c->xdt = 1;
        c->xs = (d + 3) / 4 * 4;
        if (c->prec == DPMM_PREC_TF32 && c->xs < 32) c->xs = 32;  // one 128-byte TMA box per row
    }
    if (c->sparse) return set_data_sparse(c, X, N, dt, on_device);
    const size_t esz = c->xdt == 0 ? 8 : (c->xdt == 1 ? 4 : 2);
    c->T_tiles = (int)((N + SORT_TILE - 1) / SORT_TILE);
    // ranges of the statistics step: about one per 512 points, at most 2 x SMs (the CUDA-core
    // kernels run two CTAs per SM) or 1 x SMs for the tensor-core kernel (one CTA per SM: one
    // long range per CTA fills its pipeline once)
    c->Gr = (int)std::min<int64_t>(substats_tc_supported(c) ? c->num_sms : c->G2, std::max<int64_t>(1, (N + 511) / 512));
    bool ok = true;
    auto A = [&](auto** p, size_t bytes) { ok = ok && dalloc(p, bytes) == cudaSuccess; };
    A(&c->X, (size_t)N * c->xs * esz);
    A(&c->z, sizeof(int32_t) * N);
    A(&c->zbar, N);
    A(&c->idx, sizeof(int) * N);
    A(&c->hist, sizeof(int) * (size_t)c->K_max * c->T_tiles);
    if (const size_t cb = tc_carry_bytes(c)) A(&c->tc_carry, cb);
    if (!ok) {
        cudaGetLastError();  // the failed allocation's error is not left for a later call to report
        free_data(c);
        return fail(c, DPMM_ENOMEM, "device allocation for the data failed");
    }
    CK(c, cudaDeviceSynchronize());  // the zeroing memsets ran on the legacy stream
    // centring (Gaussian, reduced precision): computed on the device from the input
    std::vector<double> cen((size_t)2 * d + (size_t)d * d, 0.0);
    CK(c, cudaMemcpyAsync(c->center, cen.data(), sizeof(double) * cen.size(), cudaMemcpyHostToDevice, c->stream));
    const bool center = c->kind == DPMM_PRIOR_NIW && c->prec != DPMM_PREC_FP64_PLAIN;
    dpmm_status s = upload(c, X, dt, on_device, center);
    if (s != DPMM_OK) return s;
    c->h_center.assign(d, 0.0);
    CK(c, cudaMemcpyAsync(c->h_center.data(), c->center, sizeof(double) * d, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    // prior in storage coordinates: [center | m0 - center (or beta) | psi0]
    for (int j = 0; j < d; ++j) cen[j] = c->h_center[j];
    if (c->kind == DPMM_PRIOR_NIW) {
        for (int j = 0; j < d; ++j) cen[d + j] = c->m0[j] - c->h_center[j];
        for (size_t q = 0; q < (size_t)d * d; ++q) cen[2 * d + q] = c->psi0[q];
    } else {
        for (int j = 0; j < d; ++j) cen[d + j] = c->beta[j];
    }
    CK(c, cudaMemcpyAsync(c->center, cen.data(), sizeof(double) * cen.size(), cudaMemcpyHostToDevice, c->stream));
    uint32_t zero = 0;
    CK(c, cudaMemcpyAsync(c->diter, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->initialized = false;
    c->h_iter = 0;
    return DPMM_OK;
}

dpmm_status dpmm_update_data(dpmm_ctx* c, const void* X, dpmm_dtype dt, int on_device) {
    if (!c) return DPMM_EINVAL;
    c->staged = false;  // values staged before are superseded
    if (!c->X) return fail(c, DPMM_ESTATE, "dpmm_set_data first");
    if (!X || dt != c->in_dt) return fail(c, DPMM_EINVAL, "same dtype as dpmm_set_data required");
    if (c->sparse) {  // new compressed rows (their length changes): the captured sweep refers to the old ones
        drop_graph(c);
        return sparse_upload(c, X, dt, on_device);
    }
    return upload(c, X, dt, on_device, false);
}

// ---- staged input: the copy of the next sweep's values overlaps the current sweep
dpmm_status dpmm_stage_data(dpmm_ctx* c, const void* X, dpmm_dtype dt) {
    if (!c) return DPMM_EINVAL;
    if (!c->X) return fail(c, DPMM_ESTATE, "dpmm_set_data first");
    if (c->sparse) return fail(c, DPMM_EINVAL, "compressed rows take new data through dpmm_set_data_csr");
    if (!X || dt != c->in_dt) return fail(c, DPMM_EINVAL, "same dtype as dpmm_set_data required");
    const size_t bytes = (size_t)c->N * c->d * dt_size(dt);
    if (!c->cstream) CK(c, cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
    if (!c->ev_copied) CK(c, cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming));
    if (!c->ev_free) {
        CK(c, cudaEventCreateWithFlags(&c->ev_free, cudaEventDisableTiming));
        CK(c, cudaEventRecord(c->ev_free, c->stream));
    }
    if (c->stage_bytes < bytes) {
        CK(c, cudaStreamSynchronize(c->cstream));
        CK(c, cudaStreamSynchronize(c->stream));
        dfree(c->stage);
        c->stage = nullptr;
        c->stage_bytes = 0;
        if (cudaMalloc(&c->stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->stage = nullptr;
            return fail(c, DPMM_ENOMEM, "device allocation for the staging buffer failed");
        }
        c->stage_bytes = bytes;
    }
    // the values staged before must have been taken by the sweep that converts them
    CK(c, cudaStreamWaitEvent(c->cstream, c->ev_free, 0));
    CK(c, cudaMemcpyAsync(c->stage, X, bytes, cudaMemcpyHostToDevice, c->cstream));
    CK(c, cudaEventRecord(c->ev_copied, c->cstream));
    c->staged = true;
    return DPMM_OK;
}

// At the start of a sweep: staged values replace the data (as dpmm_update_data would).
static dpmm_status take_staged(dpmm_ctx* c) {
    if (!c->staged) return DPMM_OK;
    c->staged = false;
    CK(c, cudaStreamWaitEvent(c->stream, c->ev_copied, 0));
    const dpmm_status s = upload(c, c->stage, c->in_dt, 1, false);
    if (s != DPMM_OK) return s;
    CK(c, cudaEventRecord(c->ev_free, c->stream));
    return DPMM_OK;
}

dpmm_status dpmm_set_data_csr(dpmm_ctx* c, const int64_t* indptr, const int32_t* indices, const int32_t* counts,
                              int64_t N) {
    if (!c) return DPMM_EINVAL;
    if (!c->sparse) return fail(c, DPMM_EINVAL, "compressed rows are taken for multinomial data of more than 256 categories");
    drop_graph(c);
    if (!indptr || N < 1 || N > 0x7FFFFFFFLL || indptr[0] != 0) return fail(c, DPMM_EINVAL, "need 1 <= N < 2^31 and indptr[0] = 0");
    const int64_t nnz = indptr[N];
    if (nnz < 0 || (nnz > 0 && (!indices || !counts))) return fail(c, DPMM_EINVAL, "bad indptr or NULL arrays");
    for (int64_t i = 0; i < N; ++i) {
        if (indptr[i + 1] < indptr[i]) return fail(c, DPMM_EINVAL, "indptr must be non-decreasing");
        for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
            if (indices[p] < 0 || indices[p] >= c->d || (p > indptr[i] && indices[p] <= indices[p - 1]))
                return fail(c, DPMM_EINVAL, "indices must be in [0, d) and increasing within each row");
            if (counts[p] < 0 || counts[p] >= (1 << 24)) return fail(c, DPMM_EINVAL, "counts must be in [0, 2^24)");
        }
    }
    CK(c, cudaStreamSynchronize(c->stream));
    dpmm_status s = sparse_alloc(c, N);
    if (s != DPMM_OK) return s;
    c->in_dt = DPMM_I32;
    c->nnz = nnz;
    bool ok = dalloc(&c->csr_idx, sizeof(int) * std::max<int64_t>(nnz, 1)) == cudaSuccess &&
              dalloc(&c->csr_val, sizeof(int) * std::max<int64_t>(nnz, 1)) == cudaSuccess;
    if (!ok) {
        free_data(c);
        return fail(c, DPMM_ENOMEM, "device allocation for the data failed");
    }
    CK(c, cudaDeviceSynchronize());
    CK(c, cudaMemcpyAsync(c->csr_ptr, indptr, sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, c->stream));
    if (nnz > 0) {
        CK(c, cudaMemcpyAsync(c->csr_idx, indices, sizeof(int) * nnz, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->csr_val, counts, sizeof(int) * nnz, cudaMemcpyHostToDevice, c->stream));
    }
    return sparse_finish(c);
}

// Initial labels (K = init_K, fair sub-label coins) and the statistics of this context's
// points.
static dpmm_status init_phase_a(dpmm_ctx* c, uint64_t seed) {
    const int K = c->init_K;
    CK(c, cudaMemcpyAsync(c->dK, &K, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->age, 0, sizeof(int) * c->K_max, c->stream));
    CK(c, cudaMemsetAsync(c->shift_new, 0, sizeof(double) * c->K_max * c->d, c->stream));
    CK(c, cudaMemsetAsync(c->shift32, 0, sizeof(float) * c->K_max * c->d, c->stream));
    CK(c, launch_init_labels(c, seed));
    if (c->sparse) {
        CK(c, launch_sparse(c, seed, 2, nullptr));
    } else {
        CK(c, launch_sort(c));
        CK(c, launch_substats(c, seed, 0));
        CK(c, launch_combine(c));
    }
    return DPMM_OK;
}

// clusters left empty by the initial draw are removed (no ages, no sweep index change)
static dpmm_status init_phase_b(dpmm_ctx* c, uint64_t seed) {
    CK(c, launch_splitmerge(c, seed, 2, 0));
    CK(c, launch_relabel(c, seed));
    c->initialized = true;
    return DPMM_OK;
}

static dpmm_status init_chain(dpmm_ctx* c, uint64_t seed) {
    dpmm_status s = init_phase_a(c, seed);
    return s != DPMM_OK ? s : init_phase_b(c, seed);
}

// The kernels of one sweep, in order, on the context's stream, in three phases: (a) the
// parameters from the statistics, the labels, sub-labels and the statistics of this
// context's points; (b) splits, merges, relabelling and the recount of the statistics
// when anything changed; (c) the sweep index.  A point-sharded sweep exchanges the
// statistics after (a) and after (b).
// ---- label-step kernel selection (Sec. 4.2: two kernels, chosen at run time)
static bool has_tc_labels(const dpmm_ctx* c) { return !c->sparse && (tc_supported(c) || x3_supported(c)); }

// the label step on the tensor cores (which = 0) or the CUDA cores (which = 1)
static cudaError_t label_step(dpmm_ctx* c, uint64_t seed, int which) {
    if (which == 1 || !has_tc_labels(c)) return launch_labels_simt(c, seed);
    return c->prec == DPMM_PREC_BF16X3 ? launch_labels_x3(c, seed) : launch_labels_tc(c, seed);
}

struct KernelKey {
    int device, kind, prec, d, logn, K_max;
    bool operator<(const KernelKey& o) const {
        return std::tie(device, kind, prec, d, logn, K_max) < std::tie(o.device, o.kind, o.prec, o.d, o.logn, o.K_max);
    }
};
struct KernelPick {
    int use;
    float ms[2];
};
static std::mutex g_kcache_mu;
static std::map<KernelKey, KernelPick> g_kcache;

static KernelKey kernel_key(const dpmm_ctx* c) {
    int logn = 0;
    while ((int64_t(2) << logn) <= c->N) ++logn;
    return KernelKey{c->device, c->kind, c->prec, c->d, logn, c->K_max};
}

// Runs on an eager sweep only (it synchronises): both label kernels three times each on
// this sweep's parameters, the first run of each a warm-up; keeps the faster.  The label
// step is a deterministic function of the parameters and the sweep counter, and the
// chosen kernel runs once more right after, so the chain is that of the chosen kernel.
static cudaError_t tune_labels(dpmm_ctx* c, uint64_t seed) {
    c->ktune = false;
    if (!has_tc_labels(c)) return cudaSuccess;  // one kernel: nothing to choose
    const KernelKey key = kernel_key(c);
    {
        std::lock_guard<std::mutex> lk(g_kcache_mu);
        auto it = g_kcache.find(key);
        if (it != g_kcache.end()) {
            c->kuse = it->second.use;
            c->kms[0] = it->second.ms[0];
            c->kms[1] = it->second.ms[1];
            return cudaSuccess;
        }
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    float best[2] = {1e30f, 1e30f};
    for (int v = 0; v < 2 && e == cudaSuccess; ++v)
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            e = cudaEventRecord(ev[0], c->stream);
            if (e == cudaSuccess) e = label_step(c, seed, v);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e == cudaSuccess && r > 0) best[v] = std::min(best[v], ms);
        }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return e;
    c->kms[0] = best[0];
    c->kms[1] = best[1];
    c->kuse = best[1] < best[0] ? 1 : 0;
    std::lock_guard<std::mutex> lk(g_kcache_mu);
    g_kcache[key] = KernelPick{c->kuse, {best[0], best[1]}};
    return cudaSuccess;
}

static cudaError_t sweep_phase_a(dpmm_ctx* c, uint64_t seed) {
    cudaError_t e = cudaSuccess;
    if (c->step_mask & 1u) {
        if ((e = launch_weights(c, seed)) != cudaSuccess) return e;
        if ((e = launch_params(c, seed)) != cudaSuccess) return e;
        if ((e = launch_derive(c)) != cudaSuccess) return e;
    }
    if ((c->step_mask & 2u) && c->sparse) {
        if ((e = launch_sparse(c, seed, 0, nullptr)) != cudaSuccess) return e;
    } else if (c->step_mask & 2u) {
        if (c->ktune) {  // never pending during graph capture: set only by calls that drop the graph
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if ((e = cudaStreamIsCapturing(c->stream, &cs)) != cudaSuccess) return e;
            if (cs == cudaStreamCaptureStatusNone && (e = tune_labels(c, seed)) != cudaSuccess) return e;
        }
        if ((e = label_step(c, seed, c->kuse)) != cudaSuccess) return e;
        if ((e = launch_sort(c)) != cudaSuccess) return e;
        if ((e = launch_substats(c, seed, 1)) != cudaSuccess) return e;
        if ((e = launch_combine(c)) != cudaSuccess) return e;
    }
    return e;
}

static cudaError_t sweep_phase_b(dpmm_ctx* c, uint64_t seed) {
    cudaError_t e = launch_splitmerge(c, seed, (c->step_mask & 2u) ? 1 : 0, (c->step_mask & 4u) ? 1 : 0);
    if (e != cudaSuccess) return e;
    return launch_relabel(c, seed);
}

static cudaError_t enqueue_sweep(dpmm_ctx* c, uint64_t seed) {
    cudaError_t e = sweep_phase_a(c, seed);
    if (e == cudaSuccess) e = sweep_phase_b(c, seed);
    if (e == cudaSuccess) e = launch_advance(c);
    return e;
}

dpmm_status dpmm_sweep(dpmm_ctx* c, int iters, uint64_t seed) {
    if (!c) return DPMM_EINVAL;
    if (!c->X) return fail(c, DPMM_ESTATE, "dpmm_set_data first");
    if (iters < 0) return fail(c, DPMM_EINVAL, "iters must be >= 0");
    {
        const dpmm_status s = take_staged(c);
        if (s != DPMM_OK) return s;
    }
    if (!c->initialized) {
        dpmm_status s = init_chain(c, seed);
        if (s != DPMM_OK) return s;
    }
    // the first sweep runs eagerly (it allocates what the kernels need); later ones
    // replay a graph of the same launches, captured once per (seed, mask)
    const bool graphs = c->use_graph && !c->profiling && c->stream != nullptr;
    for (int it = 0; it < iters; ++it) {
        if (graphs && c->graph && c->graph_seed == seed && c->graph_mask == c->step_mask) {
            CK(c, cudaGraphLaunch(c->graph, c->stream));
            c->nlaunch += c->graph_kernels;
            continue;
        }
        CK(c, enqueue_sweep(c, seed));
        if (graphs) {  // every buffer exists after the eager sweep: capture allocates nothing
            drop_graph(c);
            cudaGraph_t g = nullptr;
            CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            const int64_t before = c->nlaunch;
            cudaError_t e = enqueue_sweep(c, seed);
            c->graph_kernels = c->nlaunch - before;
            c->nlaunch = before;  // captured, not launched
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
            if (e == cudaSuccess && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&c->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                c->graph = nullptr;
                c->use_graph = false;  // run eagerly from now on
                cudaGetLastError();
                CK(c, e);
            } else {
                c->graph_seed = seed;
                c->graph_mask = c->step_mask;
                // the eager sweep above was sweep `it`; the captured one has not run yet
            }
        }
    }
    c->seed = seed;
    return DPMM_OK;
}

// ---- checkpoint: [header | z (N int32) | zbar (N bytes) | ages (K int32) | counters
// (8 int32) | statistics (2K x E doubles) | shift (K x d doubles) | weights (K doubles)],
// every array padded to a multiple of 8 bytes
struct CkptHeader {
    uint64_t magic;
    uint32_t version;
    int32_t kind, d, E;
    int64_t N;
    int32_t K;
    uint32_t iter, problem;
    int32_t pad;
};
static const uint64_t CKPT_MAGIC = 0x54504b434d4d5044ull;  // "DPMMCKPT"

static size_t ckpt_bytes(const dpmm_ctx* c, int K) {
    auto up8 = [](size_t b) { return (b + 7) / 8 * 8; };
    return sizeof(CkptHeader) + up8((size_t)c->N * 4) + up8((size_t)c->N) + up8((size_t)K * 4) + 8 * 4 +
           8 * ((size_t)2 * K * c->st.E + (size_t)K * c->d + K);
}

static dpmm_status ckpt_state(dpmm_ctx* c) {
    if (!c) return DPMM_EINVAL;
    if (!c->X || !c->initialized) return fail(c, DPMM_ESTATE, "no chain to checkpoint");
    return DPMM_OK;
}

dpmm_status dpmm_checkpoint_size(dpmm_ctx* c, size_t* bytes) {
    dpmm_status st = ckpt_state(c);
    if (st != DPMM_OK) return st;
    if (!bytes) return fail(c, DPMM_EINVAL, "null output");
    int K = 0;
    CK(c, cudaMemcpyAsync(&K, c->dK, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *bytes = ckpt_bytes(c, K);
    return DPMM_OK;
}

dpmm_status dpmm_save_checkpoint(dpmm_ctx* c, void* buf, size_t bytes) {
    dpmm_status st = ckpt_state(c);
    if (st != DPMM_OK) return st;
    CkptHeader h{};
    uint32_t it[2] = {0, 0};
    CK(c, cudaMemcpyAsync(&h.K, c->dK, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(it, c->diter, sizeof(it), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (!buf || bytes < ckpt_bytes(c, h.K)) return fail(c, DPMM_EINVAL, "checkpoint buffer too small");
    h.magic = CKPT_MAGIC;
    h.version = 1;
    h.kind = c->kind;
    h.d = c->d;
    h.E = c->st.E;
    h.N = c->N;
    h.iter = it[0];
    h.problem = it[1];
    unsigned char* q = (unsigned char*)buf;
    memcpy(q, &h, sizeof(h));
    q += sizeof(h);
    const int K = h.K;
    auto D2H = [&](void* dst, const void* src, size_t n, size_t padded) {
        if (n) CK(c, cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, c->stream));
        if (padded > n) memset((unsigned char*)dst + n, 0, padded - n);
        q += padded;
        return DPMM_OK;
    };
    auto up8 = [](size_t b) { return (b + 7) / 8 * 8; };
    const void* src[7] = {c->z, c->zbar, c->age, c->counters, c->stats, c->shift_stats, c->cweights};
    const size_t len[7] = {(size_t)c->N * 4, (size_t)c->N, (size_t)K * 4, 8 * 4, (size_t)2 * K * c->st.E * 8,
                           (size_t)K * c->d * 8, (size_t)K * 8};
    for (int a = 0; a < 7; ++a)
        if ((st = D2H(q, src[a], len[a], up8(len[a]))) != DPMM_OK) return st;
    CK(c, cudaStreamSynchronize(c->stream));
    return check_derr(c);
}

dpmm_status dpmm_load_checkpoint(dpmm_ctx* c, const void* buf, size_t bytes) {
    if (!c) return DPMM_EINVAL;
    if (!c->X) return fail(c, DPMM_ESTATE, "dpmm_set_data first");
    CkptHeader h{};
    if (!buf || bytes < sizeof(h)) return fail(c, DPMM_EINVAL, "checkpoint too short");
    memcpy(&h, buf, sizeof(h));
    if (h.magic != CKPT_MAGIC || h.version != 1) return fail(c, DPMM_EINVAL, "not a checkpoint of this format");
    if (h.kind != c->kind || h.d != c->d || h.E != c->st.E || h.N != c->N)
        return fail(c, DPMM_EINVAL, "checkpoint of another prior, dimension or data size");
    if (h.K < 1 || h.K > c->K_max || bytes < ckpt_bytes(c, h.K))
        return fail(c, DPMM_EINVAL, "checkpoint size or K out of range");
    CK(c, cudaStreamSynchronize(c->stream));
    drop_graph(c);
    const unsigned char* q = (const unsigned char*)buf + sizeof(h);
    const int K = h.K;
    auto up8 = [](size_t b) { return (b + 7) / 8 * 8; };
    // every copy is ordered on the context's stream (a legacy-stream copy is not ordered
    // with a non-blocking stream); the stream is synchronised before returning because the
    // caller's buffer only has to stay valid for the duration of this call
    auto H2D = [&](void* dst, size_t n, size_t padded) {
        if (n) CK(c, cudaMemcpyAsync(dst, q, n, cudaMemcpyHostToDevice, c->stream));
        q += padded;
        return DPMM_OK;
    };
    // labels out of range would be used as addresses by the sort: check them on the host
    const int32_t* zh = (const int32_t*)q;
    for (int64_t i = 0; i < c->N; ++i)
        if (zh[i] < 0 || zh[i] >= K) return fail(c, DPMM_EINVAL, "checkpoint label out of range");
    const uint32_t it[2] = {h.iter, h.problem};
    CK(c, cudaMemcpyAsync(c->dK, &h.K, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->diter, it, sizeof(it), cudaMemcpyHostToDevice, c->stream));
    void* dst[7] = {c->z, c->zbar, c->age, c->counters, c->stats, c->shift_stats, c->cweights};
    const size_t len[7] = {(size_t)c->N * 4, (size_t)c->N, (size_t)K * 4, 8 * 4, (size_t)2 * K * c->st.E * 8,
                           (size_t)K * c->d * 8, (size_t)K * 8};
    for (int a = 0; a < 7; ++a) {
        const dpmm_status st = H2D(dst[a], len[a], up8(len[a]));
        if (st != DPMM_OK) {
            cudaStreamSynchronize(c->stream);
            return st;
        }
    }
    // the compressed-row path's compact counts are not in the checkpoint: recount them from
    // the labels (integer sums: the same table)
    if (c->sparse) CK(c, launch_sparse(c, 0, 2, nullptr));
    CK(c, cudaStreamSynchronize(c->stream));
    c->initialized = true;
    c->h_iter = h.iter;
    return DPMM_OK;
}

dpmm_status dpmm_check_wait_timeout(dpmm_ctx* c) {
    if (!c) return DPMM_EINVAL;
    CK(c, launch_wait_selftest(c));
    return check_derr(c);
}

dpmm_status dpmm_set_problem(dpmm_ctx* c, uint32_t problem) {
    if (!c) return DPMM_EINVAL;
    CK(c, cudaMemcpyAsync(c->diter + 1, &problem, sizeof(problem), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return DPMM_OK;
}

dpmm_status dpmm_sweep_batch(dpmm_ctx* const* ctxs, int n, int iters, uint64_t seed) {
    if (!ctxs || n < 0 || iters < 0) return DPMM_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return DPMM_EINVAL;
    for (int it = 0; it < iters; ++it)
        for (int i = 0; i < n; ++i) {
            const dpmm_status s = dpmm_sweep(ctxs[i], 1, seed);
            if (s != DPMM_OK) return s;
        }
    return DPMM_OK;
}

dpmm_status dpmm_set_shard(dpmm_ctx* c, int64_t point_offset) {
    if (!c) return DPMM_EINVAL;
    if (point_offset < 0 || point_offset + c->N > 0x7FFFFFFFLL)
        return fail(c, DPMM_EINVAL, "the shard must lie within points [0, 2^31)");
    const uint32_t off = (uint32_t)point_offset;
    CK(c, cudaMemcpyAsync(c->diter + 2, &off, sizeof(off), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->poff = point_offset;
    return DPMM_OK;
}

// every shard must describe the same chain: same model, options and state
static dpmm_status shard_check(dpmm_ctx* const* sh, int G) {
    dpmm_ctx* a = sh[0];
    int64_t next = 0;
    for (int s = 0; s < G; ++s) {
        dpmm_ctx* b = sh[s];
        if (!b->X) return fail(b, DPMM_ESTATE, "every shard needs its data");
        if (b->kind != a->kind || b->d != a->d || b->K_max != a->K_max || b->prec != a->prec || b->alpha != a->alpha ||
            b->kappa0 != a->kappa0 || b->nu0 != a->nu0 || b->m0 != a->m0 || b->psi0 != a->psi0 || b->beta != a->beta ||
            b->init_K != a->init_K || b->burn_out != a->burn_out || b->step_mask != a->step_mask ||
            b->device != a->device || b->initialized != a->initialized)
            return fail(b, DPMM_EINVAL, "shards of one chain need the same prior, options, device and state");
        if (b->poff != next) return fail(b, DPMM_EINVAL, "shard s must start where shard s - 1 ends (dpmm_set_shard)");
        next += b->N;
        CK(b, cudaStreamSynchronize(b->stream));
    }
    // the shards' data were centred separately (reduced-precision Gaussian paths centre by
    // the data's mean); one chain needs one coordinate system
    for (int s = 1; s < G; ++s)
        if (sh[s]->h_center != a->h_center)
            return fail(sh[s], DPMM_EINVAL, "sharded Gaussian chains need the FP64-plain path (uncentred data)");
    return DPMM_OK;
}

static dpmm_status sync_all(dpmm_ctx* const* sh, int G) {
    for (int s = 0; s < G; ++s) CK(sh[s], cudaStreamSynchronize(sh[s]->stream));
    return DPMM_OK;
}

dpmm_status dpmm_sweep_sharded(dpmm_ctx* const* sh, int G, int iters, uint64_t seed) {
    if (!sh || G < 1 || G > 16 || iters < 0) return DPMM_EINVAL;
    for (int s = 0; s < G; ++s)
        if (!sh[s]) return DPMM_EINVAL;
    dpmm_status st = shard_check(sh, G);
    if (st != DPMM_OK) return st;
    for (int s = 0; s < G; ++s)
        if ((st = take_staged(sh[s])) != DPMM_OK) return st;
    dpmm_ctx* c0 = sh[0];
    auto phase = [&](auto&& f) -> dpmm_status {
        for (int s = 0; s < G; ++s) {
            dpmm_status r = f(sh[s]);
            if (r != DPMM_OK) return r;
        }
        return sync_all(sh, G);
    };
    auto exchange = [&](const int* gate) -> dpmm_status {
        CK(c0, shard_exchange(sh, G, gate));
        CK(c0, cudaStreamSynchronize(c0->stream));
        return DPMM_OK;
    };
    if (!c0->initialized) {
        if ((st = phase([&](dpmm_ctx* c) { return init_phase_a(c, seed); })) != DPMM_OK) return st;
        if ((st = exchange(nullptr)) != DPMM_OK) return st;
        if ((st = phase([&](dpmm_ctx* c) { return init_phase_b(c, seed); })) != DPMM_OK) return st;
        if ((st = exchange(c0->counters + 4)) != DPMM_OK) return st;
    }
    for (int it = 0; it < iters; ++it) {
        st = phase([&](dpmm_ctx* c) {
            CK(c, sweep_phase_a(c, seed));
            return DPMM_OK;
        });
        if (st != DPMM_OK) return st;
        if ((st = exchange(nullptr)) != DPMM_OK) return st;
        st = phase([&](dpmm_ctx* c) {
            CK(c, sweep_phase_b(c, seed));
            return DPMM_OK;
        });
        if (st != DPMM_OK) return st;
        if ((st = exchange(c0->counters + 4)) != DPMM_OK) return st;  // only when the shards recounted
        st = phase([&](dpmm_ctx* c) {
            CK(c, launch_advance(c));
            return DPMM_OK;
        });
        if (st != DPMM_OK) return st;
    }
    for (int s = 0; s < G; ++s) sh[s]->seed = seed;
    return DPMM_OK;
}

dpmm_status dpmm_get_info(dpmm_ctx* c, int* K, uint32_t* iter) {
    if (!c) return DPMM_EINVAL;
    int k = 0;
    uint32_t t = 0;
    CK(c, cudaMemcpyAsync(&k, c->dK, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(&t, c->diter, sizeof(t), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (K) *K = k;
    if (iter) *iter = t;
    return check_derr(c);
}

dpmm_status dpmm_get_labels(dpmm_ctx* c, int32_t* z, uint8_t* zbar) {
    if (!c) return DPMM_EINVAL;
    if (!c->X) return fail(c, DPMM_ESTATE, "no data");
    if (z) CK(c, cudaMemcpyAsync(z, c->z, sizeof(int32_t) * c->N, cudaMemcpyDeviceToHost, c->stream));
    if (zbar) CK(c, cudaMemcpyAsync(zbar, c->zbar, c->N, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return check_derr(c);
}

dpmm_status dpmm_get_counters(dpmm_ctx* c, int out[4]) {
    if (!c || !out) return DPMM_EINVAL;
    CK(c, cudaMemcpyAsync(out, c->counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return check_derr(c);
}

dpmm_status dpmm_get_stats(dpmm_ctx* c, int* Kout, int64_t* n, double* sx, double* sxx, double* weights) {
    if (!c) return DPMM_EINVAL;
    if (!c->X) return fail(c, DPMM_ESTATE, "no data");
    const int d = c->d;
    const StatLayout& L = c->st;
    int K = 0;
    std::vector<double> S((size_t)2 * c->K_max * L.E), sh((size_t)c->K_max * d), w(c->K_max);
    CK(c, cudaMemcpyAsync(&K, c->dK, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(S.data(), c->stats, sizeof(double) * S.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(sh.data(), c->shift_stats, sizeof(double) * sh.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(w.data(), c->cweights, sizeof(double) * w.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (Kout) *Kout = K;
    auto M = [&](int k, int h, int j, int l) { return S[(size_t)(2 * k + h) * L.E + L.ent(j, l)]; };
    std::vector<double> a(d), s1(d), s2((size_t)d * d);
    for (int k = 0; k < K; ++k) {
        for (int j = 0; j < d; ++j) a[j] = sh[(size_t)k * d + j] + c->h_center[j];
        for (int slot = 0; slot < 3; ++slot) {
            double nn = 0.0;
            std::fill(s1.begin(), s1.end(), 0.0);
            std::fill(s2.begin(), s2.end(), 0.0);
            for (int h = 0; h < 2; ++h) {
                if (slot != 0 && h != slot - 1) continue;
                nn += M(k, h, d, d);
                for (int j = 0; j < d; ++j) s1[j] += M(k, h, j, d);
                if (c->kind == DPMM_PRIOR_NIW)
                    for (int j = 0; j < d; ++j)
                        for (int l = j; l < d; ++l) s2[(size_t)j * d + l] += M(k, h, j, l);
            }
            const int s = 3 * k + slot;
            if (n) n[s] = (int64_t)llround(nn);
            // shifted sums back to original coordinates: x = y + a
            if (sx)
                for (int j = 0; j < d; ++j) sx[(size_t)s * d + j] = s1[j] + nn * a[j];
            if (sxx && c->kind == DPMM_PRIOR_NIW)
                for (int j = 0; j < d; ++j)
                    for (int l = 0; l < d; ++l) {
                        double y = j <= l ? s2[(size_t)j * d + l] : s2[(size_t)l * d + j];
                        sxx[((size_t)s * d + j) * d + l] = y + a[j] * s1[l] + s1[j] * a[l] + nn * a[j] * a[l];
                    }
        }
    }
    if (weights)
        for (int k = 0; k < K; ++k) weights[k] = w[k];
    return check_derr(c);
}

dpmm_status dpmm_set_state(dpmm_ctx* c, int K, const int32_t* z, const uint8_t* zbar) {
    if (!c) return DPMM_EINVAL;
    if (!c->X) return fail(c, DPMM_ESTATE, "dpmm_set_data first");
    if (K < 1 || K > c->K_max || !z || !zbar) return fail(c, DPMM_EINVAL, "bad state");
    for (int64_t i = 0; i < c->N; ++i)
        if (z[i] < 0 || z[i] >= K || zbar[i] > 1) return fail(c, DPMM_EINVAL, "label out of range");
    CK(c, cudaMemcpyAsync(c->z, z, sizeof(int32_t) * c->N, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->zbar, zbar, c->N, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->dK, &K, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->age, 0, sizeof(int) * c->K_max, c->stream));
    CK(c, cudaMemsetAsync(c->shift_new, 0, sizeof(double) * c->K_max * c->d, c->stream));
    CK(c, cudaMemsetAsync(c->shift32, 0, sizeof(float) * c->K_max * c->d, c->stream));
    if (c->sparse) {
        CK(c, launch_sparse(c, 0, 2, nullptr));
    } else {
        CK(c, launch_sort(c));
        CK(c, launch_substats(c, 0, 0));
        CK(c, launch_combine(c));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    c->initialized = true;
    return check_derr(c);
}

dpmm_status dpmm_set_kernel(dpmm_ctx* c, int choice) {
    if (!c) return DPMM_EINVAL;
    if (choice < DPMM_KERNEL_TENSOR || choice > DPMM_KERNEL_AUTO)
        return fail(c, DPMM_EINVAL, "choice: DPMM_KERNEL_TENSOR, DPMM_KERNEL_CUDA_CORE or DPMM_KERNEL_AUTO");
    drop_graph(c);
    c->kchoice = choice;
    c->kuse = choice == DPMM_KERNEL_CUDA_CORE ? 1 : 0;
    c->ktune = choice == DPMM_KERNEL_AUTO;
    c->kms[0] = c->kms[1] = -1.f;
    return DPMM_OK;
}

dpmm_status dpmm_get_kernel(dpmm_ctx* c, int* in_use, float* ms_tensor, float* ms_cuda_core) {
    if (!c) return DPMM_EINVAL;
    const bool tc = has_tc_labels(c);
    if (in_use) *in_use = (tc && c->kuse == 0) ? DPMM_KERNEL_TENSOR : DPMM_KERNEL_CUDA_CORE;
    if (ms_tensor) *ms_tensor = c->kms[0];
    if (ms_cuda_core) *ms_cuda_core = c->kms[1];
    return DPMM_OK;
}

dpmm_status dpmm_set_step_mask(dpmm_ctx* c, unsigned mask) {
    if (!c) return DPMM_EINVAL;
    drop_graph(c);
    if (mask > 7) return fail(c, DPMM_EINVAL, "mask has 3 bits");
    c->step_mask = mask;
    return DPMM_OK;
}

dpmm_status dpmm_set_iter(dpmm_ctx* c, uint32_t iter) {
    if (!c) return DPMM_EINVAL;
    CK(c, cudaMemcpyAsync(c->diter, &iter, sizeof(iter), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return DPMM_OK;
}

dpmm_status dpmm_set_params(dpmm_ctx* c, int K, const double* logw, const double* mu, const double* W,
                            const double* logdetW, const double* logtheta) {
    if (!c) return DPMM_EINVAL;
    if (!c->X) return fail(c, DPMM_ESTATE, "dpmm_set_data first");
    if (K < 1 || K > c->K_max || !logw) return fail(c, DPMM_EINVAL, "bad K or logw");
    const int d = c->d;
    const size_t S = 3 * (size_t)K;
    std::vector<double> cc(S);
    if (c->kind == DPMM_PRIOR_NIW) {
        if (!mu || !W || !logdetW) return fail(c, DPMM_EINVAL, "Gaussian parameters need mu, W, logdetW");
        std::vector<double> ms(S * d);
        for (size_t s = 0; s < S; ++s) {
            for (int j = 0; j < d; ++j) ms[s * d + j] = mu[s * d + j] - c->h_center[j];
            cc[s] = logw[s] + logdetW[s] - 0.5 * d * log(2.0 * M_PI);
        }
        CK(c, cudaMemcpyAsync(c->p_mu, ms.data(), sizeof(double) * S * d, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->p_W, W, sizeof(double) * S * d * d, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->p_logdetW, logdetW, sizeof(double) * S, cudaMemcpyHostToDevice, c->stream));
    } else {
        if (!logtheta) return fail(c, DPMM_EINVAL, "multinomial parameters need logtheta");
        for (size_t s = 0; s < S; ++s) cc[s] = logw[s];
        CK(c, cudaMemcpyAsync(c->p_logtheta, logtheta, sizeof(double) * S * d, cudaMemcpyHostToDevice, c->stream));
    }
    CK(c, cudaMemcpyAsync(c->p_logw, logw, sizeof(double) * S, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->p_c, cc.data(), sizeof(double) * S, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->dK, &K, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(c, launch_derive(c));
    CK(c, cudaStreamSynchronize(c->stream));
    return DPMM_OK;
}

dpmm_status dpmm_get_params(dpmm_ctx* c, double* logw, double* mu, double* W, double* logdetW, double* logtheta) {
    if (!c) return DPMM_EINVAL;
    if (c->kind != DPMM_PRIOR_NIW && (mu || W || logdetW)) return fail(c, DPMM_EINVAL, "Gaussian parameters of a multinomial chain");
    int K = 0;
    CK(c, cudaMemcpyAsync(&K, c->dK, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const int d = c->d;
    const size_t S = 3 * (size_t)K;
    if (logw) CK(c, cudaMemcpyAsync(logw, c->p_logw, sizeof(double) * S, cudaMemcpyDeviceToHost, c->stream));
    if (mu) CK(c, cudaMemcpyAsync(mu, c->p_mu, sizeof(double) * S * d, cudaMemcpyDeviceToHost, c->stream));
    if (W) CK(c, cudaMemcpyAsync(W, c->p_W, sizeof(double) * S * d * d, cudaMemcpyDeviceToHost, c->stream));
    if (logdetW) CK(c, cudaMemcpyAsync(logdetW, c->p_logdetW, sizeof(double) * S, cudaMemcpyDeviceToHost, c->stream));
    if (logtheta) CK(c, cudaMemcpyAsync(logtheta, c->p_logtheta, sizeof(double) * S * d, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (mu && !c->h_center.empty())
        for (size_t s = 0; s < S; ++s)
            for (int j = 0; j < d; ++j) mu[s * d + j] += c->h_center[j];
    return check_derr(c);
}

dpmm_status dpmm_label_scores(dpmm_ctx* c, double* scores) {
    if (!c || !scores) return DPMM_EINVAL;
    if (!c->X || !c->initialized) return fail(c, DPMM_ESTATE, "no chain");
    int K = 0;
    CK(c, cudaMemcpyAsync(&K, c->dK, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const size_t bytes = sizeof(double) * (size_t)c->N * K;
    CK(c, cudaMalloc(&c->dbg_scores, bytes));
    // the label kernel of this precision with the current parameters; the labels it
    // draws are put back afterwards
    int32_t* zkeep = nullptr;
    CK(c, cudaMalloc(&zkeep, sizeof(int32_t) * c->N));
    CK(c, cudaMemcpyAsync(zkeep, c->z, sizeof(int32_t) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    const bool tc = c->prec == DPMM_PREC_TF32 || c->prec == DPMM_PREC_BF16;
    cudaError_t e = c->sparse                   ? launch_sparse(c, c->seed, 3, nullptr)
                    : c->prec == DPMM_PREC_BF16X3 ? launch_labels_x3(c, c->seed)
                    : tc                        ? launch_labels_tc(c, c->seed)
                                                : launch_labels_simt(c, c->seed);
    CK(c, e);
    CK(c, cudaMemcpyAsync(scores, c->dbg_scores, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(c->z, zkeep, sizeof(int32_t) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    cudaFree(zkeep);
    cudaFree(c->dbg_scores);
    c->dbg_scores = nullptr;
    return check_derr(c);
}

dpmm_status dpmm_profile(dpmm_ctx* c, int enable) {
    if (!c) return DPMM_EINVAL;
    // profiled sweeps run eagerly (events between the launches); a captured graph is kept
    // when the mode does not change, so that resetting the counters leaves replay as it was
    if (enable != c->profiling) drop_graph(c);
    CK(c, cudaStreamSynchronize(c->stream));
    for (auto& p : c->prof)
        for (auto e : p.ev) cudaEventDestroy(e);
    c->prof.clear();
    c->profiling = enable;
    c->nlaunch = 0;
    return DPMM_OK;
}

dpmm_status dpmm_get_profile(dpmm_ctx* c, int cap, const char** names, int* launches, double* ms, int* count) {
    if (!c) return DPMM_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    int i = 0;
    for (auto& p : c->prof) {
        for (size_t q = 0; q + 1 < p.ev.size(); q += 2) {
            float t = 0.f;
            cudaEventElapsedTime(&t, p.ev[q], p.ev[q + 1]);
            p.ms += t;
            cudaEventDestroy(p.ev[q]);
            cudaEventDestroy(p.ev[q + 1]);
        }
        p.ev.clear();
        if (i < cap) {
            if (names) names[i] = p.name.c_str();
            if (launches) launches[i] = p.launches;
            if (ms) ms[i] = p.ms;
        }
        ++i;
    }
    static const char* total = "all_kernels";
    if (i < cap) {
        if (names) names[i] = total;
        if (launches) launches[i] = (int)c->nlaunch;
        if (ms) ms[i] = 0.0;
    }
    ++i;
    if (count) *count = i;
    return DPMM_OK;
}

}  // extern "C"
