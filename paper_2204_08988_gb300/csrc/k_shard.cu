// k_shard.cu -- the statistics exchange of a point-sharded sweep.
//
// When the N points of one chain are split over G contexts (one per GPU in a multi-GPU
// run, or several on one GPU), every step of Sec. 4.1 that depends on all points reads
// only the sufficient statistics (Sec. 4.4): the parameter draws (a)-(d), the split and
// merge ratios and the removal of emptied clusters.  Each shard computes the statistics
// of its own points; the chain's statistics are their sum, formed here in a fixed order
// (shard 0 + shard 1 + ... + shard G-1, entry by entry) and written back to every shard,
// so every shard then takes the same parameter, split and merge decisions with the same
// counter-based random numbers.  Integer counts are exact in any order; the FP64 sums of a
// sharded chain differ from an unsharded one's only by rounding.
#include "dpmm_internal.cuh"

namespace dpmm {

constexpr int MAX_SHARDS = 16;

template <typename T>
struct ShardPtrs {
    T* p[MAX_SHARDS];
};

// out[e] = sum_s t_s[e], s in increasing order, for e < n_per_k * K (K read on the device)
template <typename T>
__global__ void shard_sum_kernel(ShardPtrs<T> t, int G, const int* dK, int64_t per_k, const int* gate, T* out) {
    if (gate && *gate == 0) return;
    const int64_t n = per_k * (int64_t)(*dK);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        T v = t.p[0][e];
        for (int s = 1; s < G; ++s) v += t.p[s][e];
        out[e] = v;
    }
}

template <typename T>
__global__ void shard_bcast_kernel(ShardPtrs<T> t, int G, const int* dK, int64_t per_k, const int* gate, const T* in) {
    if (gate && *gate == 0) return;
    const int64_t n = per_k * (int64_t)(*dK);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const T v = in[e];
        for (int s = 0; s < G; ++s) t.p[s][e] = v;
    }
}

template <typename T>
static cudaError_t exchange_t(dpmm_ctx* const* sh, int G, T* (*field)(dpmm_ctx*), int64_t per_k, T* scratch,
                              const int* gate) {
    dpmm_ctx* c = sh[0];
    ShardPtrs<T> t{};
    for (int s = 0; s < G; ++s) t.p[s] = field(sh[s]);
    const int grid = 4 * c->num_sms;
    shard_sum_kernel<T><<<grid, 256, 0, c->stream>>>(t, G, c->dK, per_k, gate, scratch);
    shard_bcast_kernel<T><<<grid, 256, 0, c->stream>>>(t, G, c->dK, per_k, gate, scratch);
    c->nlaunch += 2;
    return cudaGetLastError();
}

static double* f_stats(dpmm_ctx* c) { return c->stats; }
static float* f_cc(dpmm_ctx* c) { return c->sp_cc; }

// Sum the shards' statistics tables (2 sub-clusters x E entries per cluster; for compressed
// rows also the compact counts, 2 x d per cluster) in shard order and give every shard the
// sum, on shard 0's stream (the caller orders the shards' streams around it).  gate: the
// device flag that says the shards recounted their statistics (NULL: always).
cudaError_t shard_exchange(dpmm_ctx* const* sh, int G, const int* gate) {
    dpmm_ctx* c = sh[0];
    if (G < 1 || G > MAX_SHARDS) return cudaErrorInvalidValue;
    if (!c->shard_scratch) {
        size_t bytes = sizeof(double) * 2 * (size_t)c->K_max * c->st.E;
        if (c->sparse) bytes = std::max(bytes, sizeof(float) * 2 * (size_t)c->K_max * c->d);
        cudaError_t e = cudaMalloc(&c->shard_scratch, bytes);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = exchange_t<double>(sh, G, f_stats, 2 * (int64_t)c->st.E, (double*)c->shard_scratch, gate);
    if (e == cudaSuccess && c->sparse)
        e = exchange_t<float>(sh, G, f_cc, 2 * (int64_t)c->d, (float*)c->shard_scratch, gate);
    return e;
}

}  // namespace dpmm
