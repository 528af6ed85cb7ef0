// k_noalloc.cu -- sufficient statistics of given labels without any allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// statistics: an application that reserves the GPU's memory up front in its own pool
// and forbids any later cudaMalloc (a serving process that owns all of HBM, a host
// framework whose plug-ins must not allocate), or latency-critical code that must not
// take the implicit device-wide synchronisation a cudaMalloc/cudaFree can cause.  This
// entry point computes, for every sub-cluster (k, h), the count, the sum of x and the
// sum of x x^T of the points labelled (z = k, zbar = h), using only the caller's
// buffers and a fixed scratch array that lives in this library's device image.  The
// scratch (NA_G x 2 NA_KMAX x NA_EMAX doubles = 5.6 MiB) is held by every GPU that
// loads the library until the process exits.
#include <cuda.h>

#include <mutex>

#include "dpmm_internal.cuh"

namespace dpmm {

constexpr int NA_G = 32;      // CTAs of the partial pass (one scratch slice each)
constexpr int NA_KMAX = 16;   // clusters
constexpr int NA_DMAX = 32;   // dimension
constexpr int NA_P = 128;     // points per tile
constexpr int NA_EMAX = 16 * (((NA_DMAX + 4) / 4) * ((NA_DMAX + 4) / 4 + 1) / 2);  // 720 entries

static __device__ __align__(256) double g_na_scratch[(size_t)NA_G * 2 * NA_KMAX * NA_EMAX];

// Pass 1: CTA g owns slice g (2K slots x E).  It clears the slice, then, tile by
// tile, groups the tile's points by slot (stable ranks) and adds each slot's 4x4
// register-block sums of xt xt^T (xt = [x, 1]) into its slice, in FP64.
__global__ void __launch_bounds__(256) na_partial_kernel(const float* __restrict__ X, int64_t N, int d,
                                                         const int32_t* __restrict__ z,
                                                         const uint8_t* __restrict__ zbar, int K,
                                                         StatLayout L, int G, double* scratch) {
    __shared__ float xs[NA_P * (NA_DMAX + 4)];
    __shared__ int slot[NA_P], order[NA_P], cnt[2 * NA_KMAX + 2];
    __shared__ float red[256 * 16];
    const int tid = threadIdx.x, nt = blockDim.x, g = blockIdx.x;
    const int S = 2 * K, dp = L.dp, nblk = L.nblk, E = L.E;
    double* slice = scratch + (size_t)g * S * E;
    for (int e = tid; e < S * E; e += nt) slice[e] = 0.0;  // the array keeps the last call's contents
    const int64_t R = (N + G - 1) / G, p0 = (int64_t)g * R, p1 = min(N, p0 + R);
    const int ngrp = max(1, nt / nblk);
    const bool worker = tid < nblk * ngrp;
    const int myblk = worker ? tid % nblk : 0, grp = worker ? tid / nblk : 0;
    int jb = 0, lb = 0;
    L.blk_coords(myblk, jb, lb);
    for (int64_t base = p0; base < p1; base += NA_P) {
        const int np = (int)min((int64_t)NA_P, p1 - base);
        __syncthreads();
        if (tid < np) {
            const int64_t i = base + tid;
            float* xr = xs + tid * dp;
            for (int j = 0; j < d; ++j) xr[j] = X[i * d + j];
            xr[d] = 1.f;
            for (int j = d + 1; j < dp; ++j) xr[j] = 0.f;
            const int zi = z[i], hi = zbar[i];
            // a label outside [0, K) x {0, 1} goes to the discard slot S and is not counted
            slot[tid] = (zi >= 0 && zi < K && hi <= 1) ? 2 * zi + hi : S;
        }
        if (tid <= S + 1) cnt[tid] = 0;
        __syncthreads();
        if (tid < np) {  // stable position of this point among the tile's points of its slot
            int s = slot[tid], r = 0;
            for (int q = 0; q < tid; ++q) r += slot[q] == s;
            order[tid] = r;
            atomicAdd(&cnt[s + 1], 1);
        }
        __syncthreads();
        if (tid == 0)
            for (int s = 0; s <= S; ++s) cnt[s + 1] += cnt[s];
        __syncthreads();
        if (tid < np) {
            int pos = cnt[slot[tid]] + order[tid];
            order[tid] = pos;  // reuse: position of point tid in slot order
        }
        __syncthreads();
        // inverse permutation into slot[] (points in slot order)
        int mypos = tid < np ? order[tid] : -1;
        __syncthreads();
        if (tid < np) slot[mypos] = tid;
        __syncthreads();
        for (int s = 0; s < S; ++s) {
            const int qs = cnt[s], qe = cnt[s + 1];
            if (qs == qe) continue;  // uniform across the block
            float acc[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[e] = 0.f;
            if (worker)
                for (int q = qs + grp; q < qe; q += ngrp) {
                    const float* xr = xs + slot[q] * dp;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u * 4 + v] += xr[jb * 4 + u] * xr[lb * 4 + v];
                }
            if (worker)
#pragma unroll
                for (int e = 0; e < 16; ++e) red[tid * 16 + e] = acc[e];
            __syncthreads();
            for (int e = tid; e < nblk * 16; e += nt) {
                const int b = e >> 4, q = e & 15;
                double v = 0.0;
                for (int gg = 0; gg < ngrp; ++gg) v += (double)red[(gg * nblk + b) * 16 + q];
                slice[(size_t)s * E + e] += v;
            }
            __syncthreads();
        }
    }
}

// Pass 2: sum the slices in CTA order (deterministic) and unpack n, sum x, sum x x^T.
__global__ void na_combine_kernel(StatLayout L, int G, int K, const double* scratch, double* n_out, double* sx_out,
                                  double* sxx_out) {
    const int s = blockIdx.x, d = L.d, S = 2 * K, E = L.E;
    auto M = [&](int j, int l) {
        const int e = L.ent(j, l);
        double v = 0.0;
        for (int g = 0; g < G; ++g) v += scratch[((size_t)g * S + s) * E + e];
        return v;
    };
    for (int q = threadIdx.x; q < d * d; q += blockDim.x) {
        const int j = q / d, l = q % d;
        sxx_out[(size_t)s * d * d + q] = j <= l ? M(j, l) : M(l, j);
    }
    for (int j = threadIdx.x; j < d; j += blockDim.x) sx_out[(size_t)s * d + j] = M(j, d);
    if (threadIdx.x == 0) n_out[s] = M(d, d);
}

// The scratch address is looked up (cudaGetSymbolAddress) once per device and per
// context: the array sits at a different address in every context the module is loaded
// into, so the cache is keyed by the context current at the call (cuCtxGetCurrent,
// resolved through the runtime's driver entry point), not by the device ordinal alone.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
static std::mutex g_na_mu;
static struct {
    CUcontext ctx;
    void* ptr;
} g_na_cache[128];

static CUcontext na_current_context() {
    static CtxGetCurrentFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)p;
    }
    CUcontext cx = nullptr;
    if (fn && fn(&cx) != CUDA_SUCCESS) cx = nullptr;
    return cx;
}

}  // namespace dpmm

using namespace dpmm;

extern "C" dpmm_status dpmm_suffstats_noalloc(const float* X, int64_t N, int d, const int32_t* z,
                                              const uint8_t* zbar, int K, double* n_out, double* sx_out,
                                              double* sxx_out, void* stream) {
    if (!X || !z || !zbar || !n_out || !sx_out || !sxx_out) return DPMM_EINVAL;
    if (N < 1 || d < 1 || d > NA_DMAX || K < 1 || K > NA_KMAX) return DPMM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return DPMM_ECUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        const CUcontext cx = na_current_context();
        if (!g_na_cache[dev].ptr || !cx || g_na_cache[dev].ctx != cx) {  // set-up, with that device current
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return DPMM_ECUDA;
            // the lookup has made the runtime's context current if none was
            g_na_cache[dev].ctx = na_current_context();
            g_na_cache[dev].ptr = p;
        }
        scratch = (double*)g_na_cache[dev].ptr;
    }
    StatLayout L;
    L.init(d, STAT_FULL);
    cudaStream_t s = (cudaStream_t)stream;
    int G = NA_G;
    // launched with cudaLaunchKernel, whose return value is this launch's own error (an
    // error left behind by an unrelated earlier launch is neither reported nor cleared)
    void* a1[] = {(void*)&X, (void*)&N, (void*)&d, (void*)&z, (void*)&zbar, (void*)&K, (void*)&L, (void*)&G,
                  (void*)&scratch};
    if (cudaLaunchKernel((const void*)na_partial_kernel, dim3(NA_G), dim3(256), a1, 0, s) != cudaSuccess)
        return DPMM_ECUDA;
    const double* cs = scratch;
    void* a2[] = {(void*)&L, (void*)&G, (void*)&K, (void*)&cs, (void*)&n_out, (void*)&sx_out, (void*)&sxx_out};
    if (cudaLaunchKernel((const void*)na_combine_kernel, dim3(2 * K), dim3(128), a2, 0, s) != cudaSuccess)
        return DPMM_ECUDA;
    return DPMM_OK;
}
