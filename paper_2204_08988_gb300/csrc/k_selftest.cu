// k_selftest.cu -- failure-detection check of the bounded device waits (no counterpart in
// the paper): one thread waits, with the bounded mbarrier wait every tensor-core kernel
// uses, on a barrier that nothing arrives at.  The wait gives up after its poll or cycle
// limit and the kernel records DPMM_ETIMEOUT in the device error word, exactly as the
// production kernels do when a wait runs out; nothing traps and the context stays usable.
#include "dpmm_internal.cuh"
#include "tc_ptx.cuh"

namespace dpmm {

__global__ void wait_selftest_kernel(int* derr) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // phase 0 of a fresh barrier completes only when one arrival lands: none will
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, &abort_flag)) atomicExch(derr, (int)DPMM_ETIMEOUT);
}

cudaError_t launch_wait_selftest(dpmm_ctx* c) {
    wait_selftest_kernel<<<1, 32, 0, c->stream>>>(c->derr);
    return cudaGetLastError();
}

}  // namespace dpmm
