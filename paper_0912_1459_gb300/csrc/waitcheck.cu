// Check of the bounded device-side wait that every tensor-core kernel uses
// (no counterpart in the paper).  One thread waits, through the kernels' own
// mbar_wait, on an mbarrier phase that nothing ever completes; the wait must
// give up after its limit, write CDS_ERR_TIMEOUT to the error word and let
// the kernel return, so the context stays usable.  Nothing traps or hangs.
#include "tcgen05.cuh"

namespace cds {
namespace {

__global__ void k_wait_unarrived(unsigned long long limit_ns, int32_t* __restrict__ err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);   // expects one arrival; none is ever made
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool done = tc::mbar_wait(&bar, 0u, err, false, limit_ns);
        if (done) atomicExch(err, (int32_t)CDS_OK);   // not reachable: the phase never completes
    }
}

}  // namespace
}  // namespace cds

extern "C" int cds_wait_check(double seconds, int32_t* err, cudaStream_t stream) {
    if (!err || !(seconds > 0.0) || seconds > 2.0) return CDS_ERR_ARG;
    const unsigned long long ns = (unsigned long long)(seconds * 1e9);
    CDS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), stream));
    cds::k_wait_unarrived<<<1, 32, 0, stream>>>(ns, err);
    CDS_LAUNCH_CHECK();
    int32_t h = 0;
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    return h;
}
