// selftest.cu -- exercises the bounded mbarrier wait that every pipeline
// wait of the stream-collide kernel goes through: a barrier that nothing
// arrives on must make the wait give up after its cycle limit, report it,
// and leave the context usable.  (No counterpart in the paper.)
#include "../../include/iblb.h"
#include "iblb_internal.h"
#include "mbarrier.cuh"

namespace iblb {
namespace {

// 32 threads wait on a barrier initialised for one arrival that never
// comes; out[0] counts the threads whose wait gave up, out[1] those whose
// wait completed
__global__ void __launch_bounds__(32) wait_timeout_kernel(long long cycles, int *out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bar, 0, cycles);
    atomicAdd(&out[ok ? 1 : 0], 1);
}

__device__ int g_selftest_out[2];

}  // namespace
}  // namespace iblb

extern "C" {

int iblb_selftest_wait_timeout(long long cycles, void *stream)
{
    using namespace iblb;
    if (cycles < 1000 || cycles > 10000000000LL)
        return IBLB_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int *d_out = nullptr;
    const int zero[2] = {0, 0};
    int res[2] = {0, 0};
    if (cudaGetSymbolAddress((void **)&d_out, g_selftest_out) != cudaSuccess ||
        cudaMemcpyAsync(d_out, zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return IBLB_E_CUDA;
    wait_timeout_kernel<<<1, 32, 0, s>>>(cycles, d_out);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(res, d_out, sizeof(res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return IBLB_E_CUDA;
    if (res[0] == 32 && res[1] == 0)
        return IBLB_E_TIMEOUT;          // every wait gave up, as it must
    return res[1] == 32 ? IBLB_OK : IBLB_E_STATE;
}

}  // extern "C"
