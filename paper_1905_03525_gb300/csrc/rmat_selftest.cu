// rmat_selftest.cu -- the failure path of the kernels' bounded waits,
// exercised without faulting anything (see rmat_selftest_bounded_wait in
// include/rmat.h).
#include <cuda_runtime.h>

#include <string>

#include "rmat_device.cuh"
#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {
namespace {

// Failure-path self-test: one warp waits on an mbarrier phase that nothing
// will complete, through the same bounded wait the generation kernels use on
// their table copies, gives up after `limit` polls and records the error in
// the device error word, exactly as a production kernel would.
__global__ void k_wait_selftest(unsigned *err, uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0 && !dev::mbar_wait_bounded(&bar, 0, limit)) atomicOr(err, 1u);
}

}  // namespace

rmat_status launch_wait_selftest(uint32_t limit, cudaStream_t stream) {
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    k_wait_selftest<<<1, 32, 0, stream>>>(props.err, limit);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("self-test launch: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

}  // namespace rmat
