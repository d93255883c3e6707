// selftest.cu -- the bounded-wait path of the tensor-core engines, exercised
// on purpose: one thread waits on an mbarrier that nothing arrives on, gives
// up after the wall-clock limit and latches VPX_ERR_TIMEOUT, exactly as an
// engine's producer, MMA issuer or epilogue would.  The context stays usable.
#include "bulk.cuh"
#include "dev_common.cuh"

namespace vpx {

__global__ void k_wait_probe(int *status, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(bulk_smem_addr(&bar), 0, limit_ns, 1000))
        set_status(status, VPX_ERR_TIMEOUT);
}

int device_check_bounded_wait(int *status_out) {
    int *d = dev_alloc<int>(1);
    VPX_CUDA(cudaMemset(d, 0, sizeof(int)));
    k_wait_probe<<<1, 32>>>(d, 20000000ull);   // 20 ms
    VPX_LAUNCH("k_wait_probe");
    VPX_CUDA(cudaDeviceSynchronize());
    VPX_CUDA(cudaMemcpy(status_out, d, sizeof(int), cudaMemcpyDeviceToHost));
    dev_free(d);
    return VPX_OK;
}

}  // namespace vpx
