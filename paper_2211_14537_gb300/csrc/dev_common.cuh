// dev_common.cuh -- CUDA helpers shared by the setup and execute translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "plan.h"

namespace vpx {

inline void cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        if (e == cudaErrorMemoryAllocation) fail(VPX_ERR_NOMEM, std::string(what) + ": " + cudaGetErrorString(e));
        if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
            fail(VPX_ERR_NODEV, std::string(what) + ": " + cudaGetErrorString(e));
        fail(VPX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}
#define VPX_CUDA(x) ::vpx::cuda_check((x), #x)
#define VPX_LAUNCH(what) ::vpx::cuda_check(cudaGetLastError(), what)

template <class T>
T *dev_alloc(size_t n) {
    T *p = nullptr;
    if (n == 0) n = 1;
    VPX_CUDA(cudaMalloc((void **)&p, n * sizeof(T)));
    return p;
}

template <class T>
T *dev_upload(const std::vector<T> &v) {
    T *p = dev_alloc<T>(v.size());
    if (!v.empty()) VPX_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

template <class T>
void dev_free(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// device status codes latched by kernels
__device__ inline void set_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

}  // namespace vpx
