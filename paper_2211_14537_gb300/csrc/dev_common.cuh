// dev_common.cuh -- CUDA helpers shared by the setup and execute translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>

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

// Programmatic dependent launch.  Every kernel of the execute path starts with
// pdl_entry(): it waits until the grids this one depends on have completed and
// their writes are visible.  Launched programmatically (launch_pdl), a kernel
// is scheduled as the previous kernel's blocks retire rather than after that
// grid's completion has been signalled, which hides part of the launch gap.
// No kernel triggers its dependents early: dependents resident before their
// inputs exist held registers and shared memory that the kernels on the other
// streams needed (the step got 13 % slower).  Without a programmatic launch
// the wait is a no-op.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

bool pdl_enabled();   // false when VPX_NO_PDL is set (read once)

// Scheduling priority of the launches made on this thread (a hint to the
// block scheduler, recorded in captured graphs): kNoPriority leaves the
// stream's own.  The execute path runs its critical chain at the device's
// greatest priority and the near field, which only has to finish by the end,
// at the least, so that it yields SMs to the chain.
constexpr int kNoPriority = -1000000;
int &launch_priority();
int priority_greatest();
int priority_least();
struct LaunchPriority {
    int prev;
    explicit LaunchPriority(int p) : prev(launch_priority()) { launch_priority() = p; }
    ~LaunchPriority() { launch_priority() = prev; }
};

// kernel<<<grid, block, smem, s>>>(args...) with the programmatic
// stream-serialization attribute: the kernel may begin while the previous
// kernel of the stream finishes (it waits in pdl_entry for that kernel's data)
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    unsigned n_attr = 1;
    if (launch_priority() != kNoPriority) {
        attr[1].id = cudaLaunchAttributePriority;
        attr[1].val.priority = launch_priority();
        n_attr = 2;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = n_attr;
    VPX_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

}  // namespace vpx
