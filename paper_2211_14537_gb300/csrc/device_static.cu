// device_static.cu -- vpx_potential_static: the volume-potential passes with
// their expansion scratch in a fixed, file-scope device array instead of the
// plan's workspace, so that the call itself allocates nothing.
//
// Who needs it: callers that must not allocate device memory at the point of
// the call -- a serving loop that has handed the whole device to its own pool
// allocator and forbids raw cudaMalloc, or a latency-bound step that cannot
// afford an allocation (or its failure) in the middle of a run.
//
// The array below (VPX_STATIC_SCRATCH_DOUBLES doubles = 16 MiB) exists on
// every GPU that loads this library, from module load until process exit.
// Its device address is looked up once per device (cudaGetSymbolAddress,
// with that device current) on the first call made on that device.
#include <mutex>

#include "dev_common.cuh"

namespace vpx {

void run_potential_scratch(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv, double *vb,
                           int64_t ldb, double *mp, double *lo, cudaStream_t s, bool fe_sliced);

static __device__ __align__(256) double g_static_scratch[VPX_STATIC_SCRATCH_DOUBLES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the static scratch array on the current device.
static double *static_scratch_address() {
    int dev = 0;
    VPX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(VPX_ERR_ARG, "device index out of range for the static scratch table");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) fail(VPX_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = (double *)ptr;
    }
    return g_addr[dev];
}

namespace {
// Makes the plan's device current for the lifetime of the guard and puts the
// caller's device back on every exit, the error paths included.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        VPX_CUDA(cudaGetDevice(&prev));
        if (prev != dev) VPX_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};
}  // namespace

void ev_record(vpx_plan *p, int i, cudaStream_t s);

void device_potential_static(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv,
                             double *vb, int64_t ldb, void *stream) {
    const int64_t per = (int64_t)nrhs * p->dt.n_boxes * 2 * p->P;   // one expansion array
    if (2 * per > (int64_t)VPX_STATIC_SCRATCH_DOUBLES)
        fail(VPX_ERR_ARG, "vpx_potential_static: nrhs * n_boxes * 4(p+1) = " + std::to_string(2 * per) +
                              " doubles exceeds the static scratch of " +
                              std::to_string((long long)VPX_STATIC_SCRATCH_DOUBLES));
    DeviceGuard guard(p->device);
    double *base = static_scratch_address();
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = stream;
    ev_record(p, 0, s);
    // the passes zero both expansion arrays at the start of every call (the
    // scratch keeps the previous call's values until then)
    run_potential_scratch(p, fe, ldfe, nrhs, v, ldv, vb, ldb, base, base + per, s, false);
}

}  // namespace vpx
