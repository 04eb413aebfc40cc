// cdg2_vjp_noalloc: the VJP entry point for callers that cannot allocate
// device memory.
//
// cdg2_vjp allocates a per-mesh workspace (cudaMalloc) the first time a theta
// gradient is requested.  Some callers cannot allow that: an application
// whose device memory is entirely reserved by its own pool allocator (a
// framework's caching allocator that has already taken the free memory), or
// a latency-critical loop that must never hit the implicit device-wide
// synchronisation of cudaMalloc / cudaFree.  This entry point computes the
// same result with its scratch in a fixed device array that is part of the
// library image: it calls no cudaMalloc, cudaFree or allocating routine.
//
// The scratch holds the per-CTA partial sums of the theta gradient (8
// doubles per CTA of the VJP kernel).  Every CTA overwrites its own 8 slots
// before the reduction reads them, so nothing in the array has to start at
// zero and no clearing pass is needed.  A second static word holds the
// domain status of the call (a pole of chi met at some quadrature point); it
// starts at zero and is cleared whenever it is reported.  Both are shared by
// every call in the process: calls that overlap on the GPU (on different
// streams, or from different threads without ordering) race on them.
//
// CUDA loads a library's device code lazily by default: the module holding
// these arrays is loaded on a device by the first call there (when it looks
// up their addresses), and that load is when the arrays take their device
// memory.  Later calls take none.
#include <mutex>

#include "cdg2_internal.h"

namespace cdg2 {

// Maximum number of VJP CTAs: 16384 x 8 doubles = 1 MiB of device memory,
// held by every GPU that loads the library until the process exits.
constexpr long long NOALLOC_MAX_CTAS = 16384;

static __device__ __align__(256) double g_noalloc_theta_part[NOALLOC_MAX_CTAS * 8];
static __device__ __align__(256) int g_noalloc_status;

struct NoallocAddr {
    double* part = nullptr;
    int* status = nullptr;
};

// Device addresses of the scratch array and the status word, looked up once
// per device with that device current.  In host code the symbols' names are
// only host-side stand-ins; the kernels must be given these addresses.
static NoallocAddr noalloc_scratch(int device, cudaError_t* err) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static NoallocAddr addr[kMaxDevices];
    *err = cudaSuccess;
    if (device < 0 || device >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return NoallocAddr{};
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device].part) {
        void* p = nullptr;
        void* q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_theta_part);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_status);
        if (e != cudaSuccess) {
            *err = e;
            return NoallocAddr{};
        }
        addr[device].part = static_cast<double*>(p);
        addr[device].status = static_cast<int*>(q);
    }
    return addr[device];
}

}  // namespace cdg2

using namespace cdg2;

extern "C" int cdg2_vjp_noalloc(const cdg2_mesh* m, const cdg2_params* p, const void* U, const void* lam, void* gU,
                                double* gtheta, int flags, double t, void* stream) {
    (void)t;
    if (!m || !p || !U || !lam || !gU) {
        set_error("cdg2_vjp_noalloc: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (gU == U || gU == lam) {
        set_error("cdg2_vjp_noalloc: gU must not overlap U or lam");
        return CDG2_ERR_INVALID_ARG;
    }
    if (flags & ~(CDG2_MINV | CDG2_FORCING | CDG2_FP32)) {
        set_error("cdg2_vjp_noalloc: unknown flag bits (CDG2_ASYNC is not accepted here)");
        return CDG2_ERR_INVALID_ARG;
    }
    const long long ctas = vjp_grid(*m);
    if (gtheta && ctas > NOALLOC_MAX_CTAS) {
        set_error("cdg2_vjp_noalloc: the mesh needs " + std::to_string(ctas) +
                  " VJP CTAs; the static scratch holds at most " + std::to_string(NOALLOC_MAX_CTAS) +
                  " (use cdg2_vjp for larger meshes)");
        return CDG2_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_vjp_noalloc: cudaGetDevice");
    const NoallocAddr a = noalloc_scratch(dev, &e);
    if (!a.part) return cuda_fail(e, "cdg2_vjp_noalloc: cudaGetSymbolAddress");
    Coef c = make_coef(*p);
    e = launch_vjp(*m, c, U, lam, gU, gtheta ? a.part : nullptr, gtheta, flags, (cudaStream_t)stream, a.status);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_vjp_noalloc");
    return take_domain_status(a.status, (cudaStream_t)stream, "cdg2_vjp_noalloc");
}
