// acm_reduce_mass_noalloc: the FP64 diagnostics of acm_reduce_mass for
// caller-owned device fields, without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want
// diagnostics: code whose device memory is owned entirely by another runtime
// (a framework's caching allocator or a fixed, pre-sized pool that must not
// fragment or grow), and loops with a hard latency budget that forbid
// allocation after start-up (cudaMalloc/cudaFree may synchronise the device).
// For them the two-pass reduction keeps its block partials and its run
// descriptor in file-scope __device__ arrays of a fixed maximum size instead
// of memory the library would otherwise cudaMalloc.  Those arrays exist on
// every GPU that loads the library, until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "acm_internal.h"

namespace {

// at most this many pass-1 blocks, i.e. partials of 8 doubles each (256 KiB)
constexpr int NOALLOC_MAX_BLOCKS = 4096;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_partials[NOALLOC_MAX_BLOCKS * 8];
static __device__ __align__(256) acm::RunDesc g_run;

// device addresses of the arrays above, resolved once per device (in host
// code the array names are host-side stand-ins, not device addresses)
double *g_partials_dev[MAX_DEVICES];
acm::RunDesc *g_run_dev[MAX_DEVICES];
std::mutex g_setup_mutex;
thread_local std::string g_noalloc_err;

// writes the run descriptor from a kernel argument: the launch copies the
// argument by value, so the call neither reads pageable host memory
// asynchronously nor waits for the stream
__global__ void k_set_run(acm::RunDesc R) { g_run = R; }

acm_status noalloc_fail(acm_status st, const std::string &msg)
{
    g_noalloc_err = msg;
    return st;
}

}  // namespace

extern "C" const char *acm_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

extern "C" acm_status acm_reduce_mass_noalloc(int dim, int nx, int ny, int nz, int precision,
                                              double rho0, const void *rho, const void *u,
                                              const void *v,
                                              const void *w, const void *u_prev,
                                              const void *v_prev, const void *w_prev, int blocks,
                                              double *out_dev, void *stream)
{
    if (dim != 2 && dim != 3) return noalloc_fail(ACM_EINVAL, "dim must be 2 or 3");
    if (nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1))
        return noalloc_fail(ACM_EINVAL, "grid sizes must be >= 1 (nz = 1 in 2D)");
    if (precision != ACM_FP64 && precision != ACM_FP32_DEV)
        return noalloc_fail(ACM_EINVAL, "bad precision");
    if (!std::isfinite(rho0)) return noalloc_fail(ACM_EINVAL, "rho0 must be finite");
    if (!rho || !u || !v || (dim == 3 && !w) || !out_dev)
        return noalloc_fail(ACM_EINVAL, "missing field or output pointer");
    if ((u_prev || v_prev || w_prev) && (!u_prev || !v_prev || (dim == 3 && !w_prev)))
        return noalloc_fail(ACM_EINVAL, "previous velocity needs every component");
    const long long n = (long long)nx * ny * nz;
    if (blocks < 0 || blocks > NOALLOC_MAX_BLOCKS)
        return noalloc_fail(ACM_EINVAL, "blocks must be 0..4096 (the fixed scratch holds the "
                                        "partials of at most 4096 blocks)");
    if (blocks == 0) blocks = (int)std::min<long long>((n + 255) / 256, 1024);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(ACM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return noalloc_fail(ACM_EINVAL, "device index too large");
    {
        // first call on this device: resolve the device addresses (no allocation)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_dev[dev]) {
            void *p = nullptr, *q = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_run);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();  // the failure must not outlive this call
                return noalloc_fail(ACM_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e));
            }
            g_run_dev[dev] = static_cast<acm::RunDesc *>(q);
            g_partials_dev[dev] = static_cast<double *>(p);
        }
    }

    // the run descriptor of the existing reduction kernels: an unpadded grid
    // holding rho - rho0
    acm::RunDesc R;
    std::memset(&R, 0, sizeof(R));
    R.nx = nx;
    R.ny = ny;
    R.nz = nz;
    R.px = nx;
    R.py = ny;
    R.pad = 0;
    R.off = 0;
    R.rho0 = rho0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_set_run<<<1, 1, 0, s>>>(R);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(ACM_ECUDA, cudaGetErrorString(e));

    if (precision == ACM_FP64) {
        acm::Fields<double> f{};
        f.f[acm::F_R] = const_cast<double *>(static_cast<const double *>(rho));
        f.f[acm::F_U] = const_cast<double *>(static_cast<const double *>(u));
        f.f[acm::F_V] = const_cast<double *>(static_cast<const double *>(v));
        f.f[acm::F_W] = const_cast<double *>(static_cast<const double *>(w));
        e = acm::launch_reduce<double>(g_run_dev[dev], 1, dim, f,
                                       static_cast<const double *>(u_prev),
                                       static_cast<const double *>(v_prev),
                                       static_cast<const double *>(w_prev), g_partials_dev[dev],
                                       blocks, out_dev, s);
    } else {
        acm::Fields<float> f{};
        f.f[acm::F_R] = const_cast<float *>(static_cast<const float *>(rho));
        f.f[acm::F_U] = const_cast<float *>(static_cast<const float *>(u));
        f.f[acm::F_V] = const_cast<float *>(static_cast<const float *>(v));
        f.f[acm::F_W] = const_cast<float *>(static_cast<const float *>(w));
        e = acm::launch_reduce<float>(g_run_dev[dev], 1, dim, f,
                                      static_cast<const float *>(u_prev),
                                      static_cast<const float *>(v_prev),
                                      static_cast<const float *>(w_prev), g_partials_dev[dev],
                                      blocks, out_dev, s);
    }
    if (e != cudaSuccess) return noalloc_fail(ACM_ECUDA, cudaGetErrorString(e));
    return ACM_OK;
}
