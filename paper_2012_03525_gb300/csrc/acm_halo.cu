// Halo exchange between the z-slabs of a 3D grid split into sub-domains
// (Huang, arXiv:2012.03525, Eqs. 2.10-2.11 in 3D).  The fused step reads
// rho', u, v, w two planes beyond each node (one plane for the fluxes and
// Laplacians of Eq. 2.11, one more through Delta rho = rho^{n+1} - rho^n of
// the density-gradient SAT), so each slab stores two ghost planes beyond
// each z face.  Before every step this kernel copies, for every pair of
// neighbouring slabs (r below, r+1 above, the last slab below the first),
// the top two planes of r into the lower ghost planes of r+1 and the bottom
// two planes of r+1 into the upper ghost planes of r -- what ranks holding
// the slabs on separate GPUs would exchange.  Planes are whole padded x-y
// planes (their x/y ghost columns included), contiguous in memory, so each
// copy is one contiguous range moved in 16-byte words.
#include "acm_internal.h"

namespace acm {
namespace {

template <typename T>
__global__ void k_halo(const RunDesc *__restrict__ runs, int nruns, long long plane, Fields<T> f)
{
    const int y = blockIdx.y;  // (run, direction, field)
    const int r = y >> 3, dir = (y >> 2) & 1, k = y & 3;
    const RunDesc &A = runs[r];
    const RunDesc &B = runs[r + 1 == nruns ? 0 : r + 1];
    long long src, dst;
    if (dir == 0) {  // top two interior planes of A -> lower ghost planes of B
        src = A.off + (long long)(A.zg + A.nz - 2) * plane;
        dst = B.off;
    } else {         // bottom two interior planes of B -> upper ghost planes of A
        src = B.off + (long long)B.zg * plane;
        dst = A.off + (long long)(A.zg + A.nz) * plane;
    }
    const long long nvec = 2 * plane * (long long)sizeof(T) / 16;
    const uint4 *s = reinterpret_cast<const uint4 *>(f.f[k] + src);
    uint4 *d = reinterpret_cast<uint4 *>(f.f[k] + dst);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvec;
         i += (long long)gridDim.x * blockDim.x)
        d[i] = s[i];
}

}  // namespace

template <typename T>
cudaError_t launch_halo(const RunDesc *druns, int nruns, long long plane, Fields<T> f,
                        cudaStream_t s)
{
    // plane (elements) is a multiple of 8 and every run offset a multiple of
    // 32 elements, so every range starts and ends on a 16-byte boundary
    dim3 grid(32, 8 * nruns);
    k_halo<T><<<grid, 256, 0, s>>>(druns, nruns, plane, f);
    return cudaGetLastError();
}

template cudaError_t launch_halo<float>(const RunDesc *, int, long long, Fields<float>,
                                        cudaStream_t);
template cudaError_t launch_halo<double>(const RunDesc *, int, long long, Fields<double>,
                                         cudaStream_t);

}  // namespace acm
