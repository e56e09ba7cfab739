// FP64 diagnostics beyond the integral sums of acm_reduce.cu:
//   * the velocity error of Eq. (3.2) (Section 3.1) against a reference
//     field staged from the host;
//   * the Laplace-law quantities of a two-phase run: the drop's area or
//     volume, its effective radius and the chemical potential of Section 2,
//     mu = 4 a phi (phi^2 - 1) - kappa Lap_iso(phi), averaged with the
//     interface weight (1 - phi^2) and over the two bulk phases, and the
//     pressure difference between them.
// Both are deterministic two-pass reductions (fixed slices per block, fixed
// trees, block partials summed in block order).
#include <cmath>

#include "acm_internal.h"

namespace acm {
namespace {

constexpr int DT = 256;  // threads per block

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *dst)
{
    __shared__ double red[NV][DT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int q = threadIdx.x;
        double x = red[q][0];
        for (int k = 1; k < DT / 32; ++k) x += red[q][k];
        dst[q] = x;
    }
}

// storage offset of node (x, y, z) of run R (unpadded coordinates)
__device__ __forceinline__ long long sidx(const RunDesc &R, int x, int y, int z)
{
    return R.off + ((long long)(z + R.zg) * R.py + (y + R.pad)) * R.px + (x + R.pad);
}

// sum (f - ref)^2 and sum ref^2 over the nodes of run R; ref is unpadded
// [z][y][x].  Blocks take rows (z, y) in turn, threads stride along x.
template <typename T>
__global__ void __launch_bounds__(DT)
    k_err(const RunDesc R, const T *__restrict__ f, const double *__restrict__ ref,
          double *partials)
{
    double v[2] = {0.0, 0.0};
    const int nrow = R.ny * R.nz;
    for (int row = blockIdx.x; row < nrow; row += gridDim.x) {
        const int z = row / R.ny, y = row - z * R.ny;
        const long long b = sidx(R, 0, y, z);
        const long long rb = (long long)row * R.nx;
        for (int x = threadIdx.x; x < R.nx; x += DT) {
            const double a = ref[rb + x];
            const double d = (double)f[b + x] - a;
            v[0] += d * d;
            v[1] += a * a;
        }
    }
    block_sum<2>(v, partials + 2 * blockIdx.x);
}

__global__ void k_err_final(const double *partials, int blocks, double *out)
{
    if (threadIdx.x != 0) return;
    double num = 0.0, den = 0.0;
    for (int b = 0; b < blocks; ++b) {
        num += partials[2 * b];
        den += partials[2 * b + 1];
    }
    *out = den > 0.0 ? sqrt(num / den) : sqrt(num);
}

constexpr int NL = 9;  // partial sums of the Laplace diagnostics

// Lap_iso(phi) at an interior node with D2Q9 (2D) or D3Q19 (3D) weights
// (the reading of the paper's "second order isotropic schemes"):
// 2D (2/3)(sum_axis - 4 phi) + (1/6)(sum_diag - 4 phi);
// 3D (1/3)(sum_axis - 6 phi) + (1/6)(sum_edge - 12 phi).
template <typename T>
__device__ double lap_iso(const RunDesc &R, int dim, const T *phi, int x, int y, int z)
{
    auto wr = [](int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); };
    auto at = [&](int dx, int dy, int dz) {
        return (double)phi[sidx(R, wr(x + dx, R.nx), wr(y + dy, R.ny),
                                dim == 3 ? wr(z + dz, R.nz) : 0)];
    };
    const double c = at(0, 0, 0);
    if (dim == 2) {
        const double ax = at(1, 0, 0) + at(-1, 0, 0) + at(0, 1, 0) + at(0, -1, 0);
        const double dg = at(1, 1, 0) + at(-1, 1, 0) + at(1, -1, 0) + at(-1, -1, 0);
        return (2.0 / 3.0) * (ax - 4.0 * c) + (1.0 / 6.0) * (dg - 4.0 * c);
    }
    const double ax = at(1, 0, 0) + at(-1, 0, 0) + at(0, 1, 0) + at(0, -1, 0) + at(0, 0, 1) +
                      at(0, 0, -1);
    const double ed = at(1, 1, 0) + at(-1, 1, 0) + at(1, -1, 0) + at(-1, -1, 0) + at(1, 0, 1) +
                      at(-1, 0, 1) + at(1, 0, -1) + at(-1, 0, -1) + at(0, 1, 1) + at(0, -1, 1) +
                      at(0, 1, -1) + at(0, -1, -1);
    return (1.0 / 3.0) * (ax - 6.0 * c) + (1.0 / 6.0) * (ed - 12.0 * c);
}

template <typename T>
__global__ void __launch_bounds__(DT)
    k_laplace(const RunDesc *__restrict__ runs, int dim, const T *phi, const T *rho,
              double *partials)
{
    const RunDesc &R = runs[blockIdx.y];
    const bool wx = R.bc[0] != ACM_BC_PERIODIC, wy = R.bc[2] != ACM_BC_PERIODIC;
    const bool wz = dim == 3 && R.bc[4] == ACM_BC_WALL;
    const double a = R.a, kappa = R.kappa;
    double v[NL] = {};
    const int nrow = R.ny * R.nz;
    for (int row = blockIdx.x; row < nrow; row += gridDim.x) {
        const int z = row / R.ny, y = row - z * R.ny;
        if ((wy && (y == 0 || y == R.ny - 1)) || (wz && (z == 0 || z == R.nz - 1))) continue;
        for (int x = threadIdx.x; x < R.nx; x += DT) {
            if (wx && (x == 0 || x == R.nx - 1)) continue;
            const long long k = sidx(R, x, y, z);
            const double p = (double)phi[k];
            const double mu = 4.0 * a * p * (p * p - 1.0) - kappa * lap_iso<T>(R, dim, phi, x, y, z);
            const double wg = 1.0 - p * p;
            v[0] += 0.5 * (1.0 + p);
            v[1] += wg;
            v[2] += mu * wg;
            if (p > 0.95) {
                v[3] += 1.0;
                v[4] += mu;
                v[5] += (double)rho[k];
            } else if (p < -0.95) {
                v[6] += 1.0;
                v[7] += mu;
                v[8] += (double)rho[k];
            }
        }
    }
    block_sum<NL>(v, partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * NL);
}

__global__ void k_laplace_final(const RunDesc *__restrict__ runs, int dim,
                                const double *partials, int blocks, double *out)
{
    const int r = blockIdx.x;
    if (threadIdx.x != 0) return;
    double s[NL] = {};
    for (int b = 0; b < blocks; ++b)
        for (int q = 0; q < NL; ++q) s[q] += partials[((long long)r * blocks + b) * NL + q];
    const RunDesc &R = runs[r];
    const double pi = 3.14159265358979323846;
    const double A = s[0];
    const double reff = dim == 2 ? sqrt(A / pi) : cbrt(3.0 * A / (4.0 * pi));
    const double sigma = sqrt(32.0 * R.a * R.kappa / 9.0);  // a = 3 sigma/(4W), kappa = 3 sigma W/8
    double *o = out + 8 * r;
    o[0] = A;
    o[1] = reff;
    o[2] = s[1] > 0.0 ? s[2] / s[1] : 0.0;
    o[3] = s[3] > 0.0 ? s[4] / s[3] : 0.0;
    o[4] = s[6] > 0.0 ? s[7] / s[6] : 0.0;
    o[5] = (s[3] > 0.0 && s[6] > 0.0) ? R.cs2 * (s[5] / s[3] - s[8] / s[6]) : 0.0;
    o[6] = reff > 0.0 ? (dim - 1) * sigma / (2.0 * reff) : 0.0;
    o[7] = s[3];
}

}  // namespace

template <typename T>
cudaError_t launch_error_l2(const RunDesc &R, const T *f, const double *ref, double *partials,
                            int blocks, double *out, cudaStream_t s)
{
    k_err<T><<<blocks, DT, 0, s>>>(R, f, ref, partials);
    k_err_final<<<1, 32, 0, s>>>(partials, blocks, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_laplace(const RunDesc *druns, int nruns, int dim, const T *phi, const T *rho,
                           double *partials, int blocks, double *out, cudaStream_t s)
{
    dim3 grid(blocks, nruns);
    k_laplace<T><<<grid, DT, 0, s>>>(druns, dim, phi, rho, partials);
    k_laplace_final<<<nruns, 32, 0, s>>>(druns, dim, partials, blocks, out);
    return cudaGetLastError();
}

template cudaError_t launch_error_l2<float>(const RunDesc &, const float *, const double *,
                                            double *, int, double *, cudaStream_t);
template cudaError_t launch_error_l2<double>(const RunDesc &, const double *, const double *,
                                             double *, int, double *, cudaStream_t);
template cudaError_t launch_laplace<float>(const RunDesc *, int, int, const float *,
                                           const float *, double *, int, double *, cudaStream_t);
template cudaError_t launch_laplace<double>(const RunDesc *, int, int, const double *,
                                            const double *, double *, int, double *,
                                            cudaStream_t);

}  // namespace acm
