// FP64 integral diagnostics and host<->storage conversion kernels.
//
// Diagnostics (Section 3 of Huang, arXiv:2012.03525: kinetic energy of the
// Taylor-Green test, the steady-state criterion max |  |u|^{n+1} - |u|^n  |
// of the cavity test) are accumulated in FP64 for both storage precisions.
// Deterministic two-pass reduction: pass 1 gives every (run, block) a fixed
// strided slice of the nodes and reduces it in a fixed tree; pass 2 sums the
// block partials of each run in block order.  The result does not depend on
// scheduling.
#include "acm_internal.h"

namespace acm {
namespace {

constexpr int RT = 256;  // reduction threads per block

__device__ __forceinline__ long long storage_index(const RunDesc &R, int dim, long long i)
{
    if (dim == 2) return R.off + i;
    const long long nxy = (long long)R.nx * R.ny;
    const long long z = i / nxy;
    const long long rem = i - z * nxy;
    const long long y = rem / R.nx;
    const long long x = rem - y * R.nx;
    return R.off + ((z + R.zg) * R.py + y + R.pad) * R.px + x + R.pad;
}

// Pass 1 walks rows of contiguous nodes: in 3D the x-rows of the padded
// storage (row = (z, y), one 32-bit division per row), in 2D chunks of
// RCHUNK consecutive nodes of the unpadded run.  Blocks take rows
// blockIdx.x, blockIdx.x + gridDim.x, ...; threads stride along the row.
constexpr int RCHUNK = 4 * RT;

template <typename F>
__device__ __forceinline__ void for_rows(const RunDesc &R, int dim, F &&node)
{
    const long long n2 = (long long)R.nx * R.ny;
    const int nrow = dim == 3 ? R.ny * R.nz : (int)((n2 + RCHUNK - 1) / RCHUNK);
    for (int row = blockIdx.x; row < nrow; row += gridDim.x) {
        long long base;
        int len;
        if (dim == 3) {
            const int z = row / R.ny, y = row - z * R.ny;
            base = R.off + ((long long)(z + R.zg) * R.py + y + R.pad) * R.px + R.pad;
            len = R.nx;
        } else {
            base = R.off + (long long)row * RCHUNK;
            len = (int)min((long long)RCHUNK, n2 - (long long)row * RCHUNK);
        }
        for (int x = threadIdx.x; x < len; x += RT) node(base + x);
    }
}

// Compensated FP32 sum (a "double-float" accumulator: s + c carries ~48
// significant bits): Knuth's two-sum of s and x, the rounding error of the
// addition goes into c.  Explicit round-to-nearest intrinsics keep the
// compiler from reassociating or contracting it.
struct CSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        c = __fadd_rn(c, err);
        s = t;
    }
    // add the exact product a * b (the product's rounding error from an FMA)
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        c = __fadd_rn(c, __fmaf_rn(a, b, -p));
        add(p);
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// FP64 diagnostics of FP64 storage: every operation in FP64 (the parity
// path).  max |u| is taken over |u|^2 and square-rooted once per thread.
__device__ __forceinline__ void reduce_node(const RunDesc &R, int dim, const double *fr,
                                            const double *fu, const double *fv, const double *fw,
                                            const double *pu, const double *pv, const double *pw,
                                            long long k, double (&s)[5], double &mdu, double &mq,
                                            double &nbad)
{
    const double r = fr[k], u = fu[k], v = fv[k];
    const double w = dim == 3 ? fw[k] : 0.0;
    const double rho = R.rho0 + r;
    s[0] += r;
    s[1] += rho * u;
    s[2] += rho * v;
    s[3] += rho * w;
    const double q = u * u + v * v + w * w;
    s[4] += q;
    mq = fmax(mq, q);
    if (pu) {
        const double a = pu[k], b = pv[k], c = dim == 3 ? pw[k] : 0.0;
        mdu = fmax(mdu, fabs(sqrt(q) - sqrt(a * a + b * b + c * c)));
    }
    nbad += (!isfinite(r) || !isfinite(u) || !isfinite(v) || !isfinite(w)) ? 1.0 : 0.0;
}

template <typename T>
__global__ void __launch_bounds__(RT)
    k_reduce(const RunDesc *__restrict__ runs, int dim, Fields<T> cur, const T *pu, const T *pv,
             const T *pw, double *partials)
{
    const RunDesc &R = runs[blockIdx.y];
    const T *fr = cur.f[F_R], *fu = cur.f[F_U], *fv = cur.f[F_V], *fw = cur.f[F_W];
    double vals[8];
    if constexpr (sizeof(T) == 8) {
        double s[5] = {0, 0, 0, 0, 0};
        double mdu = 0.0, mq = 0.0, nbad = 0.0;
        for_rows(R, dim, [&](long long k) {
            reduce_node(R, dim, fr, fu, fv, fw, pu, pv, pw, k, s, mdu, mq, nbad);
        });
        const double v8[8] = {s[0], s[1], s[2], s[3], 0.5 * s[4], mdu, sqrt(mq), nbad};
        for (int q = 0; q < 8; ++q) vals[q] = v8[q];
    } else {
        // FP32 storage: per node only FP32 arithmetic (the FP64 pipe of GB300
        // is narrow).  Sums are compensated; sum rho u_a = rho0 sum u_a +
        // sum rho' u_a with the products rho' u_a added exactly; |u|^2 and
        // the steady-state criterion | |u| - |u_prev| | =
        // |sum_a (u_a - p_a)(u_a + p_a)| / (|u| + |u_prev|) in FP32 (relative
        // error ~1e-7 of the value); max |u| from the argmax node's FP32
        // components, squared and rooted in FP64.
        CSum sr, su, sv, sw, sru, srv, srw, sq;
        float mq = -1.f, mdu = 0.f, qu = 0.f, qv = 0.f, qw = 0.f;
        int nbad = 0;
        for_rows(R, dim, [&](long long k) {
            const float r = fr[k], u = fu[k], v = fv[k];
            const float w = dim == 3 ? fw[k] : 0.f;
            sr.add(r);
            su.add(u);
            sv.add(v);
            sw.add(w);
            sru.add_prod(r, u);
            srv.add_prod(r, v);
            srw.add_prod(r, w);
            const float q = __fmaf_rn(u, u, __fmaf_rn(v, v, __fmul_rn(w, w)));
            sq.add(q);
            if (q > mq) {
                mq = q;
                qu = u;
                qv = v;
                qw = w;
            }
            if (pu) {
                const float a = pu[k], b = pv[k], c = dim == 3 ? pw[k] : 0.f;
                const float dq = __fmaf_rn(__fsub_rn(u, a), __fadd_rn(u, a),
                                           __fmaf_rn(__fsub_rn(v, b), __fadd_rn(v, b),
                                                     __fmul_rn(__fsub_rn(w, c), __fadd_rn(w, c))));
                const float qp = __fmaf_rn(a, a, __fmaf_rn(b, b, __fmul_rn(c, c)));
                const float mag = __fadd_rn(sqrtf(q), sqrtf(qp));
                if (mag > 0.f) mdu = fmaxf(mdu, fabsf(dq) / mag);
            }
            nbad += (!isfinite(r) || !isfinite(u) || !isfinite(v) || !isfinite(w)) ? 1 : 0;
        });
        const double rho0 = R.rho0;
        const double qd = (double)qu * qu + (double)qv * qv + (double)qw * qw;
        vals[0] = sr.value();
        vals[1] = rho0 * su.value() + sru.value();
        vals[2] = rho0 * sv.value() + srv.value();
        vals[3] = rho0 * sw.value() + srw.value();
        vals[4] = 0.5 * sq.value();
        vals[5] = (double)mdu;
        vals[6] = mq >= 0.f ? sqrt(qd) : 0.0;
        vals[7] = (double)nbad;
    }
    __shared__ double red[8][RT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double x = vals[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            x = (q == 5 || q == 6) ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int q = threadIdx.x;
        double x = red[q][0];
        for (int k = 1; k < RT / 32; ++k) x = (q == 5 || q == 6) ? fmax(x, red[q][k]) : x + red[q][k];
        partials[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 8 + q] = x;
    }
}

__global__ void k_reduce_final(const RunDesc *__restrict__ runs, const double *partials,
                               int blocks_per_run, double *out)
{
    const int r = blockIdx.x;
    const int q = threadIdx.x;
    if (q >= 8) return;
    double x = partials[(long long)r * blocks_per_run * 8 + q];
    for (int b = 1; b < blocks_per_run; ++b) {
        const double y = partials[((long long)r * blocks_per_run + b) * 8 + q];
        x = (q == 5 || q == 6) ? fmax(x, y) : x + y;
    }
    if (q == 0) {
        const RunDesc &R = runs[r];
        x += (double)R.nx * R.ny * R.nz * R.rho0;
    }
    out[r * 8 + q] = x;
}

// host FP64 staging (unpadded, [z][y][x]) -> storage (shifted, padded in 3D,
// ghost layers filled with the periodic images)
template <typename T>
__global__ void k_import(const double *__restrict__ src, T *__restrict__ dst, RunDesc R, int dim,
                         double shift)
{
    if (dim == 2) {
        const long long n = (long long)R.nx * R.ny;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x)
            dst[R.off + i] = (T)(src[i] - shift);
        return;
    }
    const long long n = R.px * R.py * R.nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long z = i / (R.px * R.py);
        const long long rem = i - z * R.px * R.py;
        long long y = rem / R.px - R.pad;
        long long x = rem % R.px - R.pad;
        y = ((y % R.ny) + R.ny) % R.ny;
        x = ((x % R.nx) + R.nx) % R.nx;
        dst[R.off + R.zg * R.px * R.py + i] = (T)(src[(z * R.ny + y) * R.nx + x] - shift);
    }
}

template <typename T>
__global__ void k_export(const T *__restrict__ src, double *__restrict__ dst, RunDesc R, int dim,
                         double shift)
{
    const long long n = (long long)R.nx * R.ny * R.nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[storage_index(R, dim, i)] + shift;
}

}  // namespace

template <typename T>
cudaError_t launch_reduce(const RunDesc *druns, int nruns, int dim, Fields<T> cur, const T *pu,
                          const T *pv, const T *pw, double *dpartials, int blocks_per_run,
                          double *dout, cudaStream_t s)
{
    dim3 grid(blocks_per_run, nruns);
    k_reduce<T><<<grid, RT, 0, s>>>(druns, dim, cur, pu, pv, pw, dpartials);
    k_reduce_final<<<nruns, 32, 0, s>>>(druns, dpartials, blocks_per_run, dout);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_import(const double *src, T *dst, const RunDesc &run, int dim, double shift,
                          cudaStream_t s)
{
    k_import<T><<<1024, 256, 0, s>>>(src, dst, run, dim, shift);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export(const T *src, double *dst, const RunDesc &run, int dim, double shift,
                          cudaStream_t s)
{
    k_export<T><<<1024, 256, 0, s>>>(src, dst, run, dim, shift);
    return cudaGetLastError();
}

template cudaError_t launch_reduce<float>(const RunDesc *, int, int, Fields<float>, const float *,
                                          const float *, const float *, double *, int, double *,
                                          cudaStream_t);
template cudaError_t launch_reduce<double>(const RunDesc *, int, int, Fields<double>,
                                           const double *, const double *, const double *,
                                           double *, int, double *, cudaStream_t);
template cudaError_t launch_import<float>(const double *, float *, const RunDesc &, int, double,
                                          cudaStream_t);
template cudaError_t launch_import<double>(const double *, double *, const RunDesc &, int, double,
                                           cudaStream_t);
template cudaError_t launch_export<float>(const float *, double *, const RunDesc &, int, double,
                                          cudaStream_t);
template cudaError_t launch_export<double>(const double *, double *, const RunDesc &, int, double,
                                           cudaStream_t);

}  // namespace acm
