// The MAMEs predictor-corrector of Huang, arXiv:2012.03525, Section 2
// (Eqs. 2.6-2.9), the scheme the simplified one-step update replaces, for
// periodic 2D grids (single grid or batch), kept as a comparison scheme.
//
//   predictor  rho*   = rho - dt d_a(rho u_a) + dt^2/2 d_a d_b Pi_ab
//              (rho u_a)* = rho u_a - dt d_b Pi_ab + nu dt Lap(rho u_a)
//                           + 2 nu dt d_a d_g (rho u_g)
//   corrector  rho^{n+1} = rho*,
//              (rho u_a)^{n+1} = (rho u_a)* + (nu/c_s^2 - dt/2) d_b (Pi*_ab - Pi_ab)
//   with Pi_ab = rho u_a u_b + p delta_ab, p = c_s^2 rho.
// Operators: centred first differences, compact second differences for
// d_aa, the centred four-point mixed difference for d_xy.
//
// One kernel per step, no intermediate fields in memory: a CTA stages its
// 32 x 32 tile of rho', u, v with a two-node halo in shared memory, forms
// m = rho u and Pi on the staged window, evaluates the predictor on the tile
// grown by one node (the corrector's differences of Pi* reach one node),
// keeps the increments Delta rho, Delta m and Pi* - Pi there, and applies
// the corrector on the tile.  Increments keep the FP32 storage accurate:
// Pi* - Pi = Delta m_a u*_b + m_a (u*_b - u_b) + c_s^2 Delta rho delta_ab,
// u^{n+1} = u + (delta m - Delta rho u) / rho*.  Pressure enters through
// c_s^2 rho' (the constant c_s^2 rho0 has no differences).
#include "acm_internal.h"

namespace acm {
namespace {

constexpr int RW1 = T2X + 2, RH1 = T2Y + 2, A1 = RW1 * RH1;
constexpr int RW2 = T2X + 4, RH2 = T2Y + 4, A2 = RW2 * RH2;
constexpr int NWARP = T2THREADS / 32;

__device__ __forceinline__ int wrap_p(int c, int n)
{
    if (c < 0) c += n;
    else if (c >= n) c -= n;
    if ((unsigned)c >= (unsigned)n) {  // grids narrower than the halo
        c %= n;
        if (c < 0) c += n;
    }
    return c;
}

// Visit a (RW x RH) window, 32 <= RW <= 64: warp w takes the first 32
// columns of rows w, w + 8, ...; the remaining RW - 32 columns of every row
// are packed into full warps as one flat list, handed out starting at the
// first warp with one row fewer.
template <int RW, int RH, typename F>
__device__ __forceinline__ void for_window(F f)
{
    static_assert(RW >= 32 && RW <= 64, "window width");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int ly = warp; ly < RH; ly += NWARP) f(ly, lane);
    if constexpr (RW > 32) {
        constexpr int TW = RW - 32, NT = RH * TW;
        const int t0 = (threadIdx.x + T2THREADS - (RH % NWARP) * 32) % T2THREADS;
        for (int t = t0; t < NT; t += T2THREADS) {
            const int ly = t / TW;
            f(ly, 32 + (t - ly * TW));
        }
    }
}

// shared-memory windows: staged fields and fluxes on the halo-2 window (A2),
// increments on the halo-1 window (A1)
enum { W_R, W_U, W_V, W_MX, W_MY, W_PXX, W_PXY, W_PYY, NW2 };
enum { I_DR, I_DMX, I_DMY, I_QXX, I_QXY, I_QYY, NI1 };

template <typename T>
__global__ void __launch_bounds__(T2THREADS)
    k_mames2d(const RunDesc *__restrict__ runs, const int4 *__restrict__ work, int nwork,
              Fields<T> in, Fields<T> out, unsigned *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S2 = reinterpret_cast<T *>(smem_raw);  // NW2 windows of A2
    T *S1 = S2 + NW2 * A2;                      // NI1 windows of A1
    const int lane = threadIdx.x & 31;
    bool nonfinite = false;

    for (int item = blockIdx.x; item < nwork; item += gridDim.x) {
        const int4 wk = work[item];
        const RunDesc &R = runs[wk.x];
        const int nx = R.nx, ny = R.ny;
        const int x0 = wk.y, y0 = wk.z;
        const T *C = coefs<T>(R);
        const T rho0 = C[C_RHO0], dt = C[C_DT], cs2 = C[C_CS2], nu = C[C_NU];
        const T nudt = C[C_NUDT];
        const T hdt2 = T(0.5) * dt * dt, cc = nu / cs2 - T(0.5) * dt;
        const long long off = R.off;
        const T *gr = in.f[F_R] + off, *gu = in.f[F_U] + off, *gv = in.f[F_V] + off;

        __syncthreads();  // shared memory of the previous item is free
        {
            const int ca = wrap_p(x0 - 2 + lane, nx);
            for_window<RW2, RH2>([&](int ly, int lx) {
                const long long k = (long long)wrap_p(y0 - 2 + ly, ny) * nx +
                                    (lx < 32 ? ca : wrap_p(x0 - 2 + lx, nx));
                const int i = ly * RW2 + lx;
                const T r = gr[k], u = gu[k], v = gv[k];
                const T mx = (rho0 + r) * u, my = (rho0 + r) * v;
                S2[W_R * A2 + i] = r;
                S2[W_U * A2 + i] = u;
                S2[W_V * A2 + i] = v;
                S2[W_MX * A2 + i] = mx;
                S2[W_MY * A2 + i] = my;
                S2[W_PXX * A2 + i] = mx * u + cs2 * r;
                S2[W_PXY * A2 + i] = mx * v;
                S2[W_PYY * A2 + i] = my * v + cs2 * r;
            });
        }
        __syncthreads();

        // predictor (Eqs. 2.6-2.7) on the tile grown by one node
        const T *sr = S2 + W_R * A2, *su = S2 + W_U * A2, *sv = S2 + W_V * A2;
        const T *smx = S2 + W_MX * A2, *smy = S2 + W_MY * A2;
        const T *pxx = S2 + W_PXX * A2, *pxy = S2 + W_PXY * A2, *pyy = S2 + W_PYY * A2;
        for_window<RW1, RH1>([&](int ly, int lx) {
            const int c = (ly + 1) * RW2 + (lx + 1);
            const int E = c + 1, W = c - 1, N = c + RW2, S = c - RW2;
            const int NE = N + 1, NW = N - 1, SE = S + 1, SW = S - 1;
            auto dxx = [&](const T *f) { return (f[E] + f[W]) - T(2) * f[c]; };
            auto dyy = [&](const T *f) { return (f[N] + f[S]) - T(2) * f[c]; };
            auto dxy = [&](const T *f) { return T(0.25) * ((f[NE] - f[SE]) - (f[NW] - f[SW])); };
            const T div_m = T(0.5) * (smx[E] - smx[W]) + T(0.5) * (smy[N] - smy[S]);
            const T ddpi = dxx(pxx) + T(2) * dxy(pxy) + dyy(pyy);
            const T dr = -dt * div_m + hdt2 * ddpi;
            const T lmx = dxx(smx) + dyy(smx), lmy = dxx(smy) + dyy(smy);
            const T fx = T(0.5) * (pxx[E] - pxx[W]) + T(0.5) * (pxy[N] - pxy[S]);
            const T fy = T(0.5) * (pxy[E] - pxy[W]) + T(0.5) * (pyy[N] - pyy[S]);
            const T gdx = dxx(smx) + dxy(smy), gdy = dxy(smx) + dyy(smy);
            const T dmx = -dt * fx + nudt * lmx + T(2) * nudt * gdx;
            const T dmy = -dt * fy + nudt * lmy + T(2) * nudt * gdy;
            // Pi* - Pi at this node
            const T rs = rho0 + sr[c] + dr;
            const T inv = T(1) / rs;
            const T u = su[c], v = sv[c];
            const T mx = smx[c], my = smy[c];
            const T usx = (mx + dmx) * inv, usy = (my + dmy) * inv;
            const T dux = (dmx - dr * u) * inv, duy = (dmy - dr * v) * inv;
            const int i = ly * RW1 + lx;
            S1[I_DR * A1 + i] = dr;
            S1[I_DMX * A1 + i] = dmx;
            S1[I_DMY * A1 + i] = dmy;
            S1[I_QXX * A1 + i] = dmx * usx + mx * dux + cs2 * dr;
            S1[I_QXY * A1 + i] = dmx * usy + mx * duy;
            S1[I_QYY * A1 + i] = dmy * usy + my * duy + cs2 * dr;
        });
        __syncthreads();

        // corrector (Eqs. 2.8-2.9) on the tile
        const T *qxx = S1 + I_QXX * A1, *qxy = S1 + I_QXY * A1, *qyy = S1 + I_QYY * A1;
        for_window<T2X, T2Y>([&](int ly, int lx) {
            const int gx = x0 + lx, gy = y0 + ly;
            if (gx >= nx || gy >= ny) return;
            const int c1 = (ly + 1) * RW1 + (lx + 1);
            const int c2 = (ly + 2) * RW2 + (lx + 2);
            const T dr = S1[I_DR * A1 + c1];
            const T cx = T(0.5) * (qxx[c1 + 1] - qxx[c1 - 1]) + T(0.5) * (qxy[c1 + RW1] - qxy[c1 - RW1]);
            const T cy = T(0.5) * (qxy[c1 + 1] - qxy[c1 - 1]) + T(0.5) * (qyy[c1 + RW1] - qyy[c1 - RW1]);
            const T dmx = S1[I_DMX * A1 + c1] + cc * cx;
            const T dmy = S1[I_DMY * A1 + c1] + cc * cy;
            const T r = sr[c2], u = su[c2], v = sv[c2];
            const T inv = T(1) / (rho0 + r + dr);
            const T rn = r + dr;
            const T un = u + (dmx - dr * u) * inv;
            const T vn = v + (dmy - dr * v) * inv;
            const long long gi = off + (long long)gy * nx + gx;
            out.f[F_R][gi] = rn;
            out.f[F_U][gi] = un;
            out.f[F_V][gi] = vn;
            nonfinite |= !isfinite(rn + un + vn);
        });
    }
    if (nonfinite) atomicOr(err, ERR_NONFINITE);
}

template <typename T>
size_t smem_bytes()
{
    return (size_t)(NW2 * A2 + NI1 * A1) * sizeof(T);
}

template <typename T>
int max_blocks()
{
    static int cached = -1;
    if (cached < 0) {
        cudaFuncSetAttribute(k_mames2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<T>());
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mames2d<T>, T2THREADS,
                                                          smem_bytes<T>()) != cudaSuccess)
            nb = 1;
        cached = nb > 0 ? nb : 1;
    }
    return cached;
}

}  // namespace

template <typename T>
int mames2d_max_blocks_per_sm()
{
    return max_blocks<T>();
}

template <typename T>
cudaError_t launch_mames2d(const RunDesc *druns, const int4 *dwork, int nwork, Fields<T> in,
                           Fields<T> out, unsigned *derr, int blocks, cudaStream_t s)
{
    if (nwork <= 0) return cudaSuccess;
    if (blocks > nwork) blocks = nwork;
    max_blocks<T>();
    k_mames2d<T><<<blocks, T2THREADS, smem_bytes<T>(), s>>>(druns, dwork, nwork, in, out, derr);
    return cudaGetLastError();
}

template cudaError_t launch_mames2d<float>(const RunDesc *, const int4 *, int, Fields<float>,
                                           Fields<float>, unsigned *, int, cudaStream_t);
template cudaError_t launch_mames2d<double>(const RunDesc *, const int4 *, int, Fields<double>,
                                            Fields<double>, unsigned *, int, cudaStream_t);
template int mames2d_max_blocks_per_sm<float>();
template int mames2d_max_blocks_per_sm<double>();

}  // namespace acm
