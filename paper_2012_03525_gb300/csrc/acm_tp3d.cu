// 3D two-phase step (Huang, arXiv:2012.03525, Section 2: Eqs. 2.10-2.11
// with the surface-tension force F_ST = -phi grad mu and the Cahn-Hilliard
// update of Eq. 2.14 by Heun's RK2, u^n frozen), with the D3Q19-weighted
// isotropic gradient and Laplacian (c_s^2 = 1/3: axis weight 1/18, edge
// weight 1/36).  x and y are periodic; z is periodic or bounded by
// stationary walls carrying the wetting condition
// d_n phi = -(2/W) cos(theta) (1 - phi_w^2) and d_n mu = 0 (ghost node one
// beyond the wall = mirror of the node one inside, plus 2 (2/W) cos(theta)
// (1 - phi_w^2) for phi).
//
// Five launches per step, one thread per node (3D launch grid, x fastest,
// coalesced; the 19-point neighbourhoods come through L1/L2):
//   1. mu^n from phi^n;
//   2. Delta rho = rho^{n+1} - rho^n (Eq. 2.10; wall nodes take the
//      second-order zero-normal-gradient extrapolation of rho^{n+1});
//   3. rho^{n+1}, u^{n+1} (Eq. 2.11 + F_ST + body force; wall nodes at rest)
//      and the first Heun stage phi* = phi + dt R(phi, mu);
//   4. mu* from phi*;
//   5. phi^{n+1} = (phi + phi* + dt R(phi*, mu*)) / 2,
// with R(f, m) = -u^n . grad f + M Lap m.  Scratch fields: mu, phi*,
// Delta rho.  Storage is the padded 3D layout of the single-phase step
// (periodic images are not needed: every index wraps explicitly).
#include "acm_internal.h"

namespace acm {
namespace {

constexpr int TPB = 256;

// D3Q19 velocities without the rest one: 6 axis, 12 edges.  A compile-time
// table: in the unrolled loops below every offset folds to a constant.
__host__ __device__ constexpr int vel(int i, int d)
{
    constexpr int8_t t[18][3] = {
        {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
        {1, 1, 0},  {1, -1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, 0, 1},  {1, 0, -1},
        {-1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, 1, -1},  {0, -1, 1}, {0, -1, -1}};
    return t[i][d];
}

struct Geo3 {
    int nx, ny, nz;
    bool zwall;
    long long base, px, pxy;  // storage index of (x, y, z) = base + z pxy + y px + x
    __device__ Geo3(const RunDesc &R)
        : nx(R.nx), ny(R.ny), nz(R.nz), zwall(R.bc[4] != ACM_BC_PERIODIC),
          base(R.off + (long long)R.pad * R.px + R.pad), px(R.px), pxy(R.px * R.py)
    {
    }
    __device__ __forceinline__ int wx(int x) const { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }
    __device__ __forceinline__ int wy(int y) const { return y < 0 ? y + ny : (y >= ny ? y - ny : y); }
    __device__ __forceinline__ int wz(int z) const { return z < 0 ? z + nz : (z >= nz ? z - nz : z); }
    // a node in the grid (x, y wrap; z wraps when periodic, else in range)
    __device__ __forceinline__ long long at(int x, int y, int z) const
    {
        return base + (long long)(zwall ? z : wz(z)) * pxy + (long long)wy(y) * px + wx(x);
    }
    __device__ __forceinline__ bool wall(int z) const { return zwall && (z == 0 || z == nz - 1); }
};

enum { K_MIRROR = 0, K_WET = 1 };

// Storage offsets of a node's 3 x 3 x 3 neighbourhood: x and y wrap; z wraps
// when periodic, and beyond a wall face points at the mirror plane (ghost
// node = node one inside the wall), with the wall plane kept for the
// wetting term.
struct Hood {
    long long xo[3], yo[3], zo[3], zw[3];
    bool ghost[3];
    __device__ __forceinline__ Hood(const Geo3 &g, int x, int y, int z)
    {
        xo[0] = g.wx(x - 1);
        xo[1] = x;
        xo[2] = g.wx(x + 1);
        yo[0] = (long long)g.wy(y - 1) * g.px;
        yo[1] = (long long)y * g.px;
        yo[2] = (long long)g.wy(y + 1) * g.px;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int zz = z + k - 1, wall = zz;
            ghost[k] = false;
            if (g.zwall) {
                if (zz < 0) {
                    zz = 1;
                    wall = 0;
                    ghost[k] = true;
                } else if (zz >= g.nz) {
                    zz = g.nz - 2;
                    wall = g.nz - 1;
                    ghost[k] = true;
                }
            } else {
                zz = g.wz(zz);
                wall = zz;
            }
            zo[k] = g.base + (long long)zz * g.pxy;
            zw[k] = g.base + (long long)wall * g.pxy;
        }
    }
};

// D3Q19 isotropic Laplacian (2/c_s^2) sum w_i (f_i - f_0) and gradient
// (1/c_s^2) sum w_i e_i f_i at a node; ghost nodes beyond a wall take the
// mirror value, plus (KIND == K_WET) the wetting term wet (1 - f_w^2) with
// f_w the wall node below/above them
template <typename T, int KIND>
__device__ __forceinline__ void iso_ops(const T *f, const Hood &h, T wet, T f0, T &lap, T &gx,
                                        T &gy, T &gz)
{
    T la = T(0), le = T(0), ax = T(0), ay = T(0), az = T(0), ex = T(0), ey = T(0), ez = T(0);
#pragma unroll
    for (int i = 0; i < 18; ++i) {
        const int dx = vel(i, 0), dy = vel(i, 1), dz = vel(i, 2);
        const long long xy = h.yo[dy + 1] + h.xo[dx + 1];
        T fi = f[h.zo[dz + 1] + xy];
        if (KIND == K_WET && dz != 0 && h.ghost[dz + 1]) {
            const T fw = f[h.zw[dz + 1] + xy];
            fi += wet * (T(1) - fw * fw);
        }
        if (i < 6) {
            la += fi - f0;
            ax += dx * fi;
            ay += dy * fi;
            az += dz * fi;
        } else {
            le += fi - f0;
            ex += dx * fi;
            ey += dy * fi;
            ez += dz * fi;
        }
    }
    lap = T(1.0 / 3.0) * la + T(1.0 / 6.0) * le;
    gx = T(1.0 / 6.0) * ax + T(1.0 / 12.0) * ex;
    gy = T(1.0 / 6.0) * ay + T(1.0 / 12.0) * ey;
    gz = T(1.0 / 6.0) * az + T(1.0 / 12.0) * ez;
}

// 1, 4: mu = 4 a phi (phi^2 - 1) - kappa Lap_iso(phi)
template <typename T>
__global__ void __launch_bounds__(TPB) k_mu(const RunDesc R, const T *__restrict__ phi,
                                            T *__restrict__ mu)
{
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T a = C[C_A], kappa = C[C_KAPPA], wet = C[C_WET];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x < g.nx && y < g.ny && z < g.nz) do {  // one node per thread
        const Hood h(g, x, y, z);
        const long long c = h.zo[1] + h.yo[1] + h.xo[1];
        const T f = phi[c];
        T lap, gx, gy, gz;
        iso_ops<T, K_WET>(phi, h, wet, f, lap, gx, gy, gz);
        mu[c] = T(4) * a * f * (f * f - T(1)) - kappa * lap;
    } while (0);
}

// Eq. (2.10) at a non-wall node: Delta rho = -dt div(rho u) + satc Lap(rho')
template <typename T>
__device__ __forceinline__ T drho_at(const Fields<T> &in, const Geo3 &g, int x, int y, int z,
                                     T rho0, T dt, T satc)
{
    const T *r = in.f[F_R], *u = in.f[F_U], *v = in.f[F_V], *w = in.f[F_W];
    const long long c = g.at(x, y, z);
    const long long xe = g.at(x + 1, y, z), xw = g.at(x - 1, y, z);
    const long long yn = g.at(x, y + 1, z), ys = g.at(x, y - 1, z);
    const long long zu = g.at(x, y, z + 1), zd = g.at(x, y, z - 1);
    const T div = T(0.5) * ((rho0 + r[xe]) * u[xe] - (rho0 + r[xw]) * u[xw]) +
                  T(0.5) * ((rho0 + r[yn]) * v[yn] - (rho0 + r[ys]) * v[ys]) +
                  T(0.5) * ((rho0 + r[zu]) * w[zu] - (rho0 + r[zd]) * w[zd]);
    const T lap = (r[xe] + r[xw]) + (r[yn] + r[ys]) + (r[zu] + r[zd]) - T(6) * r[c];
    return -dt * div + satc * lap;
}

// 2: Delta rho everywhere (wall nodes: (4 rho_1 - rho_2)/3 of rho^{n+1})
template <typename T>
__global__ void __launch_bounds__(TPB) k_drho(const RunDesc R, Fields<T> in, T *__restrict__ dr)
{
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T rho0 = C[C_RHO0], dt = C[C_DT], satc = C[C_SATC];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x < g.nx && y < g.ny && z < g.nz) do {  // one node per thread
        const long long c = g.at(x, y, z);
        if (!g.wall(z)) {
            dr[c] = drho_at(in, g, x, y, z, rho0, dt, satc);
            continue;
        }
        const int s = z == 0 ? 1 : -1;
        const T *r = in.f[F_R];
        const T r1 = r[g.at(x, y, z + s)] + drho_at(in, g, x, y, z + s, rho0, dt, satc);
        const T r2 = r[g.at(x, y, z + 2 * s)] + drho_at(in, g, x, y, z + 2 * s, rho0, dt, satc);
        dr[c] = (T(4) * r1 - r2) / T(3) - r[c];
    } while (0);
}

// 3: rho^{n+1}, u^{n+1} and phi*
template <typename T>
__global__ void __launch_bounds__(TPB)
    k_main(const RunDesc R, Fields<T> in, Fields<T> out, const T *__restrict__ dr,
           const T *__restrict__ mu, T *__restrict__ phs, unsigned *err)
{
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T rho0 = C[C_RHO0], dt = C[C_DT], cs2 = C[C_CS2], nudt = C[C_NUDT];
    const T satm = C[C_SATM], mob = C[C_M], wet = C[C_WET];
    const T gfx = C[C_GX], gfy = C[C_GY], gfz = C[C_GZ];
    const T *r = in.f[F_R], *u = in.f[F_U], *v = in.f[F_V], *w = in.f[F_W], *ph = in.f[F_PHI];
    bool bad = false;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x < g.nx && y < g.ny && z < g.nz) do {  // one node per thread
        const Hood h(g, x, y, z);
        const long long c = h.zo[1] + h.yo[1] + h.xo[1];
        const T r0 = r[c], d0 = dr[c];
        const T rho1 = rho0 + r0 + d0;
        const T u0 = u[c], v0 = v[c], w0 = w[c], f0 = ph[c];
        // mu^n: Laplacian for the CHE and gradient for F_ST
        T lmu, gmx, gmy, gmz;
        iso_ops<T, K_MIRROR>(mu, h, T(0), mu[c], lmu, gmx, gmy, gmz);
        T un = T(0), vn = T(0), wn = T(0);
        if (!g.wall(z)) {
            const long long nb[6] = {h.zo[1] + h.yo[1] + h.xo[2], h.zo[1] + h.yo[1] + h.xo[0],
                                     h.zo[1] + h.yo[2] + h.xo[1], h.zo[1] + h.yo[0] + h.xo[1],
                                     h.zo[2] + h.yo[1] + h.xo[1], h.zo[0] + h.yo[1] + h.xo[1]};
            T q[6], mx[6], my[6], mz[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                q[k] = rho0 + r[nb[k]];
                mx[k] = q[k] * u[nb[k]];
                my[k] = q[k] * v[nb[k]];
                mz[k] = q[k] * w[nb[k]];
            }
            const T q0 = rho0 + r0;
            const T mx0 = q0 * u0, my0 = q0 * v0, mz0 = q0 * w0;
            auto flux = [&](const T (&m)[6]) {
                return T(0.5) * ((m[0] * u[nb[0]] - m[1] * u[nb[1]]) +
                                 (m[2] * v[nb[2]] - m[3] * v[nb[3]]) +
                                 (m[4] * w[nb[4]] - m[5] * w[nb[5]]));
            };
            auto lap = [&](const T (&m)[6], T m0) {
                return ((m[0] + m[1]) + (m[2] + m[3])) + (m[4] + m[5]) - T(6) * m0;
            };
            const T ddx = T(0.5) * (dr[nb[0]] - dr[nb[1]]);
            const T ddy = T(0.5) * (dr[nb[2]] - dr[nb[3]]);
            const T ddz = T(0.5) * (dr[nb[4]] - dr[nb[5]]);
            const T fb = dt * rho1;
            T rx = -dt * flux(mx) - dt * cs2 * T(0.5) * (r[nb[0]] - r[nb[1]]) + nudt * lap(mx, mx0) -
                   satm * ddx + fb * gfx - dt * f0 * gmx;
            T ry = -dt * flux(my) - dt * cs2 * T(0.5) * (r[nb[2]] - r[nb[3]]) + nudt * lap(my, my0) -
                   satm * ddy + fb * gfy - dt * f0 * gmy;
            T rz = -dt * flux(mz) - dt * cs2 * T(0.5) * (r[nb[4]] - r[nb[5]]) + nudt * lap(mz, mz0) -
                   satm * ddz + fb * gfz - dt * f0 * gmz;
            const T inv = T(1) / rho1;
            un = u0 + (rx - d0 * u0) * inv;
            vn = v0 + (ry - d0 * v0) * inv;
            wn = w0 + (rz - d0 * w0) * inv;
        }
        // first Heun stage of Eq. (2.14), u^n frozen
        T lph, gpx, gpy, gpz;
        iso_ops<T, K_WET>(ph, h, wet, f0, lph, gpx, gpy, gpz);
        const T fs = f0 + dt * (-(u0 * gpx + v0 * gpy + w0 * gpz) + mob * lmu);
        const T rn = r0 + d0;
        out.f[F_R][c] = rn;
        out.f[F_U][c] = un;
        out.f[F_V][c] = vn;
        out.f[F_W][c] = wn;
        phs[c] = fs;
        bad |= !isfinite(rn + un + vn + wn + fs);
    } while (0);
    if (bad) atomicOr(err, ERR_NONFINITE);
}

// 5: phi^{n+1}
template <typename T>
__global__ void __launch_bounds__(TPB)
    k_phi(const RunDesc R, Fields<T> in, const T *__restrict__ phs, const T *__restrict__ mus,
          T *__restrict__ phn, unsigned *err)
{
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T dt = C[C_DT], mob = C[C_M], wet = C[C_WET];
    const T *u = in.f[F_U], *v = in.f[F_V], *w = in.f[F_W], *ph = in.f[F_PHI];
    bool bad = false;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x < g.nx && y < g.ny && z < g.nz) do {  // one node per thread
        const Hood h(g, x, y, z);
        const long long c = h.zo[1] + h.yo[1] + h.xo[1];
        T lmu, a0, a1, a2, lph, gpx, gpy, gpz;
        iso_ops<T, K_MIRROR>(mus, h, T(0), mus[c], lmu, a0, a1, a2);
        iso_ops<T, K_WET>(phs, h, wet, phs[c], lph, gpx, gpy, gpz);
        const T r2 = -(u[c] * gpx + v[c] * gpy + w[c] * gpz) + mob * lmu;
        const T f = T(0.5) * (ph[c] + phs[c] + dt * r2);
        phn[c] = f;
        bad |= !isfinite(f);
    } while (0);
    if (bad) atomicOr(err, ERR_NONFINITE);
}

}  // namespace

template <typename T>
cudaError_t launch_tp3d(const RunDesc &R, Fields<T> in, Fields<T> out, T *mu, T *phs, T *dr,
                        unsigned *err, int sms, cudaStream_t s)
{
    (void)sms;
    // one thread per node: 32 x 4 x 2 blocks (x fastest, coalesced rows)
    const dim3 blk(32, 4, 2);
    const dim3 grid((R.nx + 31) / 32, (R.ny + 3) / 4, (R.nz + 1) / 2);
    k_mu<T><<<grid, blk, 0, s>>>(R, in.f[F_PHI], mu);
    k_drho<T><<<grid, blk, 0, s>>>(R, in, dr);
    k_main<T><<<grid, blk, 0, s>>>(R, in, out, dr, mu, phs, err);
    k_mu<T><<<grid, blk, 0, s>>>(R, phs, mu);
    k_phi<T><<<grid, blk, 0, s>>>(R, in, phs, mu, out.f[F_PHI], err);
    return cudaGetLastError();
}

template cudaError_t launch_tp3d<float>(const RunDesc &, Fields<float>, Fields<float>, float *,
                                        float *, float *, unsigned *, int, cudaStream_t);
template cudaError_t launch_tp3d<double>(const RunDesc &, Fields<double>, Fields<double>,
                                         double *, double *, double *, unsigned *, int,
                                         cudaStream_t);

}  // namespace acm
