// 3D two-phase step (Huang, arXiv:2012.03525, Section 2: Eqs. 2.10-2.11
// with the surface-tension force F_ST = -phi grad mu and the Cahn-Hilliard
// update of Eq. 2.14 by Heun's RK2, u^n frozen), with the D3Q19-weighted
// isotropic gradient and Laplacian (c_s^2 = 1/3: axis weight 1/18, edge
// weight 1/36).  x and y are periodic or symmetry (mirror) planes through
// the first and last node (the quarter domains of Sections 3.6-3.7: a node
// beyond the plane is the image of the node one inside, scalars and the
// tangential velocity even, the normal velocity odd and zero on the plane);
// z is periodic or bounded by stationary walls carrying the wetting condition
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
    bool zwall, mx, my;       // z walls; symmetry planes on the x / y faces
    long long base, px, pxy;  // storage index of (x, y, z) = base + z pxy + y px + x
    __device__ Geo3(const RunDesc &R)
        : nx(R.nx), ny(R.ny), nz(R.nz), zwall(R.bc[4] != ACM_BC_PERIODIC),
          mx(R.bc[0] == ACM_BC_SYMMETRY), my(R.bc[2] == ACM_BC_SYMMETRY),
          base(R.off + (long long)R.pad * R.px + R.pad), px(R.px), pxy(R.px * R.py)
    {
    }
    // periodic wrap, or the mirror image across a symmetry plane
    __device__ __forceinline__ int wx(int x) const
    {
        if (mx) return x < 0 ? -x : (x >= nx ? 2 * (nx - 1) - x : x);
        return x < 0 ? x + nx : (x >= nx ? x - nx : x);
    }
    __device__ __forceinline__ int wy(int y) const
    {
        if (my) return y < 0 ? -y : (y >= ny ? 2 * (ny - 1) - y : y);
        return y < 0 ? y + ny : (y >= ny ? y - ny : y);
    }
    __device__ __forceinline__ int wz(int z) const { return z < 0 ? z + nz : (z >= nz ? z - nz : z); }
    // a node in the grid (x, y wrap; z wraps when periodic, else in range)
    __device__ __forceinline__ long long at(int x, int y, int z) const
    {
        return base + (long long)(zwall ? z : wz(z)) * pxy + (long long)wy(y) * px + wx(x);
    }
    __device__ __forceinline__ bool wall(int z) const { return zwall && (z == 0 || z == nz - 1); }
};

enum { K_MIRROR = 0, K_WET = 1 };

// z-marching tiles for the D3Q19 operators: a CTA of BX x BY threads owns a
// BX x BY column of the x-y plane and walks ZCH planes up it, keeping the
// planes z-1, z, z+1 of each operand field in shared memory as windows with
// a one-node halo (ghost planes beyond a wall included), so a node's 18
// neighbours are shared-memory reads and each value comes from memory about
// once per plane instead of once per neighbour.
#ifndef ACM_TP3D_ZCH
#define ACM_TP3D_ZCH 8
#endif
#ifndef ACM_TP3D_BY
#define ACM_TP3D_BY 8
#endif
constexpr int BX = 32, BY = ACM_TP3D_BY, ZCH = ACM_TP3D_ZCH;
constexpr int WX = BX + 2, WY = BY + 2, WP = WX * WY;

// index c in [-1, n + BX] wrapped into [0, n) (a full modulo only for grids
// narrower than a tile), or reflected across the symmetry planes through
// nodes 0 and n - 1 (positions beyond n belong to no node of the grid and
// only need a valid index); *refl: c was reflected (odd fields change sign)
__device__ __forceinline__ int wrapc(int c, int n, bool mirror, bool *refl)
{
    if (mirror) {
        *refl = c < 0 || c >= n;
        if (c < 0) c = -c;
        else if (c >= n) c = 2 * (n - 1) - c;
        return c < 0 ? 0 : (c >= n ? n - 1 : c);
    }
    *refl = false;
    if (c < 0) c += n;
    else if (c >= n) c -= n;
    if ((unsigned)c >= (unsigned)n) {
        c %= n;
        if (c < 0) c += n;
    }
    return c;
}

// storage offsets of a node and its six axis neighbours (x, y wrap or
// mirror; z wraps when periodic; at a wall node the z neighbours beyond it
// are not used); sx / sy: sign of u at the x neighbours / of v at the y
// neighbours (-1 for an image across a symmetry plane)
struct Axis7 {
    long long c, xe, xw, yn, ys, zu, zd;
    float sxe, sxw, syn, sys;
    __device__ __forceinline__ Axis7(const Geo3 &g, int x, int y, int z)
    {
        c = g.base + (long long)z * g.pxy + (long long)y * g.px + x;
        const bool re = g.mx && x == g.nx - 1, rw = g.mx && x == 0;
        const bool rn = g.my && y == g.ny - 1, rs = g.my && y == 0;
        xe = c + (x == g.nx - 1 ? (g.mx ? -1 : 1 - g.nx) : 1);
        xw = c - (x == 0 ? (g.mx ? -1 : 1 - g.nx) : 1);
        yn = c + (y == g.ny - 1 ? (g.my ? -g.px : (1 - g.ny) * g.px) : g.px);
        ys = c - (y == 0 ? (g.my ? -g.px : (1 - g.ny) * g.px) : g.px);
        sxe = re ? -1.f : 1.f;
        sxw = rw ? -1.f : 1.f;
        syn = rn ? -1.f : 1.f;
        sys = rs ? -1.f : 1.f;
        const bool zp = !g.zwall;
        zu = c + (zp && z == g.nz - 1 ? (1 - g.nz) * g.pxy : g.pxy);
        zd = c - (zp && z == 0 ? (1 - g.nz) * g.pxy : g.pxy);
    }
};

// The x-y part of the storage offsets of the window elements a thread loads
// (elements tid and tid + BX BY of the WX x WY window; x and y wrap): the
// same for every field and plane, so it is formed once per CTA.
struct WinXY {
    long long xy[2];
    bool rx[2], ry[2];  // the element is an image across an x / y symmetry plane
    bool has2, anyr;    // second element; some element of this thread is an image
    __device__ __forceinline__ WinXY(const Geo3 &g, int x0, int y0)
    {
        const int tid = threadIdx.y * BX + threadIdx.x;
        anyr = false;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = min(tid + k * BX * BY, WP - 1);
            const int wy = i / WX, wx = i - wy * WX;
            const int yy = wrapc(y0 - 1 + wy, g.ny, g.my, &ry[k]);
            const int xx = wrapc(x0 - 1 + wx, g.nx, g.mx, &rx[k]);
            xy[k] = g.base + (long long)yy * g.px + xx;
            anyr |= rx[k] || ry[k];
        }
        has2 = tid + BX * BY < WP;
    }
};
static_assert(WP <= 2 * BX * BY, "a window must fit two loads per thread");

// window of plane z (z in [-1, nz]) of field f: beyond a wall face the
// mirror plane, plus (KIND == K_WET) the wetting term wet (1 - f_w^2) of the
// wall plane; ODD = 1 (u) / 2 (v): the field changes sign on images across
// x / y symmetry planes (those elements are loaded synchronously)
template <typename T, int KIND, int ODD = 0>
__device__ __forceinline__ void load_window(T *dst, const T *__restrict__ f, const Geo3 &g,
                                            const WinXY &o, int z, T wet)
{
    const int tid = threadIdx.y * BX + threadIdx.x;
    const bool ghost = g.zwall && (z < 0 || z >= g.nz);
    const int zz = ghost ? (z < 0 ? 1 : g.nz - 2) : (g.zwall ? z : g.wz(z));
    const long long zo = (long long)zz * g.pxy;
    const long long zwo = (long long)(z < 0 ? 0 : g.nz - 1) * g.pxy;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (k == 1 && !o.has2) break;
        const bool flip = (ODD == 1 && o.rx[k]) || (ODD == 2 && o.ry[k]);
        if (!ghost && !flip) {  // a plain copy: asynchronous, completed by the z-march's wait
            const unsigned d =
                static_cast<unsigned>(__cvta_generic_to_shared(dst + tid + k * BX * BY));
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d),
                         "l"(f + o.xy[k] + zo), "n"(sizeof(T))
                         : "memory");
            continue;
        }
        T val = f[o.xy[k] + zo];
        if (KIND == K_WET && ghost) {
            const T fw = f[o.xy[k] + zwo];
            val += wet * (T(1) - fw * fw);
        }
        dst[tid + k * BX * BY] = flip ? -val : val;
    }
}

// D3Q19 isotropic Laplacian (2/c_s^2) sum w_i (f_i - f_0) and gradient
// (1/c_s^2) sum w_i e_i f_i at window position c, planes z-1, z, z+1 in
// wm, w0, wp
template <typename T>
__device__ __forceinline__ void iso_ops(const T *wm, const T *w0, const T *wp, int c, T &lap,
                                        T &gx, T &gy, T &gz)
{
    const T f0 = w0[c];
    T la = T(0), le = T(0), ax = T(0), ay = T(0), az = T(0), ex = T(0), ey = T(0), ez = T(0);
#pragma unroll
    for (int i = 0; i < 18; ++i) {
        const int dx = vel(i, 0), dy = vel(i, 1), dz = vel(i, 2);
        const T *pl = dz < 0 ? wm : (dz > 0 ? wp : w0);
        const T fi = pl[c + dy * WX + dx];
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

// Walk the CTA's z-chunk: `load(slot, z)` issues the copies of plane z into
// ring slot `slot` (NSL slots), `body(z, sm, s0, sp)` computes plane z from
// the slots of z-1, z, z+1.  Plane z+2 is in flight while plane z is
// computed (cp.async groups, one per plane).
constexpr int NSL = 4;
template <typename L, typename B>
__device__ __forceinline__ void zmarch(int nz, L load, B body)
{
    const int z0 = blockIdx.z * ZCH, zend = min(z0 + ZCH, nz);
    load(0, z0 - 1);
    load(1, z0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    load(2, z0 + 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int z = z0; z < zend; ++z) {
        const int k = z - z0;
        if (z + 2 <= zend) load((k + 3) % NSL, z + 2);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // planes up to z+1 landed
        __syncthreads();
        body(z, k % NSL, (k + 1) % NSL, (k + 2) % NSL);
        __syncthreads();  // slot k % NSL is refilled next
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// 1, 4: mu = 4 a phi (phi^2 - 1) - kappa Lap_iso(phi)
template <typename T>
__global__ void __launch_bounds__(BX *BY) k_mu(const RunDesc R, const T *__restrict__ phi,
                                               T *__restrict__ mu)
{
    __shared__ T win[NSL][WP];
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T a = C[C_A], kappa = C[C_KAPPA], wet = C[C_WET];
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int c = (threadIdx.y + 1) * WX + threadIdx.x + 1;
    const WinXY o(g, x0, y0);
    zmarch(
        g.nz, [&](int sl, int z) { load_window<T, K_WET>(win[sl], phi, g, o, z, wet); },
        [&](int z, int sm, int s0, int sp) {
            if (x >= g.nx || y >= g.ny) return;
            T lap, gx, gy, gz;
            iso_ops(win[sm], win[s0], win[sp], c, lap, gx, gy, gz);
            const T f = win[s0][c];
            mu[g.base + (long long)z * g.pxy + (long long)y * g.px + x] =
                T(4) * a * f * (f * f - T(1)) - kappa * lap;
        });
}

// Eq. (2.10) at a non-wall node: Delta rho = -dt div(rho u) + satc Lap(rho')
template <typename T>
__device__ __forceinline__ T drho_at(const Fields<T> &in, const Geo3 &g, int x, int y, int z,
                                     T rho0, T dt, T satc)
{
    const T *r = in.f[F_R], *u = in.f[F_U], *v = in.f[F_V], *w = in.f[F_W];
    const Axis7 a(g, x, y, z);
    const T div = T(0.5) * ((rho0 + r[a.xe]) * (T(a.sxe) * u[a.xe]) -
                            (rho0 + r[a.xw]) * (T(a.sxw) * u[a.xw])) +
                  T(0.5) * ((rho0 + r[a.yn]) * (T(a.syn) * v[a.yn]) -
                            (rho0 + r[a.ys]) * (T(a.sys) * v[a.ys])) +
                  T(0.5) * ((rho0 + r[a.zu]) * w[a.zu] - (rho0 + r[a.zd]) * w[a.zd]);
    const T lap = (r[a.xe] + r[a.xw]) + (r[a.yn] + r[a.ys]) + (r[a.zu] + r[a.zd]) - T(6) * r[a.c];
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
        const long long c = g.base + (long long)z * g.pxy + (long long)y * g.px + x;
        if (!g.wall(z)) {
            dr[c] = drho_at(in, g, x, y, z, rho0, dt, satc);
            continue;
        }
        const int s = z == 0 ? 1 : -1;
        const T *r = in.f[F_R];
        const T r1 = r[c + s * g.pxy] + drho_at(in, g, x, y, z + s, rho0, dt, satc);
        const T r2 = r[c + 2 * s * g.pxy] + drho_at(in, g, x, y, z + 2 * s, rho0, dt, satc);
        dr[c] = (T(4) * r1 - r2) / T(3) - r[c];
    } while (0);
}

// 3: rho^{n+1}, u^{n+1} and phi*.  Every operand (mu, phi with the D3Q19
// stencils; rho', u, v, w, Delta rho with the 7-point ones) comes from the
// shared-memory plane windows of the z-march.
enum { W_MU, W_PH, W_R, W_U, W_V, W_W, W_DR, NWIN };

template <typename T>
constexpr size_t main_smem()
{
    return sizeof(T) * NWIN * NSL * WP;
}

template <typename T>
__global__ void __launch_bounds__(BX *BY)
    k_main(const RunDesc R, Fields<T> in, Fields<T> out, const T *__restrict__ dr,
           const T *__restrict__ mu, T *__restrict__ phs, unsigned *err)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sw = reinterpret_cast<T *>(smraw);
    auto win = [&](int f, int slot) { return sw + (f * NSL + slot) * WP; };
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T rho0 = C[C_RHO0], dt = C[C_DT], cs2 = C[C_CS2], nudt = C[C_NUDT];
    const T satm = C[C_SATM], mob = C[C_M], wet = C[C_WET];
    const T gfx = C[C_GX], gfy = C[C_GY], gfz = C[C_GZ];
    const T *src[NWIN] = {mu, in.f[F_PHI], in.f[F_R], in.f[F_U], in.f[F_V], in.f[F_W], dr};
    bool bad = false;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int cw = (threadIdx.y + 1) * WX + threadIdx.x + 1;
    const WinXY o(g, x0, y0);
    zmarch(g.nz,
           [&](int sl, int z) {
#pragma unroll
               for (int f = 0; f < NWIN; ++f) {
                   if (f == W_PH) load_window<T, K_WET>(win(f, sl), src[f], g, o, z, wet);
                   else if (f == W_U) load_window<T, K_MIRROR, 1>(win(f, sl), src[f], g, o, z, T(0));
                   else if (f == W_V) load_window<T, K_MIRROR, 2>(win(f, sl), src[f], g, o, z, T(0));
                   else load_window<T, K_MIRROR>(win(f, sl), src[f], g, o, z, T(0));
               }
           },
           [&](int z, int sm, int s0, int sp) {
        if (x >= g.nx || y >= g.ny) return;
        const T *r = win(W_R, s0), *u = win(W_U, s0), *v = win(W_V, s0), *w = win(W_W, s0);
        const T *d = win(W_DR, s0);
        const T r0 = r[cw], d0 = d[cw];
        const T rho1 = rho0 + r0 + d0;
        const T u0 = u[cw], v0 = v[cw], w0 = w[cw], f0 = win(W_PH, s0)[cw];
        // mu^n: Laplacian for the CHE and gradient for F_ST
        T lmu, gmx, gmy, gmz;
        iso_ops(win(W_MU, sm), win(W_MU, s0), win(W_MU, sp), cw, lmu, gmx, gmy, gmz);
        T un = T(0), vn = T(0), wn = T(0);
        if (!g.wall(z)) {
            // neighbours E, W, N, S in plane z; U, D in the planes above/below
            const T rr[6] = {r[cw + 1], r[cw - 1], r[cw + WX], r[cw - WX], win(W_R, sp)[cw],
                             win(W_R, sm)[cw]};
            const T uu[6] = {u[cw + 1], u[cw - 1], u[cw + WX], u[cw - WX], win(W_U, sp)[cw],
                             win(W_U, sm)[cw]};
            const T vv[6] = {v[cw + 1], v[cw - 1], v[cw + WX], v[cw - WX], win(W_V, sp)[cw],
                             win(W_V, sm)[cw]};
            const T ww[6] = {w[cw + 1], w[cw - 1], w[cw + WX], w[cw - WX], win(W_W, sp)[cw],
                             win(W_W, sm)[cw]};
            T mx[6], my[6], mz[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const T q = rho0 + rr[k];
                mx[k] = q * uu[k];
                my[k] = q * vv[k];
                mz[k] = q * ww[k];
            }
            const T q0 = rho0 + r0;
            const T mx0 = q0 * u0, my0 = q0 * v0, mz0 = q0 * w0;
            auto flux = [&](const T (&m)[6]) {
                return T(0.5) * ((m[0] * uu[0] - m[1] * uu[1]) + (m[2] * vv[2] - m[3] * vv[3]) +
                                 (m[4] * ww[4] - m[5] * ww[5]));
            };
            auto lap = [&](const T (&m)[6], T m0) {
                return ((m[0] + m[1]) + (m[2] + m[3])) + (m[4] + m[5]) - T(6) * m0;
            };
            const T ddx = T(0.5) * (d[cw + 1] - d[cw - 1]);
            const T ddy = T(0.5) * (d[cw + WX] - d[cw - WX]);
            const T ddz = T(0.5) * (win(W_DR, sp)[cw] - win(W_DR, sm)[cw]);
            // body force: on both phases, or the Boussinesq drop force
            const T fb = dt * rho1 * (C[C_BQA] + C[C_BQB] * f0);
            T rx = -dt * flux(mx) - dt * cs2 * T(0.5) * (rr[0] - rr[1]) + nudt * lap(mx, mx0) -
                   satm * ddx + fb * gfx - dt * f0 * gmx;
            T ry = -dt * flux(my) - dt * cs2 * T(0.5) * (rr[2] - rr[3]) + nudt * lap(my, my0) -
                   satm * ddy + fb * gfy - dt * f0 * gmy;
            T rz = -dt * flux(mz) - dt * cs2 * T(0.5) * (rr[4] - rr[5]) + nudt * lap(mz, mz0) -
                   satm * ddz + fb * gfz - dt * f0 * gmz;
            const T inv = T(1) / rho1;
            un = u0 + (rx - d0 * u0) * inv;
            vn = v0 + (ry - d0 * v0) * inv;
            wn = w0 + (rz - d0 * w0) * inv;
            // the normal velocity is zero on a symmetry plane
            if (g.mx && (x == 0 || x == g.nx - 1)) un = T(0);
            if (g.my && (y == 0 || y == g.ny - 1)) vn = T(0);
        }
        // first Heun stage of Eq. (2.14), u^n frozen
        T lph, gpx, gpy, gpz;
        iso_ops(win(W_PH, sm), win(W_PH, s0), win(W_PH, sp), cw, lph, gpx, gpy, gpz);
        const T fs = f0 + dt * (-(u0 * gpx + v0 * gpy + w0 * gpz) + mob * lmu);
        const T rn = r0 + d0;
        const long long c = g.base + (long long)z * g.pxy + (long long)y * g.px + x;
        out.f[F_R][c] = rn;
        out.f[F_U][c] = un;
        out.f[F_V][c] = vn;
        out.f[F_W][c] = wn;
        phs[c] = fs;
        bad |= !isfinite(rn + un + vn + wn + fs);
           });
    if (bad) atomicOr(err, ERR_NONFINITE);
}

// 5: phi^{n+1}
template <typename T>
__global__ void __launch_bounds__(BX *BY)
    k_phi(const RunDesc R, Fields<T> in, const T *__restrict__ phs, const T *__restrict__ mus,
          T *__restrict__ phn, unsigned *err)
{
    __shared__ T wmu[NSL][WP], wps[NSL][WP];
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T dt = C[C_DT], mob = C[C_M], wet = C[C_WET];
    const T *u = in.f[F_U], *v = in.f[F_V], *w = in.f[F_W], *ph = in.f[F_PHI];
    bool bad = false;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int cw = (threadIdx.y + 1) * WX + threadIdx.x + 1;
    const WinXY o(g, x0, y0);
    zmarch(g.nz,
           [&](int sl, int z) {
               load_window<T, K_MIRROR>(wmu[sl], mus, g, o, z, T(0));
               load_window<T, K_WET>(wps[sl], phs, g, o, z, wet);
           },
           [&](int z, int sm, int s0, int sp) {
               if (x >= g.nx || y >= g.ny) return;
               const long long c = g.base + (long long)z * g.pxy + (long long)y * g.px + x;
               T lmu, a0, a1, a2, lph, gpx, gpy, gpz;
               iso_ops(wmu[sm], wmu[s0], wmu[sp], cw, lmu, a0, a1, a2);
               iso_ops(wps[sm], wps[s0], wps[sp], cw, lph, gpx, gpy, gpz);
               const T r2 = -(u[c] * gpx + v[c] * gpy + w[c] * gpz) + mob * lmu;
               const T f = T(0.5) * (ph[c] + wps[s0][cw] + dt * r2);
               phn[c] = f;
               bad |= !isfinite(f);
           });
    if (bad) atomicOr(err, ERR_NONFINITE);
}

}  // namespace

template <typename T>
void tp3d_prepare()
{
    cudaFuncSetAttribute(k_main<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)main_smem<T>());
}

template <typename T>
cudaError_t launch_tp3d(const RunDesc &R, Fields<T> in, Fields<T> out, T *mu, T *phs, T *dr,
                        unsigned *err, int sms, cudaStream_t s)
{
    (void)sms;
    // Delta rho: one thread per node, 32 x 4 x 2 blocks (x fastest, coalesced)
    const dim3 blk(32, 4, 2);
    const dim3 grid((R.nx + 31) / 32, (R.ny + 3) / 4, (R.nz + 1) / 2);
    // D3Q19 passes: BX x BY tiles marching over chunks of ZCH planes
    const dim3 tblk(BX, BY, 1);
    const dim3 tgrid((R.nx + BX - 1) / BX, (R.ny + BY - 1) / BY, (R.nz + ZCH - 1) / ZCH);
    k_mu<T><<<tgrid, tblk, 0, s>>>(R, in.f[F_PHI], mu);
    k_drho<T><<<grid, blk, 0, s>>>(R, in, dr);
    k_main<T><<<tgrid, tblk, main_smem<T>(), s>>>(R, in, out, dr, mu, phs, err);
    k_mu<T><<<tgrid, tblk, 0, s>>>(R, phs, mu);
    k_phi<T><<<tgrid, tblk, 0, s>>>(R, in, phs, mu, out.f[F_PHI], err);
    return cudaGetLastError();
}

template void tp3d_prepare<float>();
template void tp3d_prepare<double>();
template cudaError_t launch_tp3d<float>(const RunDesc &, Fields<float>, Fields<float>, float *,
                                        float *, float *, unsigned *, int, cudaStream_t);
template cudaError_t launch_tp3d<double>(const RunDesc &, Fields<double>, Fields<double>,
                                         double *, double *, double *, unsigned *, int,
                                         cudaStream_t);

}  // namespace acm
