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
// Five launches per step:
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
#include "acm_pair.h"

namespace acm {
namespace {

using pair::add2;
using pair::fma2;
using pair::mk;
using pair::mul2;
using pair::P2;
using pair::splat;
using pair::sub2;

constexpr int TPB = 256;

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
    __device__ __forceinline__ int wz(int z) const { return z < 0 ? z + nz : (z >= nz ? z - nz : z); }
    __device__ __forceinline__ bool wall(int z) const { return zwall && (z == 0 || z == nz - 1); }
};

enum { K_MIRROR = 0, K_WET = 1 };

// z-marching tiles for the D3Q19 passes: a CTA of BX x BY threads owns a
// BX x 2 BY column of the x-y plane (each thread the two y-adjacent nodes
// (x, y) and (x, y + 1), updated as one pair: packed two-lane instructions
// in FP32) and walks ZCH planes up it, keeping the planes z-1, z, z+1 of
// each operand field in shared memory as windows with a one-node halo
// (ghost planes beyond a wall included), so a pair's 28 distinct stencil
// values are shared-memory reads and each value comes from memory about
// once per plane.
#ifndef ACM_TP3D_ZCH
#define ACM_TP3D_ZCH 6
#endif
constexpr int BX = 32, BY = 8, NT = BX * BY, TR = 2 * BY, ZCH = ACM_TP3D_ZCH;
constexpr int WX = BX + 2, WY = TR + 2, WP = WX * WY;
constexpr int NLD = (WP + NT - 1) / NT;  // window elements a thread copies

// index c in [-1, n + BX] (x) or [-1, n + TR] (y) wrapped into [0, n) (a
// full modulo only for grids narrower than a tile), or reflected across the
// symmetry planes through nodes 0 and n - 1 (positions beyond n belong to no
// node of the grid and only need a valid index); *refl: c was reflected (odd
// fields change sign)
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

// The x-y offsets (from the first node of a plane) of the window elements a
// thread copies (elements tid + k NT of the WX x WY window; x and y wrap or
// reflect): the same for every field and plane, so they are formed once per
// CTA.  A plane fits 32-bit offsets.
struct WinXY {
    int xy[NLD];
    bool rx[NLD], ry[NLD];  // the element is an image across an x / y symmetry plane
    bool has[NLD];          // the element exists (the last round covers part of the window)
    bool fx, fy;            // some element of this thread is an x / y image
    __device__ __forceinline__ WinXY(const Geo3 &g, int x0, int y0)
    {
        const int tid = threadIdx.y * BX + threadIdx.x;
        fx = fy = false;
#pragma unroll
        for (int k = 0; k < NLD; ++k) {
            has[k] = tid + k * NT < WP;
            const int i = min(tid + k * NT, WP - 1);
            const int wy = i / WX, wx = i - wy * WX;
            const int yy = wrapc(y0 - 1 + wy, g.ny, g.my, &ry[k]);
            const int xx = wrapc(x0 - 1 + wx, g.nx, g.mx, &rx[k]);
            xy[k] = yy * (int)g.px + xx;
            fx |= has[k] && rx[k];
            fy |= has[k] && ry[k];
        }
    }
    // element k exists for this thread (in the full rounds, for every thread:
    // a compile-time fact)
    __device__ __forceinline__ bool in(int k) const { return (k + 1) * NT <= WP || has[k]; }
};

// 32-bit shared-memory address of this thread's first element of window w
template <typename T>
__device__ __forceinline__ unsigned sh_addr(const T *w)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(w)) +
           (threadIdx.y * BX + threadIdx.x) * (unsigned)sizeof(T);
}

template <int N>
__device__ __forceinline__ void cp_async_sh(unsigned dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(N)
                 : "memory");
}

// window of plane z (z in [-1, nz]) of field f into dst (sd: sh_addr(dst)):
// beyond a wall face the mirror plane, plus (KIND == K_WET) the wetting term
// wet (1 - f_w^2) of the wall plane; ODD = 1 (u) / 2 (v): the field changes
// sign on images across x / y symmetry planes.  A thread whose elements are
// plain copies issues them asynchronously (completed by the z-march's
// wait); ghost planes and sign-flipped images are loaded synchronously.
template <typename T, int KIND, int ODD = 0>
__device__ __forceinline__ void load_window(T *dst, unsigned sd, const T *__restrict__ f,
                                            const Geo3 &g, const WinXY &o, int z, T wet)
{
    const bool ghost = g.zwall && (z < 0 || z >= g.nz);
    const int zz = ghost ? (z < 0 ? 1 : g.nz - 2) : (g.zwall ? z : g.wz(z));
    const T *pf = f + (g.base + (long long)zz * g.pxy);
    const bool flips = (ODD == 1 && o.fx) || (ODD == 2 && o.fy);
    if (!ghost && !flips) {
#pragma unroll
        for (int k = 0; k < NLD; ++k)
            if (o.in(k)) cp_async_sh<sizeof(T)>(sd + k * NT * (unsigned)sizeof(T), pf + o.xy[k]);
        return;
    }
    const int tid = threadIdx.y * BX + threadIdx.x;
    const T *pw = f + (g.base + (long long)(z < 0 ? 0 : g.nz - 1) * g.pxy);
#pragma unroll
    for (int k = 0; k < NLD; ++k) {
        if (!o.in(k)) continue;
        const bool flip = (ODD == 1 && o.rx[k]) || (ODD == 2 && o.ry[k]);
        T val = pf[o.xy[k]];
        if (KIND == K_WET && ghost) {
            const T fw = pw[o.xy[k]];
            val += wet * (T(1) - fw * fw);
        }
        dst[tid + k * NT] = flip ? -val : val;
    }
}

// The values at window offset (dx, dy) from the pair's nodes a (window
// index c) and b (c + WX) on plane p.
template <typename T>
__device__ __forceinline__ P2<T> at2(const T *p, int c, int dx, int dy)
{
    return mk(p[c + dy * WX + dx], p[c + (dy + 1) * WX + dx]);
}

// D3Q19 isotropic Laplacian (2/c_s^2) sum w_i (f_i - f_0) = (1/3) sum over
// the 6 axis neighbours + (1/6) sum over the 12 edge neighbours of
// (f_i - f_0), for the node pair at c; planes z-1, z, z+1 in pm, p0, pp
template <typename T>
__device__ __forceinline__ P2<T> iso_lap2(const T *pm, const T *p0, const T *pp, int c)
{
    const P2<T> f0 = at2(p0, c, 0, 0);
    auto d = [&](const T *p, int dx, int dy) { return sub2(at2(p, c, dx, dy), f0); };
    const P2<T> la = add2(add2(add2(d(p0, 1, 0), d(p0, -1, 0)), add2(d(p0, 0, 1), d(p0, 0, -1))),
                          add2(d(pp, 0, 0), d(pm, 0, 0)));
    const P2<T> le = add2(
        add2(add2(add2(d(p0, 1, 1), d(p0, 1, -1)), add2(d(p0, -1, 1), d(p0, -1, -1))),
             add2(add2(d(pp, 1, 0), d(pm, 1, 0)), add2(d(pp, -1, 0), d(pm, -1, 0)))),
        add2(add2(d(pp, 0, 1), d(pm, 0, 1)), add2(d(pp, 0, -1), d(pm, 0, -1))));
    return fma2(splat(T(1.0 / 6.0)), le, mul2(splat(T(1.0 / 3.0)), la));
}

// D3Q19 isotropic gradient (1/c_s^2) sum w_i e_i f_i: per component
// (1/6) (axis neighbour + minus axis neighbour -) + (1/12) (sum of the four
// edge neighbours on the + side - sum of the four on the - side)
template <typename T>
__device__ __forceinline__ void iso_grad2(const T *pm, const T *p0, const T *pp, int c,
                                          P2<T> &gx, P2<T> &gy, P2<T> &gz)
{
    auto v = [&](const T *p, int dx, int dy) { return at2(p, c, dx, dy); };
    const P2<T> ax = sub2(v(p0, 1, 0), v(p0, -1, 0));
    const P2<T> ay = sub2(v(p0, 0, 1), v(p0, 0, -1));
    const P2<T> az = sub2(v(pp, 0, 0), v(pm, 0, 0));
    const P2<T> ex = sub2(add2(add2(v(p0, 1, 1), v(p0, 1, -1)), add2(v(pp, 1, 0), v(pm, 1, 0))),
                          add2(add2(v(p0, -1, 1), v(p0, -1, -1)), add2(v(pp, -1, 0), v(pm, -1, 0))));
    const P2<T> ey = sub2(add2(add2(v(p0, 1, 1), v(p0, -1, 1)), add2(v(pp, 0, 1), v(pm, 0, 1))),
                          add2(add2(v(p0, 1, -1), v(p0, -1, -1)), add2(v(pp, 0, -1), v(pm, 0, -1))));
    const P2<T> ez = sub2(add2(add2(v(pp, 1, 0), v(pp, -1, 0)), add2(v(pp, 0, 1), v(pp, 0, -1))),
                          add2(add2(v(pm, 1, 0), v(pm, -1, 0)), add2(v(pm, 0, 1), v(pm, 0, -1))));
    const P2<T> c6 = splat(T(1.0 / 6.0)), c12 = splat(T(1.0 / 12.0));
    gx = fma2(c12, ex, mul2(c6, ax));
    gy = fma2(c12, ey, mul2(c6, ay));
    gz = fma2(c12, ez, mul2(c6, az));
}

// Walk the CTA's z-chunk: `load(slot, z)` issues the copies of plane z into
// ring slot `slot` (NSL slots), `body(z, sm, s0, sp)` computes plane z from
// the slots of z-1, z, z+1.  Plane z+2 is in flight while plane z is
// computed (cp.async groups, one per plane); the loop is unrolled by the
// slot count, so every slot index is a constant.
constexpr int NSL = 4;
template <typename L, typename B>
__device__ __forceinline__ void zmarch(int nz, L load, B body)
{
    const int z0 = blockIdx.z * ZCH, zend = min(z0 + ZCH, nz);
    load(0, z0 - 1);
    load(1, z0);
    pair::cp_async_commit();
    load(2, z0 + 1);
    pair::cp_async_commit();
    for (int zb = z0; zb < zend; zb += NSL) {
#pragma unroll
        for (int i = 0; i < NSL; ++i) {
            const int z = zb + i;
            if (z >= zend) break;
            if (z + 2 <= zend) load((i + 3) % NSL, z + 2);
            pair::cp_async_commit();
            pair::cp_async_wait<1>();  // planes up to z+1 landed
            __syncthreads();
            body(z, i, (i + 1) % NSL, (i + 2) % NSL);
            __syncthreads();  // slot i is refilled next
        }
    }
    pair::cp_async_wait<0>();
}

// Tile geometry of a thread: node a = (x, ya), node b = (x, ya + 1); c =
// window index of a; own = storage index of a on plane 0.
struct Tile {
    int x, ya, c;
    bool act, hasb;
    long long own;
    __device__ __forceinline__ Tile(const Geo3 &g)
    {
        x = blockIdx.x * BX + threadIdx.x;
        ya = blockIdx.y * TR + 2 * threadIdx.y;
        c = (2 * threadIdx.y + 1) * WX + threadIdx.x + 1;
        act = x < g.nx && ya < g.ny;
        hasb = ya + 1 < g.ny;
        own = g.base + (long long)ya * g.px + x;
    }
};

// a pair's contribution to the blow-up check (node b only where it exists)
template <typename T>
__device__ __forceinline__ P2<T> own_part(P2<T> s, bool hasb)
{
    return hasb ? s : mk(s.x, T(0));
}

// 1, 4: mu = 4 a phi (phi^2 - 1) - kappa Lap_iso(phi)
template <typename T>
__global__ void __launch_bounds__(NT) k_mu(const RunDesc R, const T *__restrict__ phi,
                                           T *__restrict__ mu)
{
    __shared__ __align__(16) T win[NSL][WP];
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T a4 = T(4) * C[C_A], kappa = C[C_KAPPA], wet = C[C_WET];
    const Tile t(g);
    const WinXY o(g, blockIdx.x * BX, blockIdx.y * TR);
    const unsigned sd = sh_addr(&win[0][0]);
    zmarch(
        g.nz,
        [&](int sl, int z) {
            load_window<T, K_WET>(win[sl], sd + sl * WP * (unsigned)sizeof(T), phi, g, o, z, wet);
        },
        [&](int z, int sm, int s0, int sp) {
            if (!t.act) return;
            const P2<T> lap = iso_lap2(win[sm], win[s0], win[sp], t.c);
            const P2<T> f = at2(win[s0], t.c, 0, 0);
            const P2<T> m = fma2(splat(-kappa), lap,
                                 mul2(mul2(splat(a4), f), fma2(f, f, splat(T(-1)))));
            const long long i = t.own + (long long)z * g.pxy;
            mu[i] = m.x;
            if (t.hasb) mu[i + g.px] = m.y;
        });
}

// Eq. (2.10) at a non-wall node: Delta rho = -dt div(rho u) + satc Lap(rho').
// Neighbour offsets from the node: x and y wrap or mirror (32-bit: within a
// plane), z wraps when periodic (at a wall node the z neighbours beyond it
// are not used); u at an x image and v at a y image across a symmetry plane
// change sign.
template <typename T>
__device__ __forceinline__ T drho_at(const Fields<T> &in, const Geo3 &g, int x, int y, int z,
                                     T rho0, T dt, T satc)
{
    const long long c = g.base + (long long)z * g.pxy + (long long)y * g.px + x;
    const int px = (int)g.px;
    const bool xe = x == g.nx - 1, xw = x == 0, yn = y == g.ny - 1, ys = y == 0;
    const int oe = xe ? (g.mx ? -1 : 1 - g.nx) : 1;
    const int ow = xw ? (g.mx ? 1 : g.nx - 1) : -1;
    const int on = (yn ? (g.my ? -1 : 1 - g.ny) : 1) * px;
    const int os = (ys ? (g.my ? 1 : g.ny - 1) : -1) * px;
    const bool zp = !g.zwall;
    const long long ou = zp && z == g.nz - 1 ? (1 - g.nz) * g.pxy : g.pxy;
    const long long od = zp && z == 0 ? (g.nz - 1) * g.pxy : -g.pxy;
    const T *r = in.f[F_R] + c, *u = in.f[F_U] + c, *v = in.f[F_V] + c, *w = in.f[F_W] + c;
    const T ue = g.mx && xe ? -u[oe] : u[oe], uw = g.mx && xw ? -u[ow] : u[ow];
    const T vn = g.my && yn ? -v[on] : v[on], vs = g.my && ys ? -v[os] : v[os];
    const T div = T(0.5) * ((rho0 + r[oe]) * ue - (rho0 + r[ow]) * uw) +
                  T(0.5) * ((rho0 + r[on]) * vn - (rho0 + r[os]) * vs) +
                  T(0.5) * ((rho0 + r[ou]) * w[ou] - (rho0 + r[od]) * w[od]);
    const T lap = (r[oe] + r[ow]) + (r[on] + r[os]) + (r[ou] + r[od]) - T(6) * r[0];
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

#ifdef ACM_TP3D_MAIN_MINB
#define ACM_TP3D_MAIN_BOUNDS __launch_bounds__(NT, ACM_TP3D_MAIN_MINB)
#else
#define ACM_TP3D_MAIN_BOUNDS __launch_bounds__(NT)
#endif
template <typename T>
__global__ void ACM_TP3D_MAIN_BOUNDS
    k_main(const RunDesc R, Fields<T> in, Fields<T> out, const T *__restrict__ dr,
           const T *__restrict__ mu, T *__restrict__ phs, unsigned *err)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sw = reinterpret_cast<T *>(smraw);
    auto win = [&](int f, int slot) { return sw + (f * NSL + slot) * WP; };
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T rho0 = C[C_RHO0], dt = C[C_DT], nudt = C[C_NUDT];
    const T pgc = dt * C[C_CS2] * T(0.5), satm = C[C_SATM], mob = C[C_M], wet = C[C_WET];
    const T gfx = C[C_GX], gfy = C[C_GY], gfz = C[C_GZ], bqa = C[C_BQA], bqb = C[C_BQB];
    const T *src[NWIN] = {mu, in.f[F_PHI], in.f[F_R], in.f[F_U], in.f[F_V], in.f[F_W], dr};
    const Tile t(g);
    // the normal velocity is zero on a symmetry plane
    const bool zu = g.mx && (t.x == 0 || t.x == g.nx - 1);
    const bool zva = g.my && (t.ya == 0 || t.ya == g.ny - 1), zvb = g.my && t.ya + 1 == g.ny - 1;
    const WinXY o(g, blockIdx.x * BX, blockIdx.y * TR);
    const unsigned sd = sh_addr(sw);
    P2<T> fin = splat(T(0));
    zmarch(g.nz,
           [&](int sl, int z) {
#pragma unroll
               for (int f = 0; f < NWIN; ++f) {
                   T *w = win(f, sl);
                   const unsigned a = sd + (f * NSL + sl) * WP * (unsigned)sizeof(T);
                   if (f == W_PH) load_window<T, K_WET>(w, a, src[f], g, o, z, wet);
                   else if (f == W_U) load_window<T, K_MIRROR, 1>(w, a, src[f], g, o, z, T(0));
                   else if (f == W_V) load_window<T, K_MIRROR, 2>(w, a, src[f], g, o, z, T(0));
                   else load_window<T, K_MIRROR>(w, a, src[f], g, o, z, T(0));
               }
           },
           [&](int z, int sm, int s0, int sp) {
        if (!t.act) return;
        const int c = t.c;
        const T *r = win(W_R, s0), *u = win(W_U, s0), *v = win(W_V, s0), *w = win(W_W, s0);
        const T *d = win(W_DR, s0), *ph = win(W_PH, s0);
        const P2<T> r0 = at2(r, c, 0, 0), d0 = at2(d, c, 0, 0);
        const P2<T> u0 = at2(u, c, 0, 0), v0 = at2(v, c, 0, 0), w0 = at2(w, c, 0, 0);
        const P2<T> f0 = at2(ph, c, 0, 0);
        // first Heun stage of Eq. (2.14), u^n frozen: phi* = phi + dt (M Lap mu - u . grad phi)
        const P2<T> lmu = iso_lap2(win(W_MU, sm), win(W_MU, s0), win(W_MU, sp), c);
        P2<T> gpx, gpy, gpz;
        iso_grad2(win(W_PH, sm), ph, win(W_PH, sp), c, gpx, gpy, gpz);
        const P2<T> adv = fma2(w0, gpz, fma2(v0, gpy, mul2(u0, gpx)));
        const P2<T> fs = fma2(splat(dt), sub2(mul2(splat(mob), lmu), adv), f0);
        const P2<T> rn = add2(r0, d0);
        P2<T> un = splat(T(0)), vn = un, wn = un;
        if (!g.wall(z)) {
            P2<T> gmx, gmy, gmz;
            iso_grad2(win(W_MU, sm), win(W_MU, s0), win(W_MU, sp), c, gmx, gmy, gmz);
            // axis neighbours E, W, N, S in plane z; U, D in the planes above/below
            auto ax6 = [&](int f, P2<T> (&a)[6]) {
                const T *p = win(f, s0);
                a[0] = at2(p, c, 1, 0);
                a[1] = at2(p, c, -1, 0);
                a[2] = at2(p, c, 0, 1);
                a[3] = at2(p, c, 0, -1);
                a[4] = at2(win(f, sp), c, 0, 0);
                a[5] = at2(win(f, sm), c, 0, 0);
            };
            P2<T> rr[6], uu[6], vv[6], ww[6];
            ax6(W_R, rr);
            ax6(W_U, uu);
            ax6(W_V, vv);
            ax6(W_W, ww);
            P2<T> mx[6], my[6], mz[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const P2<T> q = add2(splat(rho0), rr[k]);
                mx[k] = mul2(q, uu[k]);
                my[k] = mul2(q, vv[k]);
                mz[k] = mul2(q, ww[k]);
            }
            const P2<T> q0 = add2(splat(rho0), r0);
            const P2<T> rho1 = add2(q0, d0);
            // -dt div(m u) with central differences
            auto flux = [&](const P2<T> (&m)[6]) {
                const P2<T> fx = sub2(mul2(m[0], uu[0]), mul2(m[1], uu[1]));
                const P2<T> fy = sub2(mul2(m[2], vv[2]), mul2(m[3], vv[3]));
                const P2<T> fz = sub2(mul2(m[4], ww[4]), mul2(m[5], ww[5]));
                return mul2(splat(T(-0.5) * dt), add2(add2(fx, fy), fz));
            };
            auto lap7 = [&](const P2<T> (&m)[6], P2<T> m0) {
                return fma2(splat(T(-6)), m0,
                            add2(add2(add2(m[0], m[1]), add2(m[2], m[3])), add2(m[4], m[5])));
            };
            const P2<T> ddx = mul2(splat(T(0.5)), sub2(at2(d, c, 1, 0), at2(d, c, -1, 0)));
            const P2<T> ddy = mul2(splat(T(0.5)), sub2(at2(d, c, 0, 1), at2(d, c, 0, -1)));
            const P2<T> ddz =
                mul2(splat(T(0.5)), sub2(at2(win(W_DR, sp), c, 0, 0), at2(win(W_DR, sm), c, 0, 0)));
            // body force: on both phases, or the Boussinesq drop force
            const P2<T> fb = mul2(mul2(splat(dt), rho1), fma2(splat(bqb), f0, splat(bqa)));
            const P2<T> fst = mul2(splat(-dt), f0);  // F_ST dt = -dt phi grad mu
            auto rhs = [&](const P2<T> (&m)[6], P2<T> m0, int k, P2<T> dd, T gf, P2<T> gm) {
                P2<T> a = flux(m);
                a = fma2(splat(-pgc), sub2(rr[2 * k], rr[2 * k + 1]), a);
                a = fma2(splat(nudt), lap7(m, m0), a);
                a = fma2(splat(-satm), dd, a);
                a = fma2(fb, splat(gf), a);
                return fma2(fst, gm, a);
            };
            const P2<T> rx = rhs(mx, mul2(q0, u0), 0, ddx, gfx, gmx);
            const P2<T> ry = rhs(my, mul2(q0, v0), 1, ddy, gfy, gmy);
            const P2<T> rz = rhs(mz, mul2(q0, w0), 2, ddz, gfz, gmz);
            const P2<T> inv = mk(pair::recip(rho1.x), pair::recip(rho1.y));
            un = fma2(sub2(rx, mul2(d0, u0)), inv, u0);
            vn = fma2(sub2(ry, mul2(d0, v0)), inv, v0);
            wn = fma2(sub2(rz, mul2(d0, w0)), inv, w0);
            if (zu) un = splat(T(0));
            if (zva) vn.x = T(0);
            if (zvb) vn.y = T(0);
        }
        const long long i = t.own + (long long)z * g.pxy;
        out.f[F_R][i] = rn.x;
        out.f[F_U][i] = un.x;
        out.f[F_V][i] = vn.x;
        out.f[F_W][i] = wn.x;
        phs[i] = fs.x;
        if (t.hasb) {
            const long long j = i + g.px;
            out.f[F_R][j] = rn.y;
            out.f[F_U][j] = un.y;
            out.f[F_V][j] = vn.y;
            out.f[F_W][j] = wn.y;
            phs[j] = fs.y;
        }
        fin = add2(fin, own_part<T>(add2(add2(add2(rn, un), add2(vn, wn)), fs), t.hasb));
           });
    if (!isfinite(pair::add1(fin.x, fin.y))) atomicOr(err, ERR_NONFINITE);
}

// 5: phi^{n+1}
template <typename T>
__global__ void __launch_bounds__(NT)
    k_phi(const RunDesc R, Fields<T> in, const T *__restrict__ phs, const T *__restrict__ mus,
          T *__restrict__ phn, unsigned *err)
{
    __shared__ __align__(16) T wmu[NSL][WP], wps[NSL][WP];
    const Geo3 g(R);
    const T *C = coefs<T>(R);
    const T dt = C[C_DT], mob = C[C_M], wet = C[C_WET];
    const T *u = in.f[F_U], *v = in.f[F_V], *w = in.f[F_W], *ph = in.f[F_PHI];
    const Tile t(g);
    const WinXY o(g, blockIdx.x * BX, blockIdx.y * TR);
    const unsigned smu = sh_addr(&wmu[0][0]), sps = sh_addr(&wps[0][0]);
    P2<T> fin = splat(T(0));
    zmarch(g.nz,
           [&](int sl, int z) {
               const unsigned so = sl * WP * (unsigned)sizeof(T);
               load_window<T, K_MIRROR>(wmu[sl], smu + so, mus, g, o, z, T(0));
               load_window<T, K_WET>(wps[sl], sps + so, phs, g, o, z, wet);
           },
           [&](int z, int sm, int s0, int sp) {
               if (!t.act) return;
               // node b's row is at most ny, a padding row of the layout when b is outside
               const long long i = t.own + (long long)z * g.pxy, j = i + g.px;
               const P2<T> lmu = iso_lap2(wmu[sm], wmu[s0], wmu[sp], t.c);
               P2<T> gpx, gpy, gpz;
               iso_grad2(wps[sm], wps[s0], wps[sp], t.c, gpx, gpy, gpz);
               const P2<T> adv = fma2(mk(w[i], w[j]), gpz,
                                      fma2(mk(v[i], v[j]), gpy, mul2(mk(u[i], u[j]), gpx)));
               const P2<T> r2 = sub2(mul2(splat(mob), lmu), adv);
               const P2<T> f = mul2(splat(T(0.5)), fma2(splat(dt), r2,
                                                        add2(mk(ph[i], ph[j]), at2(wps[s0], t.c, 0, 0))));
               phn[i] = f.x;
               if (t.hasb) phn[j] = f.y;
               fin = add2(fin, own_part<T>(f, t.hasb));
           });
    if (!isfinite(pair::add1(fin.x, fin.y))) atomicOr(err, ERR_NONFINITE);
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
    // D3Q19 passes: BX x 2 BY tiles (BX x BY threads) marching over chunks of ZCH planes
    const dim3 tblk(BX, BY, 1);
    const dim3 tgrid((R.nx + BX - 1) / BX, (R.ny + TR - 1) / TR, (R.nz + ZCH - 1) / ZCH);
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
