// Fused 3D time step of the simplified MAME scheme (Huang, arXiv:2012.03525,
// Section 2, Eqs. 2.10-2.11 with the 7-point extension of Eq. 2.13), periodic
// grids, single phase.
//
// Design (one kernel per step, HBM-bound):
//   * Each CTA owns a 32 x TY column of the x-y plane and marches along z over
//     a chunk of planes; each thread owns two y-adjacent nodes of the column.
//   * Input planes of rho', u, v, w (with a 2-node x-y halo) are staged in
//     shared memory by TMA tiled loads (cp.async.bulk.tensor.3d) into a ring
//     of NSLOT plane slots; loads run up to NSLOT-3 planes ahead of the one
//     the compute waits for.
//   * A thread keeps the values of its own two nodes on planes z-1..z+2 in
//     registers (a register queue along z), so z-neighbours never touch
//     shared memory; the upper/lower node of the pair serve as each other's
//     y-neighbour.
//   * Eq. (2.10) is evaluated for plane z+1 on the tile grown by one node:
//     the own nodes in registers, the one-node ring by 100 threads; Delta rho
//     of the own nodes stays in a register queue (z-1, z, z+1), the tile plane
//     goes to shared memory (one window per plane slot, so its index is a
//     compile-time constant) for the x/y neighbours, so
//     d_a rho^{n+1} - d_a rho^n of Eq. (2.11) is a centred difference of
//     Delta rho.
//   * Eq. (2.11) for plane z; u^{n+1} = u + (RHS - Delta rho u) / rho^{n+1}.
//   * Every thread keeps a running sum of its outputs (finite only if every
//     value added is finite); one flag per CTA (ERR_NONFINITE) reports a
//     blow-up without a separate pass.  Output addresses advance by one
//     plane per step.
// Storage is padded by T3PAD ghost nodes in x and y (not in z).  Every output
// node on the first/last two columns/rows is also written to its periodic
// image in the ghost layers, so the next step's TMA boxes never wrap in x/y;
// z wraps through the box coordinate, except in a sub-domain (one z-slab of
// a larger grid), whose two ghost planes beyond each z face hold the
// neighbouring slabs' planes.  Padding also keeps every box start on a
// 16-byte boundary (x start = tile x0, a multiple of 32 elements).
#include <algorithm>
#include <type_traits>

#include "acm_internal.h"

namespace acm {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// bounded wait: ~ 2^22 polls (well over a second), then give up
constexpr int WAIT_LIMIT = 1 << 22;

template <typename T>
struct Prec;
template <>
struct Prec<float> {
#ifndef ACM_STEP3D_NSLOT
#define ACM_STEP3D_NSLOT 5
#endif
    static constexpr int NSLOT = ACM_STEP3D_NSLOT;
#ifndef ACM_STEP3D_MINB
#define ACM_STEP3D_MINB 2
#endif
    static constexpr int MINB = ACM_STEP3D_MINB;  // CTAs per SM (of 256 threads) to aim for
    static __device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
};
template <>
struct Prec<double> {
    static constexpr int NSLOT = 4;
    static constexpr int MINB = 1;
    static __device__ __forceinline__ double recip(double x) { return 1.0 / x; }
};

template <typename T, int TY>
struct Geo {
    static constexpr int NSLOT = Prec<T>::NSLOT;
    static constexpr int RW = T3X + 4, RH = TY + 4, PLANE = RW * RH;
    static constexpr int PLANE_BYTES = ((PLANE * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int RW1 = T3X + 2, RH1 = TY + 2, P1 = RW1 * RH1;
    static constexpr int NRING = 2 * T3X + 2 * RH1;  // one-node ring around the tile
    static constexpr int PLANE_ELEMS = PLANE_BYTES / (int)sizeof(T);
    static constexpr int SD_BYTES = ((NSLOT * P1 * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int BAR_OFFSET = NSLOT * 4 * PLANE_BYTES + SD_BYTES;
    static constexpr int SMEM = BAR_OFFSET + 128;
    static constexpr int NT = T3X * TY / 2;
    static_assert(NRING <= NT, "ring points must fit one pass");
};

// values of the thread's two nodes (a = lower row, b = upper row) on one plane
template <typename T>
struct Col {
    T r[2], u[2], v[2], w[2];
};

// A thread's two nodes (a = lower row, b = upper row) travel as a pair
// V2<T>: float2 for FP32 storage, whose arithmetic is issued as packed FP32
// instructions (FFMA2/FADD2/FMUL2, sm_100 and later), double2 for FP64 (two
// scalar operations).  Every operation is an explicit round-to-nearest
// intrinsic, never contracted by the compiler, so a node's value does not
// depend on where its arithmetic was inlined (z-chunk prologue or loop,
// own node or a neighbour's ring) and a grid split into sub-domains gives
// the same bits as the whole grid.
template <typename T>
struct V2T;
template <>
struct V2T<float> {
    using type = float2;
};
template <>
struct V2T<double> {
    using type = double2;
};
template <typename T>
using V2 = typename V2T<T>::type;

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename T>
__device__ __forceinline__ V2<T> splat(T a)
{
    return mk(a, a);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 add2(double2 a, double2 b)
{
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 mul2(double2 a, double2 b)
{
    return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c)
{
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
// scalar counterparts (ring points of the Delta-rho window)
__device__ __forceinline__ float add1(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul1(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma1(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double add1(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double mul1(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma1(double a, double b, double c) { return __fma_rn(a, b, c); }

// 1 / rho^{n+1}.  FP32: the hardware approximation (1 ulp) suffices, since
// it only scales the increment of u, which is O(Ma^2) relative to u.
__device__ __forceinline__ float recip(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

// coefficient pairs (negated copies where a term is subtracted, so that no
// operand needs negating)
template <typename T>
struct K2 {
    V2<T> rho0, hdt, nhdt, hdtcs2, nhdtcs2, nudt, hsatm, nhsatm, m6, satc, dt, gx, gy, gz;
};

// Eq. (2.10): Delta rho from a node's 7-point neighbourhood (E, W, N, S, U,
// D), the same operation order for a pair and for a single ring node:
//   Delta rho = (1/2 cs^2 dt^2) Lap(rho) - (dt/2) [(m_E + m_N + m_U) - (m_W + m_S + m_D)]
// with m = (rho0 + rho') u_b along each axis b.  GEN = false is the
// instantiation for rho0 = 1 (the paper's reference density) without a body
// force, where m = rho' u + u is one fused multiply-add.
template <bool GEN, typename T>
__device__ __forceinline__ V2<T> delta2(const K2<T> &K, V2<T> rC, V2<T> rE, V2<T> rW, V2<T> rN,
                                        V2<T> rS, V2<T> rU, V2<T> rD, V2<T> uE, V2<T> uW,
                                        V2<T> vN, V2<T> vS, V2<T> wU, V2<T> wD)
{
    V2<T> P, N;
    if (GEN) {
        P = fma2(add2(K.rho0, rE), uE, fma2(add2(K.rho0, rN), vN, mul2(add2(K.rho0, rU), wU)));
        N = fma2(add2(K.rho0, rW), uW, fma2(add2(K.rho0, rS), vS, mul2(add2(K.rho0, rD), wD)));
    } else {
        P = fma2(rE, uE, fma2(rN, vN, fma2(rU, wU, add2(add2(uE, vN), wU))));
        N = fma2(rW, uW, fma2(rS, vS, fma2(rD, wD, add2(add2(uW, vS), wD))));
    }
    const V2<T> lap = fma2(K.m6, rC, add2(add2(add2(rE, rW), add2(rN, rS)), add2(rU, rD)));
    return fma2(K.satc, lap, fma2(K.nhdt, P, mul2(K.hdt, N)));
}
template <bool GEN, typename T>
__device__ __forceinline__ T delta1(const K2<T> &K, T rC, T rE, T rW, T rN, T rS, T rU, T rD,
                                    T uE, T uW, T vN, T vS, T wU, T wD)
{
    const T r0 = K.rho0.x;
    T P, N;
    if (GEN) {
        P = fma1(add1(r0, rE), uE, fma1(add1(r0, rN), vN, mul1(add1(r0, rU), wU)));
        N = fma1(add1(r0, rW), uW, fma1(add1(r0, rS), vS, mul1(add1(r0, rD), wD)));
    } else {
        P = fma1(rE, uE, fma1(rN, vN, fma1(rU, wU, add1(add1(uE, vN), wU))));
        N = fma1(rW, uW, fma1(rS, vS, fma1(rD, wD, add1(add1(uW, vS), wD))));
    }
    const T lap = fma1(K.m6.x, rC, add1(add1(add1(rE, rW), add1(rN, rS)), add1(rU, rD)));
    return fma1(K.satc.x, lap, fma1(K.nhdt.x, P, mul1(K.hdt.x, N)));
}

// Eq. (2.11) for a node pair; arrays in the order C, E, W, N, S, U, D of
// rho', u, v, w and Delta rho.  Differences are split into a positive and a
// negative chain: -hdt (P - N) = fma(-hdt, P, hdt N).  Then
// u^{n+1} = u + (RHS - Delta rho u) / rho^{n+1}.
template <typename T, bool GEN>
__device__ __forceinline__ void node_update2(const V2<T> (&r)[7], const V2<T> (&u)[7],
                                             const V2<T> (&v)[7], const V2<T> (&w)[7],
                                             const V2<T> (&d)[7], const K2<T> &K, V2<T> &rn,
                                             V2<T> &un, V2<T> &vn, V2<T> &wn)
{
    using P2 = V2<T>;
    P2 mx[7], my[7], mz[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        if (GEN) {
            const P2 q = add2(K.rho0, r[k]);
            mx[k] = mul2(q, u[k]);
            my[k] = mul2(q, v[k]);
            mz[k] = mul2(q, w[k]);
        } else {  // rho0 = 1
            mx[k] = fma2(r[k], u[k], u[k]);
            my[k] = fma2(r[k], v[k], v[k]);
            mz[k] = fma2(r[k], w[k], w[k]);
        }
    }
    auto lap = [&](const P2 (&m)[7]) {
        return fma2(K.m6, m[0], add2(add2(add2(m[1], m[2]), add2(m[3], m[4])), add2(m[5], m[6])));
    };
    // R - (dt/2) [twice-centred d_b (m u_b)]
    auto flux = [&](const P2 (&m)[7], P2 R) {
        const P2 P = fma2(m[1], u[1], fma2(m[3], v[3], mul2(m[5], w[5])));
        const P2 N = fma2(m[2], u[2], fma2(m[4], v[4], mul2(m[6], w[6])));
        return fma2(K.nhdt, P, fma2(K.hdt, N, R));
    };
    const P2 rho1 = add2(add2(K.rho0, r[0]), d[0]);
    const P2 inv = mk(recip(rho1.x), recip(rho1.y));
    P2 rx = flux(mx, mul2(K.nudt, lap(mx)));
    P2 ry = flux(my, mul2(K.nudt, lap(my)));
    P2 rz = flux(mz, mul2(K.nudt, lap(mz)));
    rx = fma2(K.nhdtcs2, r[1], fma2(K.hdtcs2, r[2], rx));
    ry = fma2(K.nhdtcs2, r[3], fma2(K.hdtcs2, r[4], ry));
    rz = fma2(K.nhdtcs2, r[5], fma2(K.hdtcs2, r[6], rz));
    rx = fma2(K.nhsatm, d[1], fma2(K.hsatm, d[2], rx));
    ry = fma2(K.nhsatm, d[3], fma2(K.hsatm, d[4], ry));
    rz = fma2(K.nhsatm, d[5], fma2(K.hsatm, d[6], rz));
    if (GEN) {
        const P2 fb = mul2(K.dt, rho1);
        rx = fma2(fb, K.gx, rx);
        ry = fma2(fb, K.gy, ry);
        rz = fma2(fb, K.gz, rz);
    }
    const P2 nd = mk(-d[0].x, -d[0].y);
    un = fma2(fma2(nd, u[0], rx), inv, u[0]);
    vn = fma2(fma2(nd, v[0], ry), inv, v[0]);
    wn = fma2(fma2(nd, w[0], rz), inv, w[0]);
    rn = add2(r[0], d[0]);
}

template <int J>
using IC = std::integral_constant<int, J>;

// z steps J .. N-1 of one pass over the slot ring (slot indices constant in
// each): stops after plane zend-1 or when a step reports an abort
template <int J, int N>
struct Unroll {
    template <typename F>
    __device__ __forceinline__ static bool run(F &step, int zg, int zend)
    {
        if (!step(IC<J>{}, zg) || zg + J + 1 >= zend) return false;
        return Unroll<J + 1, N>::run(step, zg, zend);
    }
};
template <int N>
struct Unroll<N, N> {
    template <typename F>
    __device__ __forceinline__ static bool run(F &, int, int)
    {
        return true;
    }
};

// Write a node's periodic images in the ghost layers (both images exist when
// the grid is narrower than 2 * T3PAD); only the threads on the first/last
// T3PAD columns/rows call it.  Explicit cases, no index arrays (which the
// compiler would place in local memory).
template <typename T>
__device__ __forceinline__ void store_images(Fields<T> out, long long gi, int gx, int gy, int nx,
                                          int ny, long long PX, T rn, T un, T vn, T wn)
{
    auto put = [&](long long off) {
        out.f[F_R][gi + off] = rn;
        out.f[F_U][gi + off] = un;
        out.f[F_V][gi + off] = vn;
        out.f[F_W][gi + off] = wn;
    };
    const bool xl = gx < T3PAD, xr = gx >= nx - T3PAD;
    const bool yl = gy < T3PAD, yr = gy >= ny - T3PAD;
    if (xl) put(nx);
    if (xr) put(-nx);
    if (yl) {
        const long long o = (long long)ny * PX;
        put(o);
        if (xl) put(o + nx);
        if (xr) put(o - nx);
    }
    if (yr) {
        const long long o = -(long long)ny * PX;
        put(o);
        if (xl) put(o + nx);
        if (xr) put(o - nx);
    }
}

template <typename T, int TY, bool GEN>
__global__ void __launch_bounds__(T3X *TY / 2, Prec<T>::MINB * 16 / TY)
    k_step3d(const __grid_constant__ CUtensorMap mr, const __grid_constant__ CUtensorMap mu_,
             const __grid_constant__ CUtensorMap mv, const __grid_constant__ CUtensorMap mw,
             Fields<T> out, const __grid_constant__ RunDesc R, int zc, unsigned *err)
{
    using G = Geo<T, TY>;
    constexpr int NSLOT = G::NSLOT, RW = G::RW, RW1 = G::RW1, PE = G::PLANE_ELEMS, P1 = G::P1;
    extern __shared__ __align__(128) unsigned char smem[];
    T *S = reinterpret_cast<T *>(smem);        // plane (slot s, field f) at (4 s + f) PE
    T *SD = S + NSLOT * 4 * PE;                  // NSLOT Delta-rho windows of P1 (one per plane slot)
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + G::BAR_OFFSET);
    int *s_abort = reinterpret_cast<int *>(bar + NSLOT);

    const int tid = threadIdx.x;
    const int tx = tid & 31, ty2 = tid >> 5;
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int ncx = (nx + T3X - 1) / T3X;
    const int nzc = (nz + zc - 1) / zc;  // chunks per column
    const int nitems = ncx * ((ny + TY - 1) / TY) * nzc;
    if ((int)blockIdx.x >= nitems) return;

    const T *C = coefs<T>(R);
    const T rho0 = C[C_RHO0], dt = C[C_DT], cs2 = C[C_CS2], nudt = C[C_NUDT];
    const T hdt = T(0.5) * dt, hdtcs2 = T(0.5) * dt * cs2;
    const T satc = C[C_SATC], hsatm = T(0.5) * C[C_SATM];
    const T gfx = C[C_GX], gfy = C[C_GY], gfz = C[C_GZ];
    constexpr uint32_t TX_BYTES = 4u * G::PLANE * sizeof(T);
    using P2 = V2<T>;
    const K2<T> K{splat(rho0), splat(hdt),   splat(-hdt),   splat(hdtcs2), splat(-hdtcs2),
                  splat(nudt), splat(hsatm), splat(-hsatm), splat(T(-6)),  splat(satc),
                  splat(dt),   splat(gfx),   splat(gfy),    splat(gfz)};

    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_abort = 0;
    }
    __syncthreads();

    // own nodes: offsets in a plane window and in a Delta-rho window
    const int ya = 2 * ty2;
    const int ca = (ya + 2) * RW + (tx + 2), cb = ca + RW;
    const int da = (ya + 1) * RW1 + (tx + 1), db = da + RW1;
    // ring point of this thread (tid < NRING): offsets in both windows
    int ring_d = -1, ring_c = 0;
    if (tid < G::NRING) {
        int lx, ly;
        if (tid < T3X) { lx = tid + 1; ly = 0; }
        else if (tid < 2 * T3X) { lx = tid - T3X + 1; ly = G::RH1 - 1; }
        else if (tid < 2 * T3X + G::RH1) { lx = 0; ly = tid - 2 * T3X; }
        else { lx = RW1 - 1; ly = tid - 2 * T3X - G::RH1; }
        ring_d = ly * RW1 + lx;
        ring_c = (ly + 1) * RW + (lx + 1);
    }
    const long long PX = R.px, PXY = R.px * R.py;
    P2 fin = splat(T(0));  // running sum of this thread's outputs (non-finite on a blow-up)

    // Every chunk puts plane zbeg-2 in slot 0, so plane p sits in slot
    // (p - zbeg + 2) % NSLOT; the loop below is unrolled by NSLOT so every
    // slot index is a compile-time constant.  Bit s of `phase` is the parity
    // of the next completion of slot s's barrier.
    uint32_t phase = 0;
    auto issue = [&](int s, int p, int x0, int y0) {
        // periodic grids wrap z; a sub-domain reads its ghost planes
        int zw = p + R.zg;
        if (R.zg == 0) {
            zw = p % nz;
            if (zw < 0) zw += nz;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[s], TX_BYTES);
        T *dst = S + s * 4 * PE;
        tma_load_3d(dst, &mr, x0, y0, zw, &bar[s]);
        tma_load_3d(dst + PE, &mu_, x0, y0, zw, &bar[s]);
        tma_load_3d(dst + 2 * PE, &mv, x0, y0, zw, &bar[s]);
        tma_load_3d(dst + 3 * PE, &mw, x0, y0, zw, &bar[s]);
    };
    auto wait = [&](int s) {
        const uint32_t par = (phase >> s) & 1u;
        phase ^= 1u << s;
        for (int it = 0; it < WAIT_LIMIT; ++it)
            if (mbar_try_wait(&bar[s], par)) return;
        *s_abort = 1;
        atomicOr(err, ERR_TIMEOUT);
    };
    auto load_col = [&](int s, Col<T> &q) {
        const T *P = S + s * 4 * PE;
        q.r[0] = P[ca];
        q.r[1] = P[cb];
        q.u[0] = P[PE + ca];
        q.u[1] = P[PE + cb];
        q.v[0] = P[2 * PE + ca];
        q.v[1] = P[2 * PE + cb];
        q.w[0] = P[3 * PE + ca];
        q.w[1] = P[3 * PE + cb];
    };
    // Eq. (2.10) on the plane in slot s0 (slots sm, sp hold planes -1, +1):
    // own nodes from registers + smem, ring from smem; result to window dw.
    auto delta_rho = [&](int sm, int s0, int sp, T *dw, const Col<T> &Cd, const Col<T> &C0,
                         const Col<T> &Cu, T (&dout)[2]) {
        const T *pr = S + s0 * 4 * PE, *pu = pr + PE, *pv = pr + 2 * PE;
        {   // both own nodes at once (lane x: node a, whose N is node b;
            // lane y: node b, whose S is node a)
            const P2 dd = delta2<GEN, T>(K, mk(C0.r[0], C0.r[1]), mk(pr[ca + 1], pr[cb + 1]),
                                    mk(pr[ca - 1], pr[cb - 1]), mk(C0.r[1], pr[cb + RW]),
                                    mk(pr[ca - RW], C0.r[0]), mk(Cu.r[0], Cu.r[1]),
                                    mk(Cd.r[0], Cd.r[1]), mk(pu[ca + 1], pu[cb + 1]),
                                    mk(pu[ca - 1], pu[cb - 1]), mk(C0.v[1], pv[cb + RW]),
                                    mk(pv[ca - RW], C0.v[0]), mk(Cu.w[0], Cu.w[1]),
                                    mk(Cd.w[0], Cd.w[1]));
            dout[0] = dd.x;
            dout[1] = dd.y;
        }
        dw[da] = dout[0];
        dw[db] = dout[1];
        if (ring_d >= 0) {
            const int c = ring_c;
            const T *rd = S + sm * 4 * PE, *wd = rd + 3 * PE;
            const T *ru = S + sp * 4 * PE, *wu = ru + 3 * PE;
            dw[ring_d] = delta1<GEN, T>(K, pr[c], pr[c + 1], pr[c - 1], pr[c + RW], pr[c - RW], ru[c],
                                   rd[c], pu[c + 1], pu[c - 1], pv[c + RW], pv[c - RW], wu[c],
                                   wd[c]);
        }
    };

    Col<T> Q[NSLOT];   // own-node values of the plane held in slot s
    T D[NSLOT][2];     // own-node Delta rho of the plane held in slot s

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        // chunk: column col, planes [zbeg, zend)
        const int col = item / nzc;
        const int zbeg = (item - col * nzc) * zc;
        const int zend = min(zbeg + zc, nz);
        const int x0 = (col % ncx) * T3X, y0 = (col / ncx) * TY;
        const int zlast = zend + 1;  // last plane this chunk needs

        // prologue: planes zbeg-2 .. zbeg+NSLOT-3 into slots 0 .. NSLOT-1
        if (tid == 0)
            for (int k = 0; k < NSLOT && zbeg - 2 + k <= zlast; ++k) issue(k, zbeg - 2 + k, x0, y0);
        for (int k = 0; k < 4; ++k) wait(k);
        __syncthreads();
        if (*s_abort) break;
        load_col(0, Q[0]);
        load_col(1, Q[1]);
        load_col(2, Q[2]);
        load_col(3, Q[3]);
        delta_rho(0, 1, 2, SD + 1 * P1, Q[0], Q[1], Q[2], D[1]);
        delta_rho(1, 2, 3, SD + 2 * P1, Q[1], Q[2], Q[3], D[2]);
        __syncthreads();  // plane zbeg-2 is no longer read
        if (tid == 0 && zbeg + NSLOT - 2 <= zlast) issue(0, zbeg + NSLOT - 2, x0, y0);

        const int gx = x0 + tx, gya = y0 + ya, gyb = gya + 1;
        // CTA-uniform: every node of the tile is inside the grid and none of
        // them has a periodic image in the ghost layers
        const bool plain_tile = x0 >= T3PAD && x0 + T3X <= nx - T3PAD && y0 >= T3PAD &&
                                y0 + TY <= ny - T3PAD;
        const bool own_a = gx < nx && gya < ny, own_b = gx < nx && gyb < ny;
        const bool edge = gx < T3PAD || gx >= nx - T3PAD || gya < T3PAD || gyb >= ny - T3PAD;
        const long long base_a =
            R.off + R.zg * PXY + (long long)(gya + T3PAD) * PX + (gx + T3PAD);
        long long gcur = base_a + (long long)zbeg * PXY;  // storage index of plane z
        auto store2 = [&](long long ga, T ra, T ua, T va, T wa, T rb, T ub, T vb, T wb) {
            if (plain_tile) {
                out.f[F_R][ga] = ra;
                out.f[F_U][ga] = ua;
                out.f[F_V][ga] = va;
                out.f[F_W][ga] = wa;
                out.f[F_R][ga + PX] = rb;
                out.f[F_U][ga + PX] = ub;
                out.f[F_V][ga + PX] = vb;
                out.f[F_W][ga + PX] = wb;
                return;
            }
            if (own_a) {
                out.f[F_R][ga] = ra;
                out.f[F_U][ga] = ua;
                out.f[F_V][ga] = va;
                out.f[F_W][ga] = wa;
                if (edge) store_images<T>(out, ga, gx, gya, nx, ny, PX, ra, ua, va, wa);
            }
            if (own_b) {
                out.f[F_R][ga + PX] = rb;
                out.f[F_U][ga + PX] = ub;
                out.f[F_V][ga + PX] = vb;
                out.f[F_W][ga + PX] = wb;
                if (edge) store_images<T>(out, ga + PX, gx, gyb, nx, ny, PX, rb, ub, vb, wb);
            }
        };

        // one z step for plane z = zg + J, with (zg - zbeg) a multiple of NSLOT
        auto step = [&](auto JC, int zg) {
            constexpr int J = decltype(JC)::value;
            constexpr int SM = (J + 1) % NSLOT, S0 = (J + 2) % NSLOT;  // planes z-1, z
            constexpr int S1 = (J + 3) % NSLOT, S2 = (J + 4) % NSLOT;  // planes z+1, z+2
            const int z = zg + J;
            // One barrier per plane: after it, plane z-1 (slot SM) is free,
            // the Delta-rho window of z (slot S0) written in
            // the previous step is complete, and every wait of the previous
            // step has returned, so the abort flag reads the same in every
            // thread.  Plane z and z+1 were waited for by each thread itself.
            __syncthreads();
            if (*s_abort) return false;
            if (tid == 0 && z + NSLOT - 1 <= zlast) issue(SM, z + NSLOT - 1, x0, y0);
            wait(S2);
            load_col(S2, Q[S2]);
            // harmless on stale data if the wait gave up (checked at the next barrier)
            delta_rho(S0, S1, S2, SD + S1 * P1, Q[S0], Q[S1], Q[S2], D[S1]);

            const T *pr = S + S0 * 4 * PE, *pu = pr + PE, *pv = pr + 2 * PE, *pw = pr + 3 * PE;
            const T *dz = SD + S0 * P1;
            const Col<T> &Xm = Q[SM], &X0 = Q[S0], &Xp = Q[S1];
            const P2 r[7] = {mk(X0.r[0], X0.r[1]), mk(pr[ca + 1], pr[cb + 1]),
                             mk(pr[ca - 1], pr[cb - 1]), mk(X0.r[1], pr[cb + RW]),
                             mk(pr[ca - RW], X0.r[0]), mk(Xp.r[0], Xp.r[1]),
                             mk(Xm.r[0], Xm.r[1])};
            const P2 u[7] = {mk(X0.u[0], X0.u[1]), mk(pu[ca + 1], pu[cb + 1]),
                             mk(pu[ca - 1], pu[cb - 1]), mk(X0.u[1], pu[cb + RW]),
                             mk(pu[ca - RW], X0.u[0]), mk(Xp.u[0], Xp.u[1]),
                             mk(Xm.u[0], Xm.u[1])};
            const P2 v[7] = {mk(X0.v[0], X0.v[1]), mk(pv[ca + 1], pv[cb + 1]),
                             mk(pv[ca - 1], pv[cb - 1]), mk(X0.v[1], pv[cb + RW]),
                             mk(pv[ca - RW], X0.v[0]), mk(Xp.v[0], Xp.v[1]),
                             mk(Xm.v[0], Xm.v[1])};
            const P2 w[7] = {mk(X0.w[0], X0.w[1]), mk(pw[ca + 1], pw[cb + 1]),
                             mk(pw[ca - 1], pw[cb - 1]), mk(X0.w[1], pw[cb + RW]),
                             mk(pw[ca - RW], X0.w[0]), mk(Xp.w[0], Xp.w[1]),
                             mk(Xm.w[0], Xm.w[1])};
            const P2 d[7] = {mk(D[S0][0], D[S0][1]), mk(dz[da + 1], dz[db + 1]),
                             mk(dz[da - 1], dz[db - 1]), mk(D[S0][1], dz[db + RW1]),
                             mk(dz[da - RW1], D[S0][0]), mk(D[S1][0], D[S1][1]),
                             mk(D[SM][0], D[SM][1])};
            P2 rn, un, vn, wn;
            node_update2<T, GEN>(r, u, v, w, d, K, rn, un, vn, wn);
            {   // blow-up check on the nodes inside the grid: a running sum
                const P2 c2 = add2(add2(rn, un), add2(vn, wn));
                fin = add2(fin, plain_tile ? c2 : mk(own_a ? c2.x : T(0), own_b ? c2.y : T(0)));
            }
            store2(gcur, rn.x, un.x, vn.x, wn.x, rn.y, un.y, vn.y, wn.y);
            gcur += PXY;
            return true;
        };

        for (int zg = zbeg; zg < zend; zg += NSLOT)
            if (!Unroll<0, NSLOT>::run(step, zg, zend)) break;
        __syncthreads();  // every read of this chunk's planes is done
        if (*s_abort) break;
    }
    const bool bad = !isfinite(add1(fin.x, fin.y));
    if (__syncthreads_or(bad) && tid == 0) atomicOr(err, ERR_NONFINITE);
}

template <typename T, int TY, bool GEN>
int max_blocks_g()
{
    static int cached = -1;
    if (cached < 0) {
        using G = Geo<T, TY>;
        cudaFuncSetAttribute(k_step3d<T, TY, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G::SMEM);
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step3d<T, TY, GEN>, G::NT,
                                                          G::SMEM) != cudaSuccess)
            nb = 1;
        cached = nb > 0 ? nb : 1;
    }
    return cached;
}

template <typename T, int TY>
int max_blocks()
{
    max_blocks_g<T, TY, true>();
    return max_blocks_g<T, TY, false>();
}

template <typename T, int TY>
cudaError_t launch(const CUtensorMap *m, Fields<T> out, const RunDesc &run, unsigned *derr,
                   int zchunks, int sms, cudaStream_t s)
{
    using G = Geo<T, TY>;
    // the fast instantiation covers rho0 = 1 without a body force
    const bool gen = run.g[0] != 0.0 || run.g[1] != 0.0 || run.g[2] != 0.0 || run.rho0 != 1.0;
    const int per_sm = gen ? max_blocks_g<T, TY, true>() : max_blocks_g<T, TY, false>();
    // chunks of zc planes; by default 16 (short enough for many CTAs, long
    // enough that the 4 extra planes per chunk cost little)
    const int nzc = zchunks > 0 ? std::min(zchunks, run.nz) : std::max(1, (run.nz + 15) / 16);
    const int zc = (run.nz + nzc - 1) / nzc;
    const long long items = (long long)((run.nx + T3X - 1) / T3X) * ((run.ny + TY - 1) / TY) *
                            ((run.nz + zc - 1) / zc);
    // persistent CTAs walk the chunks in (column, z-chunk) order, so CTAs
    // resident together work on neighbouring columns at the same depths and
    // share their halo planes through L2
    const long long grid = std::min<long long>(items, (long long)sms * per_sm);
    if (gen)
        k_step3d<T, TY, true><<<(unsigned)grid, G::NT, G::SMEM, s>>>(m[0], m[1], m[2], m[3], out,
                                                                    run, zc, derr);
    else
        k_step3d<T, TY, false><<<(unsigned)grid, G::NT, G::SMEM, s>>>(m[0], m[1], m[2], m[3], out,
                                                                     run, zc, derr);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
int step3d_max_blocks_per_sm(int t3y)
{
    return t3y == 8 ? max_blocks<T, 8>() : max_blocks<T, 16>();
}

template <typename T>
cudaError_t launch_step3d(const CUtensorMap *maps_in, Fields<T> out, const RunDesc &run,
                          unsigned *derr, int zchunks, int t3y, int sms, cudaStream_t s)
{
    if (t3y == 8) return launch<T, 8>(maps_in, out, run, derr, zchunks, sms, s);
    return launch<T, 16>(maps_in, out, run, derr, zchunks, sms, s);
}

template cudaError_t launch_step3d<float>(const CUtensorMap *, Fields<float>, const RunDesc &,
                                          unsigned *, int, int, int, cudaStream_t);
template cudaError_t launch_step3d<double>(const CUtensorMap *, Fields<double>, const RunDesc &,
                                           unsigned *, int, int, int, cudaStream_t);
template int step3d_max_blocks_per_sm<float>(int);
template int step3d_max_blocks_per_sm<double>(int);

}  // namespace acm
