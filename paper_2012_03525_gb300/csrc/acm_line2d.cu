// Fused 2D time step of the simplified MAME scheme (Huang, arXiv:2012.03525,
// Section 2, Eqs. 2.10-2.11), single phase, periodic in x and y: the line-
// marching form used for grids whose width is a multiple of 64.
//
// Design (one kernel per step, no barriers: every warp works alone):
//   * A work item is a strip of 64 columns x up to 32 rows of one run; one
//     warp owns it and marches along y.  Lane l owns the x-adjacent node
//     pair (x0 + 2l, x0 + 2l + 1): its fields are read and written as one
//     8-byte (FP32) / 16-byte (FP64) access, so a warp moves 256 (512)
//     contiguous bytes per field and row, and its arithmetic on the pair is
//     issued as packed two-lane FP32 instructions (FFMA2/FADD2/FMUL2).
//   * x-neighbours come from the adjacent lanes by warp shuffles; the two
//     lanes at the strip edges also read the node pair just outside the strip
//     (x0 - 2, x0 - 1 and x0 + 64, x0 + 65, wrapped periodically).
//   * Rows are prefetched by cp.async into a ring of LRING row slots in
//     shared memory, private to the warp (each lane copies and later reads
//     only its own pair, so no barrier is needed); the copies of a row form
//     one commit group, and a lane waits for the group of the row it needs
//     next while the next LAHEAD - 2 rows are still in flight, so memory
//     latency overlaps several rows of arithmetic.
//   * y-neighbours stay in registers: rows y-1 .. y+2 of the pair form a
//     queue, advanced one row per step; the edge lanes read their outside
//     pairs from the ring where they are used.
//   * Eq. (2.10) is evaluated one row ahead (row y+1) for the own pair and,
//     in the two edge lanes, for the node just outside the strip, so that
//     d_a rho^{n+1} - d_a rho^n of Eq. (2.11) is a centred difference of
//     Delta rho with every value on chip; Eq. (2.11) then updates row y:
//     u^{n+1} = u + (RHS - Delta rho u) / rho^{n+1}.
//   * Each warp ORs whether its outputs are finite (the running sum of the
//     pair's new values is finite only if each is) into the error word.
// Storage is the plain 2D layout (x fastest, row pitch nx); a run starts on
// a 256-byte boundary and nx is a multiple of 64, so every pair access is
// aligned.
#include <type_traits>

#include "acm_internal.h"
#include "acm_pair.h"

namespace acm {
namespace {

using namespace pair;

constexpr int LW = 64;      // columns per strip
constexpr int LROWS = 32;   // rows per work item (at most)
#ifndef ACM_LINE2D_WARPS
#define ACM_LINE2D_WARPS 8
#endif
#ifndef ACM_LINE2D_RING
#define ACM_LINE2D_RING 8
#endif
constexpr int LWARPS = ACM_LINE2D_WARPS;  // independent warps per CTA
constexpr int LRING = ACM_LINE2D_RING;    // row slots of a warp's prefetch ring (power of 2)
static_assert((LRING & (LRING - 1)) == 0 && LRING >= 8, "ring of 8, 16, ... slots");
constexpr int LAHEAD = LRING - 3; // step y issues row y + LAHEAD (3 rows beyond row y+2, read now)
#ifndef ACM_LINE2D_MINB
#define ACM_LINE2D_MINB 2
#endif
constexpr int LMINB = ACM_LINE2D_MINB;  // FP32: CTAs per SM to aim for (register budget)

// shared memory of one warp: LRING rows x 3 fields x 32 lanes own pairs, then
// LRING rows x 3 fields x 2 edge pairs
constexpr int RING_ELEMS = LRING * 3 * 32 * 2 + LRING * 3 * 2 * 2;

template <typename T>
__device__ __forceinline__ void cp_async_pair(T *dst, const T *src)
{
    cp_async<2 * sizeof(T)>(dst, src);
}

// coefficient pairs of one run (negated copies where a term is subtracted)
template <typename T>
struct K2 {
    P2<T> rho0, hdt, nhdt, hdtcs2, nhdtcs2, nudt, hsatm, nhsatm, m4, satc, dt, gx, gy;
};

// one row of the strip: the lane's own pair (the edge pairs stay in the
// ring and are read where they are used)
template <typename T>
struct Row {
    P2<T> r, u, v;
};

// x-neighbours of the own pair from the adjacent lanes: W = (west of a, a),
// E = (b, east of b)
template <typename T>
__device__ __forceinline__ void neighbours(P2<T> p, P2<T> h, int lane, P2<T> &W, P2<T> &E)
{
    const T up = __shfl_up_sync(FULL, p.y, 1);
    const T dn = __shfl_down_sync(FULL, p.x, 1);
    W = mk(lane == 0 ? h.y : up, p.x);
    E = mk(p.y, lane == 31 ? h.x : dn);
}

// Eq. (2.10) for a node pair:
//   Delta rho = (1/2 cs^2 dt^2) Lap(rho) - (dt/2) [(m_E + m_N) - (m_W + m_S)]
// with m = (rho0 + rho') u_b along each axis b; GEN = false: rho0 = 1 and
// m = rho' u + u (one fused multiply-add)
template <bool GEN, typename T>
__device__ __forceinline__ P2<T> delta2(const K2<T> &K, P2<T> rC, P2<T> rE, P2<T> rW, P2<T> rN,
                                        P2<T> rS, P2<T> uE, P2<T> uW, P2<T> vN, P2<T> vS)
{
    P2<T> P, N;
    if (GEN) {
        P = fma2(add2(K.rho0, rE), uE, mul2(add2(K.rho0, rN), vN));
        N = fma2(add2(K.rho0, rW), uW, mul2(add2(K.rho0, rS), vS));
    } else {
        P = fma2(rE, uE, fma2(rN, vN, add2(uE, vN)));
        N = fma2(rW, uW, fma2(rS, vS, add2(uW, vS)));
    }
    const P2<T> lap = fma2(K.m4, rC, add2(add2(rE, rW), add2(rN, rS)));
    return fma2(K.satc, lap, fma2(K.nhdt, P, mul2(K.hdt, N)));
}
// the same for one node (the edge lanes' node outside the strip)
template <bool GEN, typename T>
__device__ __forceinline__ T delta1(const K2<T> &K, T rC, T rE, T rW, T rN, T rS, T uE, T uW,
                                    T vN, T vS)
{
    const T r0 = K.rho0.x;
    T P, N;
    if (GEN) {
        P = fma1(add1(r0, rE), uE, mul1(add1(r0, rN), vN));
        N = fma1(add1(r0, rW), uW, mul1(add1(r0, rS), vS));
    } else {
        P = fma1(rE, uE, fma1(rN, vN, add1(uE, vN)));
        N = fma1(rW, uW, fma1(rS, vS, add1(uW, vS)));
    }
    const T lap = fma1(K.m4.x, rC, add1(add1(rE, rW), add1(rN, rS)));
    return fma1(K.satc.x, lap, fma1(K.nhdt.x, P, mul1(K.hdt.x, N)));
}

template <int J>
using IC = std::integral_constant<int, J>;

// steps J .. N-1 of one pass over the 4-row queue (slot indices constant in
// each); stops after row `rows - 1` of the item
template <int J, int N>
struct Unroll {
    template <typename F>
    __device__ __forceinline__ static void run(F &step, int base, int rows)
    {
        if (base + J >= rows) return;
        step(IC<J>{}, base);
        Unroll<J + 1, N>::run(step, base, rows);
    }
};
template <int N>
struct Unroll<N, N> {
    template <typename F>
    __device__ __forceinline__ static void run(F &, int, int)
    {
    }
};

template <typename T, bool GEN>
__global__ void __launch_bounds__(32 * LWARPS, sizeof(T) == 4 ? LMINB : 1)
    k_line2d(const RunDesc *__restrict__ runs, const int4 *__restrict__ work, int nwork,
             Fields<T> in, Fields<T> out, unsigned *err)
{
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * LWARPS + (threadIdx.x >> 5);
    if (item >= nwork) return;  // warp-uniform: the warp has no work item
    const int4 wk = work[item];
    const RunDesc &R = runs[wk.x];
    const int nx = R.nx, ny = R.ny;
    const int x0 = wk.y, y0 = wk.z, rows = wk.w;
    const T *C = coefs<T>(R);
    const T dt = C[C_DT], hdt = T(0.5) * dt, hdtcs2 = T(0.5) * dt * C[C_CS2];
    const T hsatm = T(0.5) * C[C_SATM];
    const K2<T> K{splat(C[C_RHO0]), splat(hdt),       splat(-hdt),     splat(hdtcs2),
                  splat(-hdtcs2),  splat(C[C_NUDT]),  splat(hsatm),    splat(-hsatm),
                  splat(T(-4)),    splat(C[C_SATC]),  splat(dt),       splat(C[C_GX]),
                  splat(C[C_GY])};
    const T *gr = in.f[F_R] + R.off, *gu = in.f[F_U] + R.off, *gv = in.f[F_V] + R.off;
    const int xa = x0 + 2 * lane;
    // edge pair column: lane 0 west of the strip, lane 31 east (periodic)
    const bool edge = lane == 0 || lane == 31;
    int xh = lane == 0 ? x0 - 2 : x0 + LW;
    if (xh < 0) xh += nx;
    else if (xh >= nx) xh -= nx;
    const bool L0 = lane == 0;

    // the warp's ring: own pair of (slot k, field f) at ring + ((k*3 + f)*32 + lane)*2,
    // edge pair at hring + ((k*3 + f)*2 + (lane == 31))*2
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw) + (threadIdx.x >> 5) * RING_ELEMS;
    T *hring = ring + LRING * 3 * 32 * 2;
    T *own_slot = ring + lane * 2;
    T *edge_slot = hring + (lane == 31 ? 2 : 0);
    const int last = y0 + rows + 1;  // last row the item reads

    auto wrapy = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };
    // prefetch row y (rows past `last` are not needed: an empty group keeps
    // the group count uniform)
    auto issue_row = [&](int y) {
        if (y <= last) {
            const int k = (y - y0 + 2) & (LRING - 1);
            const long long o = (long long)wrapy(y) * nx;
            cp_async_pair(own_slot + (k * 3 + 0) * 64, gr + o + xa);
            cp_async_pair(own_slot + (k * 3 + 1) * 64, gu + o + xa);
            cp_async_pair(own_slot + (k * 3 + 2) * 64, gv + o + xa);
            if (edge) {
                cp_async_pair(edge_slot + (k * 3 + 0) * 4, gr + o + xh);
                cp_async_pair(edge_slot + (k * 3 + 1) * 4, gu + o + xh);
                cp_async_pair(edge_slot + (k * 3 + 2) * 4, gv + o + xh);
            }
        }
        cp_async_commit();
    };
    // read row y's own pair from its slot (its group has completed)
    auto read_row = [&](int y, Row<T> &q) {
        const int k = (y - y0 + 2) & (LRING - 1);
        q.r = *reinterpret_cast<const P2<T> *>(own_slot + (k * 3 + 0) * 64);
        q.u = *reinterpret_cast<const P2<T> *>(own_slot + (k * 3 + 1) * 64);
        q.v = *reinterpret_cast<const P2<T> *>(own_slot + (k * 3 + 2) * 64);
    };
    // edge pair of field f of row y (meaningful in lanes 0 and 31; the other
    // lanes read lane 0's slot and ignore it)
    auto edge_of = [&](int y, int f) {
        const int k = (y - y0 + 2) & (LRING - 1);
        return *reinterpret_cast<const P2<T> *>(edge_slot + (k * 3 + f) * 4);
    };
    // Eq. (2.10) on row y of (q0, q1, q2) = rows (y-1, y, y+1): the own pair
    // into d, the edge lanes' outside node into dh
    auto delta_row = [&](int y, const Row<T> &q0, const Row<T> &q1, const Row<T> &q2, P2<T> &d,
                         T &dh) {
        const P2<T> h1r = edge_of(y, 0), h1u = edge_of(y, 1);
        P2<T> rW, rE, uW, uE;
        neighbours<T>(q1.r, h1r, lane, rW, rE);
        neighbours<T>(q1.u, h1u, lane, uW, uE);
        d = delta2<GEN, T>(K, q1.r, rE, rW, q2.r, q0.r, uE, uW, q2.v, q0.v);
        // outside node: lane 0 at x0-1 (W x0-2, E x0), lane 31 at x0+64
        // (W x0+63, E x0+65); N and S from the edge pairs of rows y+1, y-1
        const P2<T> h2r = edge_of(y + 1, 0), h0r = edge_of(y - 1, 0);
        const P2<T> h2v = edge_of(y + 1, 2), h0v = edge_of(y - 1, 2);
        const T c = L0 ? h1r.y : h1r.x;
        const T e = L0 ? q1.r.x : h1r.y, w = L0 ? h1r.x : q1.r.y;
        const T ue = L0 ? q1.u.x : h1u.y, uw = L0 ? h1u.x : q1.u.y;
        const T n = L0 ? h2r.y : h2r.x, s = L0 ? h0r.y : h0r.x;
        const T vn = L0 ? h2v.y : h2v.x, vs = L0 ? h0v.y : h0v.x;
        dh = delta1<GEN, T>(K, c, e, w, n, s, ue, uw, vn, vs);
    };

    Row<T> Q[4];     // rows y-1 .. y+2 of the step in slots (J+1 .. J+4) & 3
    P2<T> D[4];      // own-pair Delta rho of those rows
    T DH[4];         // edge lanes' outside-node Delta rho
    // prologue: rows y0-2 .. y0+LAHEAD-1 in flight; rows y0-2 .. y0+1 into
    // queue slots 0 .. 3; Delta rho of y0-1, y0
    for (int k = 0; k < LAHEAD + 2; ++k) issue_row(y0 - 2 + k);  // rows y0-2 .. y0+LAHEAD-1
    cp_async_wait<LAHEAD - 2>();  // groups of rows y0-2 .. y0+1 complete
    read_row(y0 - 2, Q[0]);
    read_row(y0 - 1, Q[1]);
    read_row(y0, Q[2]);
    read_row(y0 + 1, Q[3]);
    delta_row(y0 - 1, Q[0], Q[1], Q[2], D[1], DH[1]);
    delta_row(y0, Q[1], Q[2], Q[3], D[2], DH[2]);

    T *orr = out.f[F_R] + R.off, *ou = out.f[F_U] + R.off, *ov = out.f[F_V] + R.off;
    P2<T> acc = splat(T(0));

    // row y = y0 + base + J: slots SM = y-1, S0 = y, S1 = y+1, S2 = y+2
    auto step = [&](auto JC, int base) {
        constexpr int J = decltype(JC)::value;
        constexpr int SM = (J + 1) & 3, S0 = (J + 2) & 3, S1 = (J + 3) & 3, S2 = J & 3;
        const int y = y0 + base + J;
        // groups issued so far: rows y0-2 .. y+LAHEAD-1; row y+2's group is
        // complete once at most LAHEAD - 3 newer ones are pending.  Then row
        // y+LAHEAD goes into the slot of row y+LAHEAD-LRING = y-3, which was
        // read into registers five steps ago.
        cp_async_wait<LAHEAD - 3>();
        read_row(y + 2, Q[S2]);
        issue_row(y + LAHEAD);
        delta_row(y + 1, Q[S0], Q[S1], Q[S2], D[S1], DH[S1]);

        // Eq. (2.11) on row y
        const Row<T> &c = Q[S0], &n = Q[S1], &s = Q[SM];
        P2<T> rW, rE, uW, uE, vW, vE, dW, dE;
        neighbours<T>(c.r, edge_of(y, 0), lane, rW, rE);
        neighbours<T>(c.u, edge_of(y, 1), lane, uW, uE);
        neighbours<T>(c.v, edge_of(y, 2), lane, vW, vE);
        {
            const P2<T> d0 = D[S0];
            const T up = __shfl_up_sync(FULL, d0.y, 1);
            const T dn = __shfl_down_sync(FULL, d0.x, 1);
            dW = mk(L0 ? DH[S0] : up, d0.x);
            dE = mk(d0.y, lane == 31 ? DH[S0] : dn);
        }
        // momenta m = (rho0 + rho') u of C, E, W, N, S
        P2<T> mx[5], my[5];
        const P2<T> rr[5] = {c.r, rE, rW, n.r, s.r};
        const P2<T> uu[5] = {c.u, uE, uW, n.u, s.u};
        const P2<T> vv[5] = {c.v, vE, vW, n.v, s.v};
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (GEN) {
                const P2<T> q = add2(K.rho0, rr[k]);
                mx[k] = mul2(q, uu[k]);
                my[k] = mul2(q, vv[k]);
            } else {
                mx[k] = fma2(rr[k], uu[k], uu[k]);
                my[k] = fma2(rr[k], vv[k], vv[k]);
            }
        }
        auto lap = [&](const P2<T> (&m)[5]) {
            return fma2(K.m4, m[0], add2(add2(m[1], m[2]), add2(m[3], m[4])));
        };
        // R - (dt/2) [centred d_b (m u_b)]: P the E/N terms, N the W/S terms
        auto flux = [&](const P2<T> (&m)[5], P2<T> Rt) {
            const P2<T> P = fma2(m[1], uu[1], mul2(m[3], vv[3]));
            const P2<T> N = fma2(m[2], uu[2], mul2(m[4], vv[4]));
            return fma2(K.nhdt, P, fma2(K.hdt, N, Rt));
        };
        const P2<T> d0 = D[S0];
        const P2<T> rho1 = add2(add2(K.rho0, c.r), d0);
        const P2<T> inv = mk(recip(rho1.x), recip(rho1.y));
        P2<T> rx = flux(mx, mul2(K.nudt, lap(mx)));
        P2<T> ry = flux(my, mul2(K.nudt, lap(my)));
        rx = fma2(K.nhdtcs2, rE, fma2(K.hdtcs2, rW, rx));
        ry = fma2(K.nhdtcs2, n.r, fma2(K.hdtcs2, s.r, ry));
        rx = fma2(K.nhsatm, dE, fma2(K.hsatm, dW, rx));
        ry = fma2(K.nhsatm, D[S1], fma2(K.hsatm, D[SM], ry));
        if (GEN) {
            const P2<T> fb = mul2(K.dt, rho1);
            rx = fma2(fb, K.gx, rx);
            ry = fma2(fb, K.gy, ry);
        }
        const P2<T> nd = mk(-d0.x, -d0.y);
        const P2<T> un = fma2(fma2(nd, c.u, rx), inv, c.u);
        const P2<T> vn = fma2(fma2(nd, c.v, ry), inv, c.v);
        const P2<T> rn = add2(c.r, d0);
        const long long o = (long long)y * nx + xa;
        *reinterpret_cast<P2<T> *>(orr + o) = rn;
        *reinterpret_cast<P2<T> *>(ou + o) = un;
        *reinterpret_cast<P2<T> *>(ov + o) = vn;
        acc = add2(acc, add2(add2(rn, un), vn));
    };
    for (int base = 0; base < rows; base += 4) Unroll<0, 4>::run(step, base, rows);
    cp_async_wait<0>();  // no copy in flight at exit
    // a NaN or infinity in any output makes the running sum non-finite
    const bool bad = !isfinite(add1(acc.x, acc.y));
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, ERR_NONFINITE);
}

}  // namespace

int line2d_rows() { return LROWS; }
int line2d_width() { return LW; }

template <typename T>
void line2d_prepare()
{
    const int smem = (int)(LWARPS * RING_ELEMS * sizeof(T));
    cudaFuncSetAttribute(k_line2d<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_line2d<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
#ifdef ACM_LINE2D_CARVE
    cudaFuncSetAttribute(k_line2d<T, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         ACM_LINE2D_CARVE);
    cudaFuncSetAttribute(k_line2d<T, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         ACM_LINE2D_CARVE);
#endif
}

template <typename T>
cudaError_t launch_line2d(const RunDesc *druns, const int4 *dwork, int nwork, bool gen,
                          Fields<T> in, Fields<T> out, unsigned *derr, cudaStream_t s)
{
    if (nwork <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((nwork + LWARPS - 1) / LWARPS);
    const size_t smem = (size_t)LWARPS * RING_ELEMS * sizeof(T);
    if (gen)
        k_line2d<T, true><<<grid, 32 * LWARPS, smem, s>>>(druns, dwork, nwork, in, out, derr);
    else
        k_line2d<T, false><<<grid, 32 * LWARPS, smem, s>>>(druns, dwork, nwork, in, out, derr);
    return cudaGetLastError();
}

template void line2d_prepare<float>();
template void line2d_prepare<double>();
template cudaError_t launch_line2d<float>(const RunDesc *, const int4 *, int, bool, Fields<float>,
                                          Fields<float>, unsigned *, cudaStream_t);
template cudaError_t launch_line2d<double>(const RunDesc *, const int4 *, int, bool,
                                           Fields<double>, Fields<double>, unsigned *,
                                           cudaStream_t);

}  // namespace acm
