// Fused 2D two-phase time step (Huang, arXiv:2012.03525, Section 2:
// Eqs. 2.10-2.11 with F_ST = -phi grad mu and Heun's RK2 step of the
// Cahn-Hilliard Eq. 2.14, u^n frozen, mu recomputed from phi*), line-
// marching form for runs periodic on all four faces.
//
// Design (one kernel per step, no barriers: every warp works alone):
//   * A work item is a strip of one run: the warp holds 64 columns
//     x0 .. x0+63 (lane l the pair x0+2l, x0+2l+1, each node wrapped
//     periodically) and marches along y.  The D2Q9 operators take their x
//     neighbours from the adjacent lanes by shuffles; no lane special-cases
//     the strip edge.  Instead every stage of the step (mu^n, phi*, mu*,
//     phi^{n+1}) is valid on one node fewer at each end than the stage it
//     reads, so after the four stages lanes 2 .. 29 (56 columns, x0+4 ..
//     x0+59) hold correct values: strips start every 56 columns and write
//     those only.
//   * Along y the stages form a pipeline: at row y the warp reads phi of row
//     y+4 and rho', u, v of row y+2, computes mu^n(y+3), Delta rho(y+1) (Eq.
//     2.10), phi*(y+2), mu*(y+1) and then the new state of row y (Eq. 2.11
//     with F_ST, the second Heun stage).  Computed rows live in register
//     queues of five rows (the loop is unrolled by five so slot indices are
//     constants); the march starts TLEAD rows before the item so the queues
//     are full when its first row is written.
//   * Rows are prefetched by cp.async into per-warp rings in shared memory
//     (each lane copies and later reads only its own pair), TAHEAD rows
//     ahead of the rows being read.
//   * Each warp ORs whether its written outputs are finite into the error
//     word.
// The D2Q9-weighted operators (c_s^2 = 1/3): Lap f = (2/3) sum_axis (f_i -
// f_0) + (1/6) sum_diag (f_i - f_0); d_x f = (1/3)(f_E - f_W) + (1/12)
// ((f_NE - f_NW) + (f_SE - f_SW)), d_y likewise.
#include <type_traits>

#include "acm_internal.h"
#include "acm_pair.h"

namespace acm {
namespace {

using namespace pair;

constexpr int TW = 64;       // columns held per strip (32 lanes x 2)
constexpr int TOUT = 56;     // columns written per strip (lanes 2 .. 29)
constexpr int TROWS = 64;    // rows per work item (at most)
#ifndef ACM_LINE2D_TP_WARPS
#define ACM_LINE2D_TP_WARPS 4
#endif
#ifndef ACM_LINE2D_TP_MINB
#define ACM_LINE2D_TP_MINB 2
#endif
constexpr int TWARPS = ACM_LINE2D_TP_WARPS;  // independent warps per CTA
constexpr int TMINB = ACM_LINE2D_TP_MINB;    // FP32: CTAs per SM to aim for (register budget)
constexpr int TRING = 8;     // row slots of the rho', u, v ring (power of 2)
constexpr int TRINGP = 16;   // row slots of the phi ring (rows y .. y+4 stay readable)
constexpr int TAHEAD = 4;    // rows prefetched beyond the rows read at a step
constexpr int TLEAD = 8;     // rows the march runs before the item's first row
constexpr int TQ = 5;        // register queue period

// per warp: ring of rho', u, v rows, then ring of phi rows; [slot][field][lane][2]
constexpr int RUV_ELEMS = TRING * 3 * 64;
constexpr int PHI_ELEMS = TRINGP * 64;
constexpr int TRING_ELEMS = RUV_ELEMS + PHI_ELEMS;

template <typename T>
struct K2 {
    P2<T> rho0, hdt, hdtcs2, nudt, hsatm, satc, dt, gx, gy;
    P2<T> a4, nkappa, mob, ndt, bqa, bqb;
};

template <typename T>
struct Iso {
    P2<T> lap, gx, gy;
};

// D2Q9 operators at the pair of row c from rows s (y-1), c, n (y+1)
template <typename T>
__device__ __forceinline__ Iso<T> iso(P2<T> s, P2<T> c, P2<T> n)
{
    P2<T> sW, sE, cW, cE, nW, nE;
    shuffle_we<T>(s, sW, sE);
    shuffle_we<T>(c, cW, cE);
    shuffle_we<T>(n, nW, nE);
    const P2<T> axis = add2(add2(sub2(cE, c), sub2(cW, c)), add2(sub2(n, c), sub2(s, c)));
    const P2<T> diag = add2(add2(sub2(nE, c), sub2(nW, c)), add2(sub2(sE, c), sub2(sW, c)));
    Iso<T> r;
    r.lap = fma2(splat(T(2.0 / 3.0)), axis, mul2(splat(T(1.0 / 6.0)), diag));
    r.gx = fma2(splat(T(1.0 / 3.0)), sub2(cE, cW),
                mul2(splat(T(1.0 / 12.0)), add2(sub2(nE, nW), sub2(sE, sW))));
    r.gy = fma2(splat(T(1.0 / 3.0)), sub2(n, s),
                mul2(splat(T(1.0 / 12.0)), add2(sub2(nE, sE), sub2(nW, sW))));
    return r;
}

// mu = 4 a phi (phi^2 - 1) - kappa Lap(phi)
template <typename T>
__device__ __forceinline__ P2<T> chem_pot(const K2<T> &K, P2<T> s, P2<T> c, P2<T> n)
{
    const Iso<T> o = iso<T>(s, c, n);
    const P2<T> t = fma2(c, c, splat(T(-1)));
    return fma2(mul2(K.a4, c), t, mul2(K.nkappa, o.lap));
}

template <int J>
using IC = std::integral_constant<int, J>;

template <int J, int N>
struct Unroll {
    template <typename F>
    __device__ __forceinline__ static void run(F &step, int base, int steps)
    {
        if (base + J >= steps) return;
        step(IC<J>{}, base);
        Unroll<J + 1, N>::run(step, base, steps);
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
__global__ void __launch_bounds__(32 * TWARPS, sizeof(T) == 4 ? TMINB : 1)
    k_line2d_tp(const RunDesc *__restrict__ runs, const int4 *__restrict__ work, int nwork,
                Fields<T> in, Fields<T> out, unsigned *err)
{
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * TWARPS + (threadIdx.x >> 5);
    if (item >= nwork) return;  // warp-uniform
    const int4 wk = work[item];
    const RunDesc &R = runs[wk.x];
    const int nx = R.nx, ny = R.ny;
    const int x0 = wk.y, y0 = wk.z, rows = wk.w;
    const T *C = coefs<T>(R);
    const T dt = C[C_DT], hdt = T(0.5) * dt, hdtcs2 = T(0.5) * dt * C[C_CS2];
    const T hsatm = T(0.5) * C[C_SATM];
    const K2<T> K{splat(C[C_RHO0]),     splat(hdt),          splat(hdtcs2),
                  splat(C[C_NUDT]),     splat(hsatm),        splat(C[C_SATC]),
                  splat(dt),            splat(C[C_GX]),      splat(C[C_GY]),
                  splat(T(4) * C[C_A]), splat(-C[C_KAPPA]),  splat(C[C_M]),
                  splat(-dt),           splat(C[C_BQA]),     splat(C[C_BQB])};
    const long long off = R.off;

    // the lane's two columns, wrapped (x0 may be -4)
    auto wrapx = [&](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
    const int xa = wrapx(x0 + 2 * lane), xb = wrapx(x0 + 2 * lane + 1);
    auto wrapy = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ruv = reinterpret_cast<T *>(smem_raw) + (threadIdx.x >> 5) * TRING_ELEMS + lane * 2;
    T *phr = ruv + RUV_ELEMS;

    const int ys = y0 - TLEAD;           // first row of the march
    const int steps = TLEAD + rows;      // rows ys .. y0+rows-1
    const int phi_last = y0 + rows + 3;  // last phi row read
    const int ruv_first = y0 - 2, ruv_last = y0 + rows + 1;
    // prefetch group of step y: phi row y+4+TAHEAD, rho'/u/v row y+2+TAHEAD
    auto issue = [&](int y) {
        const int rp = y + 4 + TAHEAD, rr = y + 2 + TAHEAD;
        if (rp <= phi_last) {
            const long long o = (long long)wrapy(rp) * nx;
            T *d = phr + (rp & (TRINGP - 1)) * 64;
            cp_async<sizeof(T)>(d, in.f[F_PHI] + off + o + xa);
            cp_async<sizeof(T)>(d + 1, in.f[F_PHI] + off + o + xb);
        }
        if (rr >= ruv_first && rr <= ruv_last) {
            const long long o = (long long)wrapy(rr) * nx;
            T *d = ruv + (rr & (TRING - 1)) * 192;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                cp_async<sizeof(T)>(d + f * 64, in.f[f] + off + o + xa);
                cp_async<sizeof(T)>(d + f * 64 + 1, in.f[f] + off + o + xb);
            }
        }
        cp_async_commit();
    };
    auto phi_row = [&](int r) {
        return *reinterpret_cast<const P2<T> *>(phr + (r & (TRINGP - 1)) * 64);
    };
    auto ruv_row = [&](int r, int f) {
        return *reinterpret_cast<const P2<T> *>(ruv + (r & (TRING - 1)) * 192 + f * 64);
    };
    // phi rows ys+4 .. ys+3+TAHEAD and rho'/u/v rows ys+2 .. ys+1+TAHEAD in
    // flight before the first step (the groups of "steps" ys-TAHEAD .. ys-1)
    for (int k = -TAHEAD; k < 0; ++k) issue(ys + k);

    P2<T> MU[TQ], PS[TQ], MS[TQ], D[TQ];  // computed rows r in slot (r - ys) mod 5
#pragma unroll
    for (int k = 0; k < TQ; ++k) MU[k] = PS[k] = MS[k] = D[k] = splat(T(0));

    const bool own = lane >= 2 && lane < 30;
    const int oxa = x0 + 2 * lane, oxb = oxa + 1;  // written columns (not wrapped)
    const bool wa = own && oxa < nx, wb = own && oxb < nx;
    P2<T> acc = splat(T(0));

    auto step = [&](auto JC, int base) {
        constexpr int J = decltype(JC)::value;
        // slot of row y + k
        constexpr int Q0 = J % TQ, Q1 = (J + 1) % TQ, Q2 = (J + 2) % TQ, Q3 = (J + 3) % TQ,
                      QM = (J + TQ - 1) % TQ;
        const int y = ys + base + J;
        // the group of step y - TAHEAD (phi row y+4, rho'/u/v row y+2) is
        // complete once at most TAHEAD - 1 newer ones are pending
        cp_async_wait<TAHEAD - 1>();
        issue(y);
        // phi rows y .. y+4 from the ring (rows below the march's first
        // loaded row hold stale values; stages built on them are never used)
        const P2<T> p1 = phi_row(y + 1), p2 = phi_row(y + 2), p3 = phi_row(y + 3);
        // mu^n(y+3)
        MU[Q3] = chem_pot<T>(K, p2, p3, phi_row(y + 4));
        // Eq. (2.10): Delta rho(y+1) from rho', u, v of rows y .. y+2
        if (y + 1 >= y0 - 1) {
            const P2<T> rc = ruv_row(y + 1, 0), uc = ruv_row(y + 1, 1);
            const P2<T> rn = ruv_row(y + 2, 0), rs = ruv_row(y, 0);
            const P2<T> vn = ruv_row(y + 2, 2), vs = ruv_row(y, 2);
            P2<T> rW, rE, uW, uE;
            shuffle_we<T>(rc, rW, rE);
            shuffle_we<T>(uc, uW, uE);
            P2<T> P, N;
            if (GEN) {
                P = fma2(add2(K.rho0, rE), uE, mul2(add2(K.rho0, rn), vn));
                N = fma2(add2(K.rho0, rW), uW, mul2(add2(K.rho0, rs), vs));
            } else {
                P = fma2(rE, uE, fma2(rn, vn, add2(uE, vn)));
                N = fma2(rW, uW, fma2(rs, vs, add2(uW, vs)));
            }
            const P2<T> lap = fma2(splat(T(-4)), rc, add2(add2(rE, rW), add2(rn, rs)));
            D[Q1] = fma2(K.satc, lap, mul2(K.hdt, sub2(N, P)));
        }
        // first Heun stage phi*(y+2) = phi + dt (-u . grad phi + M Lap mu^n)
        {
            const Iso<T> gp = iso<T>(p1, p2, p3);
            const Iso<T> lm = iso<T>(MU[Q1], MU[Q2], MU[Q3]);
            const P2<T> u2 = ruv_row(y + 2, 1), v2 = ruv_row(y + 2, 2);
            const P2<T> adv = fma2(u2, gp.gx, mul2(v2, gp.gy));
            PS[Q2] = fma2(K.dt, fma2(K.mob, lm.lap, mk(-adv.x, -adv.y)), p2);
        }
        // mu*(y+1)
        MS[Q1] = chem_pot<T>(K, PS[Q0], PS[Q1], PS[Q2]);
        if (y < y0) return;

        // Eq. (2.11) with F_ST = -phi grad mu^n on row y
        const P2<T> r0 = ruv_row(y, 0), u0 = ruv_row(y, 1), v0 = ruv_row(y, 2);
        const P2<T> rN = ruv_row(y + 1, 0), uN = ruv_row(y + 1, 1), vN = ruv_row(y + 1, 2);
        const P2<T> rS = ruv_row(y - 1, 0), uS = ruv_row(y - 1, 1), vS = ruv_row(y - 1, 2);
        P2<T> rW, rE, uW, uE, vW, vE, dW, dE;
        shuffle_we<T>(r0, rW, rE);
        shuffle_we<T>(u0, uW, uE);
        shuffle_we<T>(v0, vW, vE);
        const P2<T> d0 = D[Q0];
        shuffle_we<T>(d0, dW, dE);
        P2<T> mx[5], my[5];
        const P2<T> rr[5] = {r0, rE, rW, rN, rS};
        const P2<T> uu[5] = {u0, uE, uW, uN, uS};
        const P2<T> vv[5] = {v0, vE, vW, vN, vS};
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
        auto lap5 = [&](const P2<T> (&m)[5]) {
            return fma2(splat(T(-4)), m[0], add2(add2(m[1], m[2]), add2(m[3], m[4])));
        };
        // Rt - (dt/2) [(E and N flux terms) - (W and S flux terms)]
        auto flux = [&](const P2<T> (&m)[5], P2<T> Rt) {
            const P2<T> P = fma2(m[1], uu[1], mul2(m[3], vv[3]));
            const P2<T> N = fma2(m[2], uu[2], mul2(m[4], vv[4]));
            return fma2(K.hdt, sub2(N, P), Rt);
        };
        const P2<T> ph0 = phi_row(y);
        const Iso<T> gm = iso<T>(MU[QM], MU[Q0], MU[Q1]);
        const P2<T> rho1 = add2(add2(K.rho0, r0), d0);
        const P2<T> inv = mk(recip(rho1.x), recip(rho1.y));
        P2<T> rx = flux(mx, mul2(K.nudt, lap5(mx)));
        P2<T> ry = flux(my, mul2(K.nudt, lap5(my)));
        rx = fma2(K.hdtcs2, sub2(rW, rE), rx);
        ry = fma2(K.hdtcs2, sub2(rS, rN), ry);
        rx = fma2(K.hsatm, sub2(dW, dE), rx);
        ry = fma2(K.hsatm, sub2(D[QM], D[Q1]), ry);
        const P2<T> fst = mul2(K.ndt, ph0);  // dt F_ST = -dt phi grad mu
        rx = fma2(fst, gm.gx, rx);
        ry = fma2(fst, gm.gy, ry);
        if (GEN) {  // body force dt rho^{n+1} g (A + B phi^n)
            const P2<T> fb = mul2(mul2(K.dt, rho1), fma2(K.bqb, ph0, K.bqa));
            rx = fma2(fb, K.gx, rx);
            ry = fma2(fb, K.gy, ry);
        }
        const P2<T> nd = mk(-d0.x, -d0.y);
        const P2<T> un = fma2(fma2(nd, u0, rx), inv, u0);
        const P2<T> vn = fma2(fma2(nd, v0, ry), inv, v0);
        const P2<T> rn = add2(r0, d0);
        // second Heun stage: phi^{n+1} = (phi + phi* + dt (-u . grad phi* + M Lap mu*)) / 2
        const Iso<T> gs = iso<T>(PS[QM], PS[Q0], PS[Q1]);
        const Iso<T> ls = iso<T>(MS[QM], MS[Q0], MS[Q1]);
        const P2<T> adv = fma2(u0, gs.gx, mul2(v0, gs.gy));
        const P2<T> r2 = fma2(K.mob, ls.lap, mk(-adv.x, -adv.y));
        const P2<T> pn = mul2(splat(T(0.5)), fma2(K.dt, r2, add2(ph0, PS[Q0])));

        const long long o = off + (long long)y * nx + oxa;
        if (wa) {
            out.f[F_R][o] = rn.x;
            out.f[F_U][o] = un.x;
            out.f[F_V][o] = vn.x;
            out.f[F_PHI][o] = pn.x;
        }
        if (wb) {
            out.f[F_R][o + 1] = rn.y;
            out.f[F_U][o + 1] = un.y;
            out.f[F_V][o + 1] = vn.y;
            out.f[F_PHI][o + 1] = pn.y;
        }
        const P2<T> sum = add2(add2(rn, un), add2(vn, pn));
        acc = add2(acc, mk(wa ? sum.x : T(0), wb ? sum.y : T(0)));
    };
    for (int base = 0; base < steps; base += TQ) Unroll<0, TQ>::run(step, base, steps);
    cp_async_wait<0>();  // no copy in flight at exit
    const bool bad = !isfinite(add1(acc.x, acc.y));
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, ERR_NONFINITE);
}

}  // namespace

int line2d_tp_rows() { return TROWS; }
int line2d_tp_stride() { return TOUT; }

template <typename T>
void line2d_tp_prepare()
{
    const int smem = (int)(TWARPS * TRING_ELEMS * sizeof(T));
    cudaFuncSetAttribute(k_line2d_tp<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_line2d_tp<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
}

template <typename T>
cudaError_t launch_line2d_tp(const RunDesc *druns, const int4 *dwork, int nwork, bool gen,
                             Fields<T> in, Fields<T> out, unsigned *derr, cudaStream_t s)
{
    if (nwork <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((nwork + TWARPS - 1) / TWARPS);
    const size_t smem = (size_t)TWARPS * TRING_ELEMS * sizeof(T);
    if (gen)
        k_line2d_tp<T, true><<<grid, 32 * TWARPS, smem, s>>>(druns, dwork, nwork, in, out, derr);
    else
        k_line2d_tp<T, false><<<grid, 32 * TWARPS, smem, s>>>(druns, dwork, nwork, in, out, derr);
    return cudaGetLastError();
}

template void line2d_tp_prepare<float>();
template void line2d_tp_prepare<double>();
template cudaError_t launch_line2d_tp<float>(const RunDesc *, const int4 *, int, bool,
                                             Fields<float>, Fields<float>, unsigned *,
                                             cudaStream_t);
template cudaError_t launch_line2d_tp<double>(const RunDesc *, const int4 *, int, bool,
                                              Fields<double>, Fields<double>, unsigned *,
                                              cudaStream_t);

}  // namespace acm
