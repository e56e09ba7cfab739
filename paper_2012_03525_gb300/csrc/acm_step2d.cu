// Fused 2D time step of the simplified MAME scheme (Huang, arXiv:2012.03525,
// Section 2): continuity Eq. (2.10) and momentum Eq. (2.11) in one kernel,
// optionally with the two-phase extension (F_ST = -phi grad mu and a Heun
// step of the Cahn-Hilliard Eq. 2.14), for one grid or a batch of grids.
//
// Work decomposition: a persistent grid of CTAs walks a list of
// (run, tile_x0, tile_y0) items.  Each item is a T2X x T2Y tile of outputs.
// The CTA stages the tile plus its halo (radius 2 for rho', u, v; radius 4
// for phi) in shared memory -- asynchronously (cp.async) into one of two
// staging sets, the next item's copies in flight while the current item is
// computed -- then computes, all on chip:
//   1. Delta rho = rho^{n+1} - rho^n on the tile grown by one node (Eq. 2.10),
//      so that d_a rho^{n+1} - d_a rho^n of Eq. (2.11) is a centred
//      difference of Delta rho; wall nodes take the second-order
//      zero-normal-gradient extrapolation of rho^{n+1};
//   2. (two-phase) mu^n on the tile grown by 3, phi* (first Heun stage) grown
//      by 2, mu* grown by 1;
//   3. the new velocity u^{n+1} = u^n + (RHS - Delta rho u^n) / rho^{n+1}
//      (deviation form of Eq. 2.11: RHS is every term after (rho u)^n) and,
//      two-phase, phi^{n+1} = (phi + phi* + dt R(phi*, u^n)) / 2.
// Fields are stored as rho' = rho - rho0, u, v (and phi), so the O(Ma^2)
// density signal keeps its digits in FP32.  Each node is read once from
// DRAM (halo re-reads hit L2) and written once.
//
// Tiles are placed at x0 = min(k T2X, nx - T2X): the last tile of a row
// overlaps its neighbour instead of running past the grid, so a wall node
// always has the two interior nodes its extrapolation needs inside the tile.
// Overlapping tiles compute bit-identical values for the shared nodes.
#include "acm_internal.h"

namespace acm {
namespace {

constexpr int RW1 = T2X + 2, RH1 = T2Y + 2, A1 = RW1 * RH1;
constexpr int RW2 = T2X + 4, RH2 = T2Y + 4, A2 = RW2 * RH2;
constexpr int RW3 = T2X + 6, RH3 = T2Y + 6, A3 = RW3 * RH3;
constexpr int RW4 = T2X + 8, RH4 = T2Y + 8, A4 = RW4 * RH4;

constexpr int NWARP = T2THREADS / 32;

// grid index of window column/row c (may lie up to 4 nodes outside the grid):
// periodic directions wrap, wall directions clamp (those values are unused)
__device__ __forceinline__ int wrap_or_clamp(int c, int n, bool periodic)
{
    if (periodic) {
        if (c < 0) c += n;
        else if (c >= n) c -= n;
        if ((unsigned)c >= (unsigned)n) {  // grids narrower than the halo
            c %= n;
            if (c < 0) c += n;
        }
        return c;
    }
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// Visit a (RW x RH) window, 32 <= RW <= 64: warp w takes the first 32
// columns of rows w, w + 8, ... (lane = column: consecutive lanes touch
// consecutive shared-memory words); the remaining RW - 32 columns of every
// row are packed into full warps as one flat list (element t: row t / TW,
// column 32 + t % TW), handed out starting at the first warp with one row
// fewer, so that no warp issues an instruction for a handful of lanes.
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
// Lattice-weighted (D2Q9) isotropic operators on a window of row width RW.
// The Laplacian sums neighbour differences (f_i - f_0), which are exact or
// nearly so for a smooth field, so mu = 4a phi(phi^2-1) - kappa Lap(phi) keeps
// its digits where the two terms nearly cancel (an interface near equilibrium).
template <typename T, int RW>
__device__ __forceinline__ T lap_iso(const T *f, int c)
{
    const T f0 = f[c];
    const T axis = (f[c + 1] - f0) + (f[c - 1] - f0) + (f[c + RW] - f0) + (f[c - RW] - f0);
    const T diag = (f[c + RW + 1] - f0) + (f[c + RW - 1] - f0) + (f[c - RW + 1] - f0) +
                   (f[c - RW - 1] - f0);
    return T(2.0 / 3.0) * axis + T(1.0 / 6.0) * diag;
}
template <typename T, int RW>
__device__ __forceinline__ T gx_iso(const T *f, int c)
{
    return T(1.0 / 3.0) * (f[c + 1] - f[c - 1]) +
           T(1.0 / 12.0) * (f[c + RW + 1] + f[c - RW + 1] - f[c + RW - 1] - f[c - RW - 1]);
}
template <typename T, int RW>
__device__ __forceinline__ T gy_iso(const T *f, int c)
{
    return T(1.0 / 3.0) * (f[c + RW] - f[c - RW]) +
           T(1.0 / 12.0) * (f[c + RW + 1] + f[c + RW - 1] - f[c - RW + 1] - f[c - RW - 1]);
}

// Two-phase wall boundary conditions on a window of the tile (halo H) whose
// first element is node (x0 - H, y0 - H): the ghost node one beyond a wall
// face takes the value of the node one inside the wall (zero normal
// derivative, for mu) plus, for the order parameter (wet != 0), the wetting
// term wet (1 - f_w^2) with f_w the wall node (Section 2: d_n phi =
// -(2/W) cos(theta) (1 - phi_w^2), centred difference).  A corner ghost is
// mirrored through both walls and takes both walls' terms, each evaluated at
// the corner node.  x faces first, then y faces (which overwrite the
// corners); deeper ghost nodes are never read.
template <typename T, int RW, int RH, int H>
__device__ __forceinline__ void wall_ghosts(T *f, int x0, int y0, int nx, int ny, bool perx,
                                            bool pery, T wet)
{
    if (!perx) {
        for_window<RW, RH>([&](int ly, int lx) {
            const int gx = x0 - H + lx;
            if (gx != -1 && gx != nx) return;
            const int s = gx == -1 ? 1 : -1;
            const T fw = f[ly * RW + lx + s];
            f[ly * RW + lx] = f[ly * RW + lx + 2 * s] + wet * (T(1) - fw * fw);
        });
        __syncthreads();
    }
    if (!pery) {
        for_window<RW, RH>([&](int ly, int lx) {
            const int gy = y0 - H + ly;
            if (gy != -1 && gy != ny) return;
            const int gx = x0 - H + lx;
            const int s = gy == -1 ? RW : -RW;
            if (!perx && (gx == -1 || gx == nx)) {
                const int t = s + (gx == -1 ? 1 : -1);
                const T fw = f[ly * RW + lx + t];
                f[ly * RW + lx] = f[ly * RW + lx + 2 * t] + T(2) * wet * (T(1) - fw * fw);
                return;
            }
            const T fw = f[ly * RW + lx + s];
            f[ly * RW + lx] = f[ly * RW + lx + 2 * s] + wet * (T(1) - fw * fw);
        });
        __syncthreads();
    }
}

// asynchronous global -> shared copy of one element (cp.async, bypasses the
// registers), grouped per work item so the next item's staging overlaps
// the current item's compute
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(sizeof(T))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ bool bad(T x)
{
    return !isfinite(x);
}

template <typename T, bool TP>
__global__ void __launch_bounds__(T2THREADS)
    k_step2d(const RunDesc *__restrict__ runs, const int4 *__restrict__ work, int nwork,
             Fields<T> in, Fields<T> out, unsigned *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // two staging sets (rho', u, v with halo 2; phi with halo 4): the next
    // work item is copied in while the current one is computed
    constexpr int STAGE = 3 * A2 + (TP ? A4 : 0);
    T *stage0 = reinterpret_cast<T *>(smem_raw);
    T *sdr = stage0 + 2 * STAGE;
    T *smu = sdr + A1;    // two-phase only from here on
    T *sphs = smu + A3;
    T *smus = sphs + A2;
    const int tid = threadIdx.x, lane = tid & 31;
    bool nonfinite = false;

    // issue the asynchronous copies of work item `it` into staging set `b`
    auto stage = [&](int it, int b) {
        const int4 wk = work[it];
        const RunDesc &R = runs[wk.x];
        const int nx = R.nx, ny = R.ny;
        const int x0 = wk.y, y0 = wk.z;
        const bool perx = R.bc[0] == ACM_BC_PERIODIC;
        const bool pery = R.bc[2] == ACM_BC_PERIODIC;
        const long long off = R.off;
        const T *gr = in.f[F_R] + off, *gu = in.f[F_U] + off, *gv = in.f[F_V] + off;
        T *dr_ = stage0 + b * STAGE, *du = dr_ + A2, *dv = du + A2, *dp = dv + A2;
        // window column of this lane in the first 32 columns (halo 2: rho',
        // u, v; halo 4: phi); the packed columns beyond wrap per element
        const int c2a = wrap_or_clamp(x0 - 2 + lane, nx, perx);
        for_window<RW2, RH2>([&](int ly, int lx) {
            const long long row = (long long)wrap_or_clamp(y0 - 2 + ly, ny, pery) * nx;
            const long long k = row + (lx < 32 ? c2a : wrap_or_clamp(x0 - 2 + lx, nx, perx));
            const int i = ly * RW2 + lx;
            cp_async_elem(dr_ + i, gr + k);
            cp_async_elem(du + i, gu + k);
            cp_async_elem(dv + i, gv + k);
        });
        if (TP) {
            const T *gp = in.f[F_PHI] + off;
            const int c4a = wrap_or_clamp(x0 - 4 + lane, nx, perx);
            for_window<RW4, RH4>([&](int ly, int lx) {
                const long long row = (long long)wrap_or_clamp(y0 - 4 + ly, ny, pery) * nx;
                cp_async_elem(dp + ly * RW4 + lx,
                              gp + row + (lx < 32 ? c4a : wrap_or_clamp(x0 - 4 + lx, nx, perx)));
            });
        }
    };

    if ((int)blockIdx.x < nwork) stage(blockIdx.x, 0);
    cp_async_commit();
    int buf = 0;
    for (int item = blockIdx.x; item < nwork; item += gridDim.x, buf ^= 1) {
        const int4 wk = work[item];
        const RunDesc &R = runs[wk.x];
        const int nx = R.nx, ny = R.ny;
        const int x0 = wk.y, y0 = wk.z;
        const bool perx = R.bc[0] == ACM_BC_PERIODIC;
        const bool pery = R.bc[2] == ACM_BC_PERIODIC;
        const T *C = coefs<T>(R);
        const T rho0 = C[C_RHO0], dt = C[C_DT], nudt = C[C_NUDT], satc = C[C_SATC];
        const T cs2 = C[C_CS2];
        const long long off = R.off;
        T *sr = stage0 + buf * STAGE, *su = sr + A2, *sv = su + A2, *sphi = sv + A2;

        __syncthreads();  // the previous item no longer reads shared memory
        if (item + (int)gridDim.x < nwork) stage(item + gridDim.x, buf ^ 1);
        cp_async_commit();
        cp_async_wait<1>();  // this item's copies (issued one item earlier) have landed
        __syncthreads();

        const T a = C[C_A], kappa = C[C_KAPPA], mob = C[C_M];
        const bool walls = !perx || !pery;
        if (TP && walls)
            wall_ghosts<T, RW4, RH4, 4>(sphi, x0, y0, nx, ny, perx, pery, C[C_WET]);
        if (TP) {
            // mu^n on the tile grown by 3 (window origin x0-3)
            for_window<RW3, RH3>([&](int ly, int lx) {
                const int c4 = (ly + 1) * RW4 + (lx + 1);
                const T f = sphi[c4];
                smu[ly * RW3 + lx] =
                    T(4) * a * f * (f * f - T(1)) - kappa * lap_iso<T, RW4>(sphi, c4);
            });
        }
        // Eq. (2.10): Delta rho on the tile grown by 1 (interior nodes)
        for_window<RW1, RH1>([&](int ly, int lx) {
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            bool active = true;
            if (!perx && (gx <= 0 || gx >= nx - 1)) active = false;
            if (!pery && (gy <= 0 || gy >= ny - 1)) active = false;
            T d = T(0);
            if (active) {
                const int c = (ly + 1) * RW2 + (lx + 1);
                const T mxE = (rho0 + sr[c + 1]) * su[c + 1];
                const T mxW = (rho0 + sr[c - 1]) * su[c - 1];
                const T myN = (rho0 + sr[c + RW2]) * sv[c + RW2];
                const T myS = (rho0 + sr[c - RW2]) * sv[c - RW2];
                d = -dt * (T(0.5) * (mxE - mxW) + T(0.5) * (myN - myS));
                d += satc * (sr[c + 1] + sr[c - 1] + sr[c + RW2] + sr[c - RW2] - T(4) * sr[c]);
            }
            sdr[ly * RW1 + lx] = d;
        });
        if (!perx || !pery) {
            // wall density: rho_w^{n+1} = (4 rho_1^{n+1} - rho_2^{n+1}) / 3, x faces
            // first, then y faces (corners end with the y extrapolation)
            for (int pass = 0; pass < 2; ++pass) {
                const bool per = pass == 0 ? perx : pery;
                if (per) continue;
                __syncthreads();
                const int n = pass == 0 ? nx : ny;
                for (int i = tid; i < A1; i += T2THREADS) {
                    int ly = i / RW1, lx = i - ly * RW1;
                    int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
                    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
                    const int g = pass == 0 ? gx : gy;
                    if (g != 0 && g != n - 1) continue;
                    const int s1 = (g == 0 ? 1 : -1) * (pass == 0 ? 1 : RW1);
                    const int s2 = (g == 0 ? 1 : -1) * (pass == 0 ? 1 : RW2);
                    const int c = (ly + 1) * RW2 + (lx + 1);
                    const T r1 = sr[c + s2] + sdr[i + s1];
                    const T r2 = sr[c + 2 * s2] + sdr[i + 2 * s1];
                    sdr[i] = (T(4) * r1 - r2) / T(3) - sr[c];
                }
            }
        }
        __syncthreads();
        if (TP && walls) wall_ghosts<T, RW3, RH3, 3>(smu, x0, y0, nx, ny, perx, pery, T(0));
        if (TP) {
            // first Heun stage phi* on the tile grown by 2
            for_window<RW2, RH2>([&](int ly, int lx) {
                const int i = ly * RW2 + lx;
                const int c4 = (ly + 2) * RW4 + (lx + 2);
                const int c3 = (ly + 1) * RW3 + (lx + 1);
                const T adv = su[i] * gx_iso<T, RW4>(sphi, c4) + sv[i] * gy_iso<T, RW4>(sphi, c4);
                sphs[i] = sphi[c4] + dt * (-adv + mob * lap_iso<T, RW3>(smu, c3));
            });
            __syncthreads();
            if (walls) wall_ghosts<T, RW2, RH2, 2>(sphs, x0, y0, nx, ny, perx, pery, C[C_WET]);
            // mu* on the tile grown by 1
            for_window<RW1, RH1>([&](int ly, int lx) {
                const int c2 = (ly + 1) * RW2 + (lx + 1);
                const T f = sphs[c2];
                smus[ly * RW1 + lx] =
                    T(4) * a * f * (f * f - T(1)) - kappa * lap_iso<T, RW2>(sphs, c2);
            });
            __syncthreads();
            if (walls) wall_ghosts<T, RW1, RH1, 1>(smus, x0, y0, nx, ny, perx, pery, T(0));
        }

        // Eq. (2.11) on the tile interior; write the new state
        const T satm = C[C_SATM];
        const T gxb = C[C_GX], gyb = C[C_GY];
        for_window<T2X, T2Y>([&](int ly, int lx) {
            const int gx = x0 + lx, gy = y0 + ly;
            if (gx >= nx || gy >= ny) return;
            const int c = (ly + 2) * RW2 + (lx + 2);
            const int c1 = (ly + 1) * RW1 + (lx + 1);
            const T r0 = sr[c], u0 = su[c], v0 = sv[c], d0 = sdr[c1];
            const T rho1 = rho0 + r0 + d0;
            T un, vn;
            const bool xw = !perx && (gx == 0 || gx == nx - 1);
            const bool yw = !pery && (gy == 0 || gy == ny - 1);
            if (xw || yw) {
                // stationary walls win at corners shared with a lid
                bool stationary = (!perx && ((gx == 0 && R.bc[0] == ACM_BC_WALL) ||
                                             (gx == nx - 1 && R.bc[1] == ACM_BC_WALL))) ||
                                  (!pery && ((gy == 0 && R.bc[2] == ACM_BC_WALL) ||
                                             (gy == ny - 1 && R.bc[3] == ACM_BC_WALL)));
                un = stationary ? T(0) : C[C_LIDX];
                vn = stationary ? T(0) : C[C_LIDY];
            } else {
                const T mx0 = (rho0 + r0) * u0, my0 = (rho0 + r0) * v0;
                const T rE = sr[c + 1], rW = sr[c - 1], rN = sr[c + RW2], rS = sr[c - RW2];
                const T uE = su[c + 1], uW = su[c - 1], uN = su[c + RW2], uS = su[c - RW2];
                const T vE = sv[c + 1], vW = sv[c - 1], vN = sv[c + RW2], vS = sv[c - RW2];
                const T mxE = (rho0 + rE) * uE, mxW = (rho0 + rW) * uW;
                const T mxN = (rho0 + rN) * uN, mxS = (rho0 + rS) * uS;
                const T myE = (rho0 + rE) * vE, myW = (rho0 + rW) * vW;
                const T myN = (rho0 + rN) * vN, myS = (rho0 + rS) * vS;
                const T fx = T(0.5) * (mxE * uE - mxW * uW) + T(0.5) * (mxN * vN - mxS * vS) +
                             cs2 * T(0.5) * (rE - rW);
                const T fy = T(0.5) * (myE * uE - myW * uW) + T(0.5) * (myN * vN - myS * vS) +
                             cs2 * T(0.5) * (rN - rS);
                const T lmx = mxE + mxW + mxN + mxS - T(4) * mx0;
                const T lmy = myE + myW + myN + myS - T(4) * my0;
                const T ddx = T(0.5) * (sdr[c1 + 1] - sdr[c1 - 1]);
                const T ddy = T(0.5) * (sdr[c1 + RW1] - sdr[c1 - RW1]);
                T gfx = gxb, gfy = gyb;
                if (TP) {  // body-force factor: 1, or the Boussinesq drop force
                    const T fac = C[C_BQA] + C[C_BQB] * sphi[(ly + 4) * RW4 + (lx + 4)];
                    gfx = gxb * fac;
                    gfy = gyb * fac;
                }
                T rhsx = -dt * fx + nudt * lmx - satm * ddx + dt * rho1 * gfx;
                T rhsy = -dt * fy + nudt * lmy - satm * ddy + dt * rho1 * gfy;
                if (TP) {
                    const int c3 = (ly + 3) * RW3 + (lx + 3);
                    const int c4 = (ly + 4) * RW4 + (lx + 4);
                    const T ph = sphi[c4];
                    rhsx += dt * (-ph * gx_iso<T, RW3>(smu, c3));
                    rhsy += dt * (-ph * gy_iso<T, RW3>(smu, c3));
                }
                const T inv = T(1) / rho1;
                un = u0 + (rhsx - d0 * u0) * inv;
                vn = v0 + (rhsy - d0 * v0) * inv;
            }
            const long long gi = off + (long long)gy * nx + gx;
            const T rn = r0 + d0;
            out.f[F_R][gi] = rn;
            out.f[F_U][gi] = un;
            out.f[F_V][gi] = vn;
            T chk = rn + un + vn;
            if (TP) {
                const int c4 = (ly + 4) * RW4 + (lx + 4);
                const int c2 = (ly + 2) * RW2 + (lx + 2);
                const T adv = u0 * gx_iso<T, RW2>(sphs, c2) + v0 * gy_iso<T, RW2>(sphs, c2);
                const T r2 = -adv + mob * lap_iso<T, RW1>(smus, c1);
                const T phn = T(0.5) * (sphi[c4] + sphs[c2] + dt * r2);
                out.f[F_PHI][gi] = phn;
                chk += phn;
            }
            nonfinite |= bad(chk);
        });
    }
    cp_async_wait<0>();  // no copy left in flight at exit
    if (nonfinite) atomicOr(err, ERR_NONFINITE);
}

template <typename T, bool TP>
size_t smem_bytes()
{
    size_t n = 2 * (3 * A2 + (TP ? A4 : 0)) + A1;
    if (TP) n += A3 + A2 + A1;
    return n * sizeof(T);
}

template <typename T, bool TP>
int max_blocks()
{
    static int cached = -1;
    if (cached < 0) {
        cudaFuncSetAttribute(k_step2d<T, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<T, TP>());
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step2d<T, TP>, T2THREADS,
                                                          smem_bytes<T, TP>()) != cudaSuccess)
            nb = 1;
        cached = nb > 0 ? nb : 1;
    }
    return cached;
}

}  // namespace

template <typename T>
int step2d_max_blocks_per_sm(int two_phase)
{
    return two_phase ? max_blocks<T, true>() : max_blocks<T, false>();
}

template <typename T>
cudaError_t launch_step2d(const RunDesc *druns, const int4 *dwork, int nwork, int two_phase,
                          Fields<T> in, Fields<T> out, unsigned *derr, int blocks,
                          cudaStream_t s)
{
    if (nwork <= 0) return cudaSuccess;
    if (blocks > nwork) blocks = nwork;
    if (two_phase) {
        max_blocks<T, true>();
        k_step2d<T, true><<<blocks, T2THREADS, smem_bytes<T, true>(), s>>>(druns, dwork, nwork,
                                                                          in, out, derr);
    } else {
        max_blocks<T, false>();
        k_step2d<T, false><<<blocks, T2THREADS, smem_bytes<T, false>(), s>>>(druns, dwork,
                                                                            nwork, in, out, derr);
    }
    return cudaGetLastError();
}

template cudaError_t launch_step2d<float>(const RunDesc *, const int4 *, int, int, Fields<float>,
                                          Fields<float>, unsigned *, int, cudaStream_t);
template cudaError_t launch_step2d<double>(const RunDesc *, const int4 *, int, int,
                                           Fields<double>, Fields<double>, unsigned *, int,
                                           cudaStream_t);
template int step2d_max_blocks_per_sm<float>(int);
template int step2d_max_blocks_per_sm<double>(int);

}  // namespace acm
