// Fused 3D time step of the simplified MAME scheme (Huang, arXiv:2012.03525,
// Section 2, Eqs. 2.10-2.11 with the 7-point extension of Eq. 2.13), periodic
// grids, single phase.
//
// Design (one kernel per step, HBM-bound):
//   * Each CTA owns a T3X x TY column of the x-y plane and marches along z
//     over a chunk of planes.  Input planes of rho', u, v, w (with a 2-node
//     x-y halo) are staged in shared memory by TMA tiled loads
//     (cp.async.bulk.tensor.3d) into a ring of T3SLOTS plane slots; the load
//     of plane z+3 is in flight while plane z is computed.
//   * Eq. (2.10) is evaluated on the plane z+1 grown by one node and kept in a
//     ring of three Delta-rho planes, so d_a rho^{n+1} - d_a rho^n of
//     Eq. (2.11) is a centred difference of Delta rho read from shared memory.
//   * Eq. (2.11) for plane z; u^{n+1} = u + (RHS - Delta rho u) / rho^{n+1}.
// Storage is padded by T3PAD ghost nodes in x and y (not in z).  Every output
// node on the first/last two columns/rows is also written to its periodic
// image in the ghost layers, so the next step's TMA boxes never wrap in x/y;
// z wraps through the box coordinate.  Padding also keeps every box start on a
// 16-byte boundary (x start = tile x0, a multiple of 32 elements).
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

template <typename T, int TY>
struct Geo {
    static constexpr int RW = T3X + 4, RH = TY + 4, PLANE = RW * RH;
    static constexpr int PLANE_BYTES = ((PLANE * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int RW1 = T3X + 2, RH1 = TY + 2, P1 = RW1 * RH1;
    static constexpr int SD_BYTES = ((3 * P1 * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int SMEM = T3SLOTS * 4 * PLANE_BYTES + SD_BYTES + 128;
    static constexpr int NT = T3X * TY;
};

template <typename T, int TY>
__global__ void __launch_bounds__(T3X *TY)
    k_step3d(const __grid_constant__ CUtensorMap mr, const __grid_constant__ CUtensorMap mu_,
             const __grid_constant__ CUtensorMap mv, const __grid_constant__ CUtensorMap mw,
             Fields<T> out, const __grid_constant__ RunDesc R, int zc, unsigned *err)
{
    using G = Geo<T, TY>;
    extern __shared__ __align__(128) unsigned char smem[];
    T *sd = reinterpret_cast<T *>(smem + T3SLOTS * 4 * G::PLANE_BYTES);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + T3SLOTS * 4 * G::PLANE_BYTES + G::SD_BYTES);
    int *s_abort = reinterpret_cast<int *>(bar + T3SLOTS);
    auto plane = [&](int slot, int f) -> T * {
        return reinterpret_cast<T *>(smem + (slot * 4 + f) * G::PLANE_BYTES);
    };

    const int tid = threadIdx.x;
    const int tx = tid % T3X, ty = tid / T3X;
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int x0 = blockIdx.x * T3X, y0 = blockIdx.y * TY;
    const int zbeg = blockIdx.z * zc;
    const int zend = min(zbeg + zc, nz);
    if (zbeg >= zend) return;
    const T *C = coefs<T>(R);
    const T rho0 = C[C_RHO0], dt = C[C_DT], cs2 = C[C_CS2], nudt = C[C_NUDT];
    const T satc = C[C_SATC], satm = C[C_SATM];
    const T gxb = C[C_GX], gyb = C[C_GY], gzb = C[C_GZ];
    constexpr uint32_t TX_BYTES = 4u * G::PLANE * sizeof(T);

    if (tid == 0) {
        for (int s = 0; s < T3SLOTS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_abort = 0;
    }
    __syncthreads();

    // plane zz (zbeg-2 <= zz <= zend+1) lives in slot (zz - zbeg + 2) % T3SLOTS
    auto issue = [&](int zz) {
        const int k = zz - zbeg + 2;
        const int s = k % T3SLOTS;
        int zw = zz % nz;
        if (zw < 0) zw += nz;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[s], TX_BYTES);
        tma_load_3d(plane(s, F_R), &mr, x0, y0, zw, &bar[s]);
        tma_load_3d(plane(s, F_U), &mu_, x0, y0, zw, &bar[s]);
        tma_load_3d(plane(s, F_V), &mv, x0, y0, zw, &bar[s]);
        tma_load_3d(plane(s, F_W), &mw, x0, y0, zw, &bar[s]);
    };
    auto wait = [&](int zz) {
        const int k = zz - zbeg + 2;
        const int s = k % T3SLOTS;
        const uint32_t par = (uint32_t)((k / T3SLOTS) & 1);
        for (int it = 0; it < WAIT_LIMIT; ++it)
            if (mbar_try_wait(&bar[s], par)) return;
        *s_abort = 1;
        atomicOr(err, ERR_TIMEOUT);
    };
    auto slot_of = [&](int zz) { return (zz - zbeg + 2) % T3SLOTS; };
    auto sdp = [&](int zz) { return sd + ((zz - zbeg + 3) % 3) * G::P1; };

    // Eq. (2.10) on plane zz grown by one node: needs planes zz-1, zz, zz+1
    auto delta_rho = [&](int zz) {
        const int sm = slot_of(zz - 1), s0 = slot_of(zz), sp = slot_of(zz + 1);
        const T *r0 = plane(s0, F_R), *u0 = plane(s0, F_U), *v0 = plane(s0, F_V);
        const T *rm = plane(sm, F_R), *wm = plane(sm, F_W);
        const T *rp = plane(sp, F_R), *wp = plane(sp, F_W);
        T *dst = sdp(zz);
        for (int i = tid; i < G::P1; i += G::NT) {
            const int ly = i / G::RW1, lx = i - ly * G::RW1;
            const int c = (ly + 1) * G::RW + (lx + 1);
            const T div = T(0.5) * ((rho0 + r0[c + 1]) * u0[c + 1] - (rho0 + r0[c - 1]) * u0[c - 1]) +
                          T(0.5) * ((rho0 + r0[c + G::RW]) * v0[c + G::RW] -
                                    (rho0 + r0[c - G::RW]) * v0[c - G::RW]) +
                          T(0.5) * ((rho0 + rp[c]) * wp[c] - (rho0 + rm[c]) * wm[c]);
            const T lap = r0[c + 1] + r0[c - 1] + r0[c + G::RW] + r0[c - G::RW] + rp[c] + rm[c] -
                          T(6) * r0[c];
            dst[i] = -dt * div + satc * lap;
        }
    };

    // prologue: planes zbeg-2 .. zbeg+2, Delta rho of zbeg-1 and zbeg
    if (tid == 0)
        for (int zz = zbeg - 2; zz <= zbeg + 2; ++zz) issue(zz);
    wait(zbeg - 2);
    wait(zbeg - 1);
    wait(zbeg);
    __syncthreads();
    if (*s_abort) return;
    delta_rho(zbeg - 1);
    wait(zbeg + 1);
    __syncthreads();
    if (*s_abort) return;
    delta_rho(zbeg);

    const int gx = x0 + tx, gy = y0 + ty;
    const bool owner = gx < nx && gy < ny;
    const long long PX = R.px, PXY = R.px * R.py;
    const long long base = R.off + (long long)(gy + T3PAD) * PX + (gx + T3PAD);
    const bool edge = gx < T3PAD || gx >= nx - T3PAD || gy < T3PAD || gy >= ny - T3PAD;
    const int c = (ty + 2) * G::RW + (tx + 2);
    const int c1 = (ty + 1) * G::RW1 + (tx + 1);

    for (int z = zbeg; z < zend; ++z) {
        __syncthreads();  // slot of plane z-2 and Delta-rho ring slot of z-2 are free
        if (tid == 0 && z + 3 <= zend + 1) issue(z + 3);
        wait(z + 2);
        delta_rho(z + 1);  // harmless on stale data if the wait gave up
        __syncthreads();
        if (*s_abort) break;

        if (owner) {
            const int sm = slot_of(z - 1), s0 = slot_of(z), sp = slot_of(z + 1);
            const T *r = plane(s0, F_R), *u = plane(s0, F_U), *v = plane(s0, F_V),
                    *w = plane(s0, F_W);
            const T *rm = plane(sm, F_R), *um = plane(sm, F_U), *vm = plane(sm, F_V),
                    *wm = plane(sm, F_W);
            const T *rp = plane(sp, F_R), *up = plane(sp, F_U), *vp = plane(sp, F_V),
                    *wp = plane(sp, F_W);
            const T *d0 = sdp(z), *dm = sdp(z - 1), *dp = sdp(z + 1);

            const T r0 = r[c], u0 = u[c], v0 = v[c], w0 = w[c], dr = d0[c1];
            // neighbour densities rho0 + rho'
            const T qE = rho0 + r[c + 1], qW = rho0 + r[c - 1];
            const T qN = rho0 + r[c + G::RW], qS = rho0 + r[c - G::RW];
            const T qU = rho0 + rp[c], qD = rho0 + rm[c];
            const T uE = u[c + 1], uW = u[c - 1], uN = u[c + G::RW], uS = u[c - G::RW],
                    uU = up[c], uD = um[c];
            const T vE = v[c + 1], vW = v[c - 1], vN = v[c + G::RW], vS = v[c - G::RW],
                    vU = vp[c], vD = vm[c];
            const T wE = w[c + 1], wW = w[c - 1], wN = w[c + G::RW], wS = w[c - G::RW],
                    wU = wp[c], wD = wm[c];
            const T q0 = rho0 + r0;
            const T rho1 = q0 + dr;
            const T inv = T(1) / rho1;
            const T ddx = T(0.5) * (d0[c1 + 1] - d0[c1 - 1]);
            const T ddy = T(0.5) * (d0[c1 + G::RW1] - d0[c1 - G::RW1]);
            const T ddz = T(0.5) * (dp[c1] - dm[c1]);
            // flux d_b(rho u_a u_b) + c_s^2 d_a rho', viscous nu Lap(rho u_a)
            auto comp = [&](T aE, T aW, T aN, T aS, T aU, T aD, T a0, T dpress, T dd, T gb) {
                const T mE = qE * aE, mW = qW * aW, mN = qN * aN, mS = qS * aS, mU = qU * aU,
                        mD = qD * aD;
                const T flux = T(0.5) * (mE * uE - mW * uW) + T(0.5) * (mN * vN - mS * vS) +
                               T(0.5) * (mU * wU - mD * wD) + cs2 * dpress;
                const T lapm = mE + mW + mN + mS + mU + mD - T(6) * (q0 * a0);
                const T rhs = -dt * flux + nudt * lapm - satm * dd + dt * rho1 * gb;
                return a0 + (rhs - dr * a0) * inv;
            };
            const T un = comp(uE, uW, uN, uS, uU, uD, u0, T(0.5) * (r[c + 1] - r[c - 1]), ddx, gxb);
            const T vn = comp(vE, vW, vN, vS, vU, vD, v0, T(0.5) * (r[c + G::RW] - r[c - G::RW]),
                              ddy, gyb);
            const T wn = comp(wE, wW, wN, wS, wU, wD, w0, T(0.5) * (rp[c] - rm[c]), ddz, gzb);
            const T rn = r0 + dr;

            // write the node; threads on the first/last T3PAD columns/rows also
            // write its periodic images in the ghost layers (both images exist
            // when the grid is narrower than 2 * T3PAD)
            const long long gi = base + (long long)z * PXY;
            out.f[F_R][gi] = rn;
            out.f[F_U][gi] = un;
            out.f[F_V][gi] = vn;
            out.f[F_W][gi] = wn;
            if (edge) {
                int xs[3], ys[3], nxs = 1, nys = 1;
                xs[0] = 0;
                ys[0] = 0;
                if (gx < T3PAD) xs[nxs++] = nx;
                if (gx >= nx - T3PAD) xs[nxs++] = -nx;
                if (gy < T3PAD) ys[nys++] = ny;
                if (gy >= ny - T3PAD) ys[nys++] = -ny;
                for (int jy = 0; jy < nys; ++jy)
                    for (int jx = 0; jx < nxs; ++jx) {
                        if (jx == 0 && jy == 0) continue;
                        const long long gk = gi + (long long)ys[jy] * PX + xs[jx];
                        out.f[F_R][gk] = rn;
                        out.f[F_U][gk] = un;
                        out.f[F_V][gk] = vn;
                        out.f[F_W][gk] = wn;
                    }
            }
            if (!isfinite(rn) || !isfinite(un) || !isfinite(vn) || !isfinite(wn))
                atomicOr(err, ERR_NONFINITE);
        }
    }
}

template <typename T, int TY>
int max_blocks()
{
    static int cached = -1;
    if (cached < 0) {
        using G = Geo<T, TY>;
        cudaFuncSetAttribute(k_step3d<T, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G::SMEM);
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step3d<T, TY>, G::NT, G::SMEM) !=
            cudaSuccess)
            nb = 1;
        cached = nb > 0 ? nb : 1;
    }
    return cached;
}

template <typename T, int TY>
cudaError_t launch(const CUtensorMap *m, Fields<T> out, const RunDesc &run, unsigned *derr,
                   int zchunks, cudaStream_t s)
{
    using G = Geo<T, TY>;
    max_blocks<T, TY>();
    if (zchunks < 1) zchunks = 1;
    if (zchunks > run.nz) zchunks = run.nz;
    const int zc = (run.nz + zchunks - 1) / zchunks;
    dim3 grid((run.nx + T3X - 1) / T3X, (run.ny + TY - 1) / TY, (run.nz + zc - 1) / zc);
    k_step3d<T, TY><<<grid, G::NT, G::SMEM, s>>>(m[0], m[1], m[2], m[3], out, run, zc, derr);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
int step3d_max_blocks_per_sm(int t3y)
{
    return t3y == 16 ? max_blocks<T, 16>() : max_blocks<T, 8>();
}

template <typename T>
cudaError_t launch_step3d(const CUtensorMap *maps_in, Fields<T> out, const RunDesc &run,
                          unsigned *derr, int zchunks, int t3y, cudaStream_t s)
{
    if (t3y == 16) return launch<T, 16>(maps_in, out, run, derr, zchunks, s);
    return launch<T, 8>(maps_in, out, run, derr, zchunks, s);
}

template cudaError_t launch_step3d<float>(const CUtensorMap *, Fields<float>, const RunDesc &,
                                          unsigned *, int, int, cudaStream_t);
template cudaError_t launch_step3d<double>(const CUtensorMap *, Fields<double>, const RunDesc &,
                                           unsigned *, int, int, cudaStream_t);
template int step3d_max_blocks_per_sm<float>(int);
template int step3d_max_blocks_per_sm<double>(int);

}  // namespace acm
