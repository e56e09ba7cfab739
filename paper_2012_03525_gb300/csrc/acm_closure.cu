// Learned closure: a 3-layer 3x3 convolutional network (3 -> 32 -> 32 -> 3,
// ReLU after the first two layers) that corrects a coarse-grid state
// (rho', u, v) after solver steps, with its training on the GPU.
//
// All convolutions are periodic 2D cross-correlations on the tensor cores,
// BF16 operands and FP32 accumulation:
//   * forward:        Y[p, co] = sum_K X[p + off(tap), ci] A[co, K], K = (tap, ci),
//                     A = W in [co][tap][ci] order -- tcgen05.mma with the
//                     accumulator in tensor memory (k_conv_tc);
//   * data gradient:  dX = (W flipped, channels swapped) applied to dY -- the
//                     same kernel with a rearranged weight matrix;
//   * weight gradient: dW[co, (tap, ci)] = sum_p dY[co, p] X[p + off(tap), ci]
//                     -- a GEMM whose reduction runs over pixels, on tcgen05
//                     with MN-major operands (k_wgrad_tc); per-CTA partials
//                     are summed in a fixed order (deterministic).
// Activations and gradients are stored as BF16 NHWC (channels contiguous),
// the master weights, Adam moments, losses and corrections in FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "acm_internal.h"

namespace acm {
namespace {

typedef __nv_bfloat16 bf16;


// real / padded channel counts of the three layers
constexpr int NL = 3;
constexpr int CIN[NL] = {3, 32, 32}, COUT[NL] = {32, 32, 3};
constexpr int CINP[NL] = {16, 32, 32}, COUTP[NL] = {32, 32, 16};

enum { OUT_RELU_BF16 = 0, OUT_MASK_BF16 = 1, OUT_F32_NCHW = 2 };

// ---- 5th-generation tensor cores (tcgen05) ---------------------------------
// One 3x3 convolution layer (or its data gradient) as per-tap GEMMs issued by
// one thread of the CTA: for each tap (dy, dx) and 16-channel slice,
//   D[p, co] += sum_ci X[p + (dy, dx), ci] A[co, (tap, ci)]
// with M = the 128 pixels of a 16 x 8 tile, N = CO, K = 16, BF16 operands
// from shared memory and the FP32 accumulator D in tensor memory (TMEM).
// Both operands are in the no-swizzle K-major layout of 8 x 16-byte "core
// matrices": the (16 + 2) x (8 + 2) halo of X is staged once (periodic wrap
// applied while staging); the 8-pixel row groups of the A operand of tap
// (dy, dx) are the tile rows, which start at halo pixel (row + dy + 1) * 10
// + dx + 1, so one descriptor with a 10-pixel stride between groups covers
// the tap; the weights as [tap][ci / 8][co][8].  Persistent CTAs of 4 warps walk
// the tiles, staging the next tile (cp.async) while the tensor cores work on
// the current one; the epilogue reads D with tcgen05.ld (warp w holds TMEM
// lanes 32w .. 32w + 31, i.e. tile rows 4w .. 4w + 3).
constexpr int TC_THREADS = 128;
// pixel tile of every convolution kernel: 16 rows x 8 columns (M = 128
// pixels, eight per row, so the 8-pixel core-matrix groups of a tap's
// operand are the tile rows, equally spaced in one staged halo)
constexpr int FTH = 16, FTW = 8;
constexpr int FHW = FTW + 2, FHP = (FTH + 2) * FHW;  // halo row width, halo pixels

template <int CI, int CO>
struct TcGeo {
    static constexpr int XBUF = FHP * CI * 2;     // one staged forward tile
    static constexpr int WBYTES = 9 * CI * CO * 2;
    static constexpr int BAR = 2 * XBUF + WBYTES;
    static constexpr int SMEM = BAR + 16;
    static constexpr int TCOLS = 32;              // TMEM columns (>= CO, a power of 2 >= 32)
    static_assert(CO == 16 || CO == 32, "N of the MMA");
    static_assert(CI % 16 == 0, "K slices of 16");
};

__device__ __forceinline__ uint32_t tc_smem(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: no swizzle, start address, leading (K)
// and stride (M/N) byte offsets between core matrices, version 1 (sm_100)
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc_smem(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ bool tc_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// D row of this thread (TMEM lane 32 w + lane): N FP32 columns
template <int N>
__device__ __forceinline__ void tc_load_row(uint32_t taddr, float (&v)[N]);
template <>
__device__ __forceinline__ void tc_load_row<32>(uint32_t ta, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tc_load_row<16>(uint32_t ta, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// bounded wait: ~2^22 polls (well over a second), then give up
constexpr int TC_WAIT_LIMIT = 1 << 22;

// index in [-1, n] wrapped into [0, n)
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// The (16 + 2) x (8 + 2) halo of the 16 x 8 tile at (y0, x0) of image xi
// (NHWC, periodic): chunk j (channels 8j .. 8j + 7) of halo pixel hp = hr * 10
// + c at [j][hp][8].  Consecutive threads take consecutive 16-byte chunks of
// global memory (the chunks of a pixel, then the next pixel of the row).
template <int CI>
__device__ __forceinline__ void stage_tile(unsigned char *dst, const bf16 *xi, int H, int W,
                                           int y0, int x0, int tid)
{
    constexpr int NJ = CI / 8;
    for (int i = tid; i < FHP * NJ; i += TC_THREADS) {
        const int hp = i / NJ, j = i - hp * NJ;
        const int hr = hp / FHW, c = hp - hr * FHW;
        const int gy = wrap1(y0 - 1 + hr, H), gx = wrap1(x0 - 1 + c, W);
        cp_async16(dst + (j * FHP + hp) * 16, xi + ((size_t)gy * W + gx) * CI + 8 * j);
    }
}

template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(TC_THREADS)
    k_conv_tc(const bf16 *__restrict__ x, const bf16 *__restrict__ A,
              const float *__restrict__ bias, const bf16 *__restrict__ mask, void *__restrict__ out,
              int H, int W, int nout, int ntiles, unsigned *err)
{
    using G = TcGeo<CI, CO>;
    extern __shared__ __align__(1024) unsigned char tsm[];
    bf16 *ws = reinterpret_cast<bf16 *>(tsm + 2 * G::XBUF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(tsm + G::BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tsm + G::BAR + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / FTW, tiles_img = tiles_x * (H / FTH);

    // weights [co][tap * CI + ci] -> [tap][ci / 8][co][8] (16-byte chunks)
    for (int i = tid; i < CO * 9 * CI / 8; i += TC_THREADS) {
        const int co = i / (9 * CI / 8), k0 = 8 * (i - co * (9 * CI / 8));
        const int tap = k0 / CI, cc = (k0 - tap * CI) / 8;
        *reinterpret_cast<uint4 *>(&ws[((tap * (CI / 8) + cc) * CO + co) * 8]) =
            *reinterpret_cast<const uint4 *>(&A[(size_t)co * 9 * CI + k0]);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem(tslot)),
                     "r"(G::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }

    // stage tile t (periodic halo) into buffer b
    auto stage = [&](int t, int b) {
        const int img = t / tiles_img, r = t - img * tiles_img;
        const int y0 = (r / tiles_x) * FTH, x0 = (r % tiles_x) * FTW;
        stage_tile<CI>(tsm + b * G::XBUF, x + (size_t)img * H * W * CI, H, W, y0, x0, tid);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    int t = blockIdx.x;
    if (t < ntiles) stage(t, 0);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // kind::f16 instruction descriptor: D F32, A and B BF16, both K-major,
    // N >> 3 at bit 17, M >> 4 at bit 24 (M = 128)
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CO >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    uint32_t phase = 0;
    int b = 0;
    for (; t < ntiles; t += gridDim.x, b ^= 1) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        // the tile's copies (generic proxy) become visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t xb = tc_smem(tsm + b * G::XBUF), wb = tc_smem(ws);
            int k = 0;
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dxi = tap % 3;  // dy + 1, dx + 1
#pragma unroll
                for (int kc = 0; kc < CI / 16; ++kc, ++k) {
                    // A: 8-pixel group g (tile row g) of tap (dy, dx) starts at
                    // halo pixel (g + dy) * 10 + dx: stride 10 pixels between
                    // groups, FHP pixels between the two 8-channel chunks of K
                    const uint64_t ad = tc_desc(xb + 2 * kc * FHP * 16 + (dy * FHW + dxi) * 16,
                                                FHP * 16, FHW * 16);
                    const uint64_t bd = tc_desc(wb + (tap * (CI / 8) + 2 * kc) * CO * 16, CO * 16,
                                                128);
                    tc_mma(tmem, ad, bd, idesc, k > 0);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    tc_smem(bar))
                : "memory");
        }
        // stage the next tile into the other buffer while the MMAs run
        const int tn = t + gridDim.x;
        if (tn < ntiles) stage(tn, b ^ 1);
        bool ok = false;
        for (int it = 0; it < TC_WAIT_LIMIT && !ok; ++it) ok = tc_try_wait(bar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, ERR_TIMEOUT);
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float v[CO];
        tc_load_row<CO>(tmem + ((uint32_t)(32 * warp) << 16), v);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");

        // epilogue: this thread's pixel p = 32 warp + lane of the tile (row
        // p / 8, column p % 8)
        const int img = t / tiles_img, r = t - img * tiles_img;
        const int p = 32 * warp + lane;
        const int py = (r / tiles_x) * FTH + p / FTW, px = (r % tiles_x) * FTW + p % FTW;
        const size_t pix = (size_t)img * H * W + (size_t)py * W + px;
        if (MODE == OUT_F32_NCHW) {
            float *o = static_cast<float *>(out);
#pragma unroll
            for (int co = 0; co < CO; ++co)
                if (co < nout)
                    o[((size_t)img * nout + co) * H * W + (size_t)py * W + px] = v[co] + bias[co];
        } else {
            bf16 *o = static_cast<bf16 *>(out) + pix * CO;
#pragma unroll
            for (int c8 = 0; c8 < CO / 8; ++c8) {
                __align__(16) bf16 h[8];
                if (MODE == OUT_RELU_BF16) {
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        h[e] = __float2bfloat16_rn(fmaxf(v[8 * c8 + e] + bias[8 * c8 + e], 0.f));
                } else {
                    __align__(16) bf16 mk[8];
                    *reinterpret_cast<uint4 *>(mk) =
                        *reinterpret_cast<const uint4 *>(mask + pix * CO + 8 * c8);
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        h[e] = __float2bfloat16_rn(__bfloat162float(mk[e]) > 0.f ? v[8 * c8 + e]
                                                                                  : 0.f);
                }
                *reinterpret_cast<uint4 *>(o + 8 * c8) = *reinterpret_cast<const uint4 *>(h);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy in flight at exit
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(G::TCOLS)
                     : "memory");
    }
}

// persistent launch of k_conv_tc: min(tiles, SMs x resident CTAs) CTAs
template <int CI, int CO, int MODE>
cudaError_t conv_tc(const bf16 *x, const bf16 *A, const float *bias, const bf16 *mask, void *out,
                    int H, int W, int nout, int batch, unsigned *err, cudaStream_t s)
{
    using G = TcGeo<CI, CO>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CI, CO, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, smem = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        // CTAs resident per SM, bounded by shared memory (1 KB per CTA is
        // reserved); TMEM (32 of 512 columns each) and registers allow more
        const int per = std::max(1, std::min(8, smem / (G::SMEM + 1024)));
        grid_cap = std::max(1, sms) * per;
    }
    const int ntiles = batch * (H / FTH) * (W / FTW);
    const int grid = std::min(ntiles, grid_cap);
    k_conv_tc<CI, CO, MODE><<<grid, TC_THREADS, G::SMEM, s>>>(x, A, bias, mask, out, H, W, nout,
                                                              ntiles, err);
    return cudaGetLastError();
}

// Weight gradient on tcgen05: dW[co, (tap, ci)] = sum_p dY[p, co] X[p + off(tap), ci]
// as, per tap, D[co, ci] += A[co, p] B[ci, p] with the reduction (K) over the
// 16 pixels of each MMA and the accumulator in TMEM across all the tiles a
// CTA walks (columns tap * CI .. tap * CI + CI - 1).  Both operands are read
// MN-major (the channel index contiguous in 16-byte core-matrix rows, one row
// per pixel), i.e. in the re-blocked NHWC layout the forward kernel stages:
// the 16 x 8 tile's dY as [co / 8][pixel][8] and its X halo as [ci / 8][halo
// pixel][8], so the 16 pixels (two tile rows) of K step k of tap (dy, dx)
// are two 8-pixel groups of the halo, 10 pixels apart, the first at halo
// pixel (2k + dy + 1) * 10 + dx + 1.  M = 128 is the smallest MMA height; rows co >= CO read other
// shared memory and land in accumulator rows no one reads.  One CTA per SM
// (9 * CI columns of TMEM), persistent over the tiles of all images; the
// bias gradient sum_p dY[p, co] is summed by threads from the staged tile.
template <int CI, int CO>
struct WgGeo {
    static constexpr int TP = FTH * FTW;                   // 128 pixels per tile
    static constexpr int YBUF = 16 * TP * 16;              // dY staging, room for 16 row groups
    static constexpr int BUF = YBUF + FHP * CI * 2;        // one staged tile (dY, X halo)
    static constexpr int BAR = 2 * BUF;
    static constexpr int SMEM = BAR + 16;
    static constexpr int NCOL = 9 * CI;
    static constexpr int TCOLS = NCOL <= 256 ? 256 : 512;  // TMEM allocation (power of 2)
    static_assert(CO % 8 == 0 && CO <= 128, "M rows of the MMA");
    static_assert(CI == 16 || CI == 32, "N of the MMA");
};

template <int CI, int CO>
__global__ void __launch_bounds__(TC_THREADS)
    k_wgrad_tc(const bf16 *__restrict__ dy, const bf16 *__restrict__ x, float *__restrict__ partial,
               int H, int W, int ntiles, unsigned *err)
{
    using G = WgGeo<CI, CO>;
    extern __shared__ __align__(1024) unsigned char wsm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(wsm + G::BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(wsm + G::BAR + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / FTW, tiles_img = tiles_x * (H / FTH);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem(tslot)),
                     "r"(G::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // stage tile t into buffer b: dY re-blocked [co/8][p][8] (p = 8 row +
    // column); X halo [ci/8][hp][8] (periodic wrap while staging).  dY chunk
    // i = p * YNJ + j: consecutive threads take consecutive 16-byte chunks of
    // global memory, and every thread keeps the same channel chunk j
    constexpr int YNJ = CO / 8;
    static_assert(TC_THREADS % YNJ == 0, "a thread's dY chunks share one channel chunk");
    const int yj = tid % YNJ;
    auto stage = [&](int t, int b) {
        const int img = t / tiles_img, r = t - img * tiles_img;
        const int y0 = (r / tiles_x) * FTH, x0 = (r % tiles_x) * FTW;
        unsigned char *buf = wsm + b * G::BUF;
        const bf16 *dyi = dy + (size_t)img * H * W * CO;
        for (int i = tid; i < G::TP * YNJ; i += TC_THREADS) {
            const int p = i / YNJ;
            cp_async16(buf + (yj * G::TP + p) * 16,
                       dyi + ((size_t)(y0 + p / FTW) * W + x0 + p % FTW) * CO + 8 * yj);
        }
        stage_tile<CI>(buf + G::YBUF, x + (size_t)img * H * W * CI, H, W, y0, x0, tid);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    int t = blockIdx.x;
    if (t < ntiles) stage(t, 0);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // kind::f16: D F32, A and B BF16, both MN-major (bits 15, 16), N = CI, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                           ((uint32_t)(CI >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    uint32_t phase = 0;
    bool first = true, ok = true;
    float bacc[8] = {};  // bias-gradient sums of this thread's channels 8 yj .. 8 yj + 7
    int b = 0;
    for (; t < ntiles; t += gridDim.x, b ^= 1) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned char *buf = wsm + b * G::BUF;
        if (tid == 0) {
            const uint32_t yb = tc_smem(buf), xb = tc_smem(buf + G::YBUF);
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dxi = tap % 3;
#pragma unroll 1
                for (int k = 0; k < G::TP / 16; ++k) {
                    // MN-major, no swizzle: the leading byte offset is the
                    // stride between 8-pixel (K) groups (128), the stride
                    // byte offset that between 8-channel (M/N) groups (as for
                    // K-major operands; checked against the CPU by a probe)
                    const uint64_t ad = tc_desc(yb + k * 256, 128, G::TP * 16);
                    const uint64_t bd = tc_desc(xb + ((2 * k + dy) * FHW + dxi) * 16, FHW * 16,
                                                FHP * 16);
                    tc_mma(tmem + tap * CI, ad, bd, idesc, (first && k == 0) ? 0u : 1u);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    tc_smem(bar))
                : "memory");
        }
        first = false;
        // stage the next tile into the other buffer while the MMAs run
        const int tn = t + gridDim.x;
        if (tn < ntiles) stage(tn, b ^ 1);
        // bias gradient: this thread's own staged dY chunks of the tile
        for (int i = tid; i < G::TP * YNJ; i += TC_THREADS) {
            __align__(16) bf16 h[8];
            *reinterpret_cast<uint4 *>(h) =
                *reinterpret_cast<const uint4 *>(buf + (yj * G::TP + i / YNJ) * 16);
#pragma unroll
            for (int e = 0; e < 8; ++e) bacc[e] += __bfloat162float(h[e]);
        }
        bool done = false;
        for (int it = 0; it < TC_WAIT_LIMIT && !done; ++it) done = tc_try_wait(bar, phase);
        phase ^= 1;
        if (__syncthreads_or(!done)) {
            if (tid == 0) atomicOr(err, ERR_TIMEOUT);
            ok = false;
            break;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the CTA's partial: [CO][9 CI] then the bias partial [CO]
    float *dst = partial + (size_t)blockIdx.x * (CO * G::NCOL + CO);
    if (ok && warp == 0) {  // TMEM lanes 0..31 hold rows co = lane
#pragma unroll 1
        for (int c0 = 0; c0 < G::NCOL; c0 += 16) {
            float v[16];
            tc_load_row<16>(tmem + c0, v);
            if (lane < CO)
#pragma unroll
                for (int e = 0; e < 16; ++e) dst[lane * G::NCOL + c0 + e] = v[e];
        }
    }
    // bias partial: sum over the threads that own channel chunk j (after
    // every read of the staging buffers, which now hold the per-thread sums)
    __syncthreads();
    float *bs = reinterpret_cast<float *>(wsm);
#pragma unroll
    for (int e = 0; e < 8; ++e) bs[tid * 8 + e] = bacc[e];
    __syncthreads();
    if (tid < CO) {
        const int j = tid / 8, e = tid % 8;
        float sacc = 0.f;
        for (int q = j; q < TC_THREADS; q += YNJ) sacc += bs[q * 8 + e];  // threads with yj == j
        dst[CO * G::NCOL + tid] = sacc;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(G::TCOLS)
                     : "memory");
    }
}

// one CTA per SM for 512-column allocations, two for 256
template <int CI, int CO>
cudaError_t wgrad_tc(const bf16 *dy, const bf16 *x, float *partial, int H, int W, int batch,
                     unsigned *err, int *nparts, cudaStream_t s)
{
    using G = WgGeo<CI, CO>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<CI, CO>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, smem = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int per = std::max(1, std::min(512 / G::TCOLS, smem / (G::SMEM + 1024)));
        grid_cap = std::max(1, sms) * per;
    }
    const int ntiles = batch * (H / FTH) * (W / FTW);
    const int grid = std::min(ntiles, grid_cap);
    *nparts = grid;
    k_wgrad_tc<CI, CO><<<grid, TC_THREADS, G::SMEM, s>>>(dy, x, partial, H, W, ntiles, err);
    return cudaGetLastError();
}

// one thread per weight of the largest layer (32 x 32 x 9 + 32)
constexpr int WGSUM_BLOCKS = (32 * 32 * 9 + 32 + 255) / 256;

// Sum the partials in a fixed order and scatter into the master layout
// (per layer W[co][ci][3][3] then b[co]; padded channels dropped).
__global__ void k_wgrad_sum(const float *__restrict__ partial, int nparts, int cin, int cout,
                            int cinp, int coutp, float *__restrict__ grad)
{
    const int N = 9 * cinp, stride = coutp * N + coutp;
    const int total = cout * cin * 9 + cout;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x) {
        int src;
        if (j < cout * cin * 9) {
            const int co = j / (cin * 9), rem = j - co * cin * 9, ci = rem / 9, tap = rem % 9;
            src = co * N + tap * cinp + ci;
        } else {
            src = coutp * N + (j - cout * cin * 9);
        }
        // eight interleaved running sums (loads in flight), combined in a
        // fixed order: the result does not depend on scheduling
        float s8[8] = {};
        int b = 0;
        for (; b + 8 <= nparts; b += 8)
#pragma unroll
            for (int q = 0; q < 8; ++q) s8[q] += partial[(size_t)(b + q) * stride + src];
        for (; b < nparts; ++b) s8[b & 7] += partial[(size_t)b * stride + src];
        grad[j] = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
    }
}

// master FP32 weights -> forward matrices A_l [COUTP][9][CINP] and the
// data-gradient matrices B_l [CINP][9][COUTP] with B[ci][t][co] = W[co][ci][8 - t]
__global__ void k_prep_weights(const float *__restrict__ master, bf16 *A0, bf16 *A1, bf16 *A2,
                               bf16 *B1, bf16 *B2, float *b0, float *b1, float *b2)
{
    bf16 *As[NL] = {A0, A1, A2};
    bf16 *Bs[NL] = {nullptr, B1, B2};
    float *bs[NL] = {b0, b1, b2};
    const int cins[NL] = {3, 32, 32}, couts[NL] = {32, 32, 3};
    const int cinps[NL] = {16, 32, 32}, coutps[NL] = {32, 32, 16};
    int off = 0;
    for (int l = 0; l < NL; ++l) {
        const int cin = cins[l], cout = couts[l], cinp = cinps[l], coutp = coutps[l];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < coutp * 9 * cinp;
             i += gridDim.x * blockDim.x) {
            const int co = i / (9 * cinp), rem = i - co * 9 * cinp, tap = rem / cinp,
                      ci = rem - tap * cinp;
            const float v = (co < cout && ci < cin) ? master[off + (co * cin + ci) * 9 + tap] : 0.f;
            As[l][i] = __float2bfloat16_rn(v);
            if (Bs[l]) {
                // element (co, tap, ci) of W feeds B[ci][8 - tap][co]
                Bs[l][(ci * 9 + (8 - tap)) * coutp + co] = __float2bfloat16_rn(v);
            }
        }
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < coutp; i += gridDim.x * blockDim.x)
            bs[l][i] = i < cout ? master[off + cout * cin * 9 + i] : 0.f;
        off += cout * cin * 9 + cout;
    }
}

// normalised FP32 NCHW state (3 channels) -> BF16 NHWC with 16 channels
__global__ void k_pack_nhwc(const float *__restrict__ xin, bf16 *__restrict__ x16, int HW,
                            int batch)
{
    const long long n = (long long)batch * HW;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long img = i / HW, p = i - img * HW;
        __align__(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c)
            v[c] = __float2bfloat16_rn(c < 3 ? xin[(img * 3 + c) * HW + p] : 0.f);
        uint4 *d = reinterpret_cast<uint4 *>(&x16[i * 16]);
        d[0] = *reinterpret_cast<uint4 *>(&v[0]);
        d[1] = *reinterpret_cast<uint4 *>(&v[8]);
    }
}

// residual r = x + net - target; loss partials (FP64) and d(loss)/d(net) as
// BF16 NHWC (16 channels)
__global__ void k_loss(const float *__restrict__ x, const float *__restrict__ net,
                       const float *__restrict__ target, bf16 *__restrict__ d16,
                       double *__restrict__ lpart, int HW, int batch, float scale, float w0,
                       float w1, float w2)
{
    const float wc[3] = {w0, w1, w2};
    const long long n = (long long)batch * HW;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long img = i / HW, p = i - img * HW;
        __align__(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long k = (img * 3 + c) * HW + p;
            const float r = wc[c] * (x[k] + net[k] - target[k]);
            s += (double)r * r;
            v[c] = __float2bfloat16_rn(scale * wc[c] * r);
        }
        uint4 *d = reinterpret_cast<uint4 *>(&d16[i * 16]);
        d[0] = *reinterpret_cast<uint4 *>(&v[0]);
        d[1] = *reinterpret_cast<uint4 *>(&v[8]);
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

// Training-input noise: x_noisy = x + sigma N(0, 1) on the channels whose
// loss weight is non-zero.  Normal variates from a counter-based generator:
// SplitMix64 (Steele, Lea and Flood 2014) of (seed, call, element) gives two
// uniforms, the Box-Muller transform one normal.  The corrected state is the
// noisy one (loss = |x_noisy + net(x_noisy) - target|^2), so the network
// learns to pull a perturbed state back toward the reference.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_add_noise(const float *__restrict__ x, float *__restrict__ xn, int HW,
                            int batch, float sigma, uint64_t key, float w0, float w1, float w2)
{
    const float wc[3] = {w0, w1, w2};
    const long long n = (long long)batch * 3 * HW;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)((i / HW) % 3);
        float v = x[i];
        if (wc[c] != 0.f) {
            const uint64_t h = splitmix64(key ^ splitmix64((uint64_t)i));
            const float u1 = ((float)(h >> 40) + 0.5f) * (1.0f / 16777216.0f);  // (0, 1)
            const float u2 = (float)((h >> 16) & 0xFFFFFF) * (1.0f / 16777216.0f);
            v += sigma * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
        }
        xn[i] = v;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// handle fields (FP32 deviation SoA) -> normalised NCHW input, and back
__global__ void k_gather_state(const float *__restrict__ r, const float *__restrict__ u,
                               const float *__restrict__ v, float *__restrict__ xo, int HW,
                               float sr, float su)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += gridDim.x * blockDim.x) {
        xo[i] = r[i] * sr;
        xo[HW + i] = u[i] * su;
        xo[2 * HW + i] = v[i] * su;
    }
}

__global__ void k_add_correction(float *__restrict__ r, float *__restrict__ u,
                                 float *__restrict__ v, const float *__restrict__ net, int HW,
                                 float sr, float su, float w0)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += gridDim.x * blockDim.x) {
        if (w0 != 0.f) r[i] += net[i] / sr;
        u[i] += net[HW + i] / su;
        v[i] += net[2 * HW + i] / su;
    }
}

}  // namespace
}  // namespace acm

using namespace acm;

struct acm_closure {
    int nx = 0, ny = 0, batch = 0;
    size_t nparam = 0;
    float scales[3] = {1.f, 1.f, 1.f};
    float weights[3] = {1.f, 1.f, 1.f};  // loss weight per channel (0 = not corrected)
    float *master = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    int adam_t = 0;
    bf16 *A[NL] = {}, *Bm[NL] = {};
    float *bias[NL] = {};
    bf16 *x16 = nullptr, *h1 = nullptr, *h2 = nullptr, *d16 = nullptr, *dh2 = nullptr,
         *dh1 = nullptr;
    float *net = nullptr, *xbuf = nullptr, *partial = nullptr;
    double *lpart = nullptr;
    unsigned *derr = nullptr;  // device error word (ERR_TIMEOUT of a bounded wait)
    float noise = 0.f;         // training-input noise (standard deviation, normalised units)
    uint64_t noise_seed = 0, noise_calls = 0;
    float *xnoisy = nullptr;
    int loss_blocks = 0, wg_parts = 0;
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_cl_err;

acm_status cfail(acm_closure *c, acm_status st, const std::string &m)
{
    if (c) c->err = m;
    else g_cl_err = m;
    return st;
}

#define CKC(c, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (void)cudaGetLastError(); /* a non-sticky failure must not outlive this call */ \
            return cfail((c), e_ == cudaErrorMemoryAllocation ? ACM_ENOMEM : ACM_ECUDA,      \
                         std::string(#call) + ": " + cudaGetErrorString(e_));               \
        }                                                                                   \
    } while (0)

size_t n_params()
{
    size_t n = 0;
    for (int l = 0; l < NL; ++l) n += (size_t)COUT[l] * CIN[l] * 9 + COUT[l];
    return n;
}

cudaError_t prep(acm_closure *c)
{
    k_prep_weights<<<32, 256, 0, c->stream>>>(c->master, c->A[0], c->A[1], c->A[2], c->Bm[1],
                                              c->Bm[2], c->bias[0], c->bias[1], c->bias[2]);
    return cudaGetLastError();
}

// net = closure(x) for normalised x (FP32 NCHW), keeping h1, h2
cudaError_t forward(acm_closure *c, const float *x)
{
    const int HW = c->nx * c->ny;
    k_pack_nhwc<<<256, 256, 0, c->stream>>>(x, c->x16, HW, c->batch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = conv_tc<16, 32, OUT_RELU_BF16>(c->x16, c->A[0], c->bias[0], nullptr, c->h1, c->ny,
                                           c->nx, 32, c->batch, c->derr, c->stream);
    if (e == cudaSuccess)
        e = conv_tc<32, 32, OUT_RELU_BF16>(c->h1, c->A[1], c->bias[1], nullptr, c->h2, c->ny,
                                           c->nx, 32, c->batch, c->derr, c->stream);
    if (e == cudaSuccess)
        e = conv_tc<32, 16, OUT_F32_NCHW>(c->h2, c->A[2], c->bias[2], nullptr, c->net, c->ny,
                                          c->nx, 3, c->batch, c->derr, c->stream);
    return e;
}

uint64_t splitmix64_host(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// loss and gradients (into c->grad) for input x and target (normalised)
cudaError_t loss_grad(acm_closure *c, const float *x, const float *target, double *loss)
{
    const int HW0 = c->nx * c->ny;
    if (c->noise > 0.f) {
        const uint64_t key = splitmix64_host(c->noise_seed) ^ (0xD1B54A32D192ED03ull * ++c->noise_calls);
        k_add_noise<<<256, 256, 0, c->stream>>>(x, c->xnoisy, HW0, c->batch, c->noise, key,
                                                c->weights[0], c->weights[1], c->weights[2]);
        x = c->xnoisy;
    }
    cudaError_t e = forward(c, x);
    if (e != cudaSuccess) return e;
    const int HW = c->nx * c->ny;
    const double nel = 3.0 * HW * c->batch;
    k_loss<<<c->loss_blocks, 256, 0, c->stream>>>(x, c->net, target, c->d16, c->lpart, HW,
                                                  c->batch, (float)(2.0 / nel), c->weights[0],
                                                  c->weights[1], c->weights[2]);
    // data gradients with the ReLU masks of h2 and h1
    e = conv_tc<16, 32, OUT_MASK_BF16>(c->d16, c->Bm[2], nullptr, c->h2, c->dh2, c->ny, c->nx,
                                       32, c->batch, c->derr, c->stream);
    if (e == cudaSuccess)
        e = conv_tc<32, 32, OUT_MASK_BF16>(c->dh2, c->Bm[1], nullptr, c->h1, c->dh1, c->ny,
                                           c->nx, 32, c->batch, c->derr, c->stream);
    if (e != cudaSuccess) return e;
    // weight gradients (tcgen05), per-CTA partials summed in a fixed order
    int np = 0;
    e = wgrad_tc<32, 16>(c->d16, c->h2, c->partial, c->ny, c->nx, c->batch, c->derr, &np,
                         c->stream);
    if (e != cudaSuccess) return e;
    k_wgrad_sum<<<WGSUM_BLOCKS, 256, 0, c->stream>>>(c->partial, np, CIN[2], COUT[2], CINP[2], COUTP[2],
                                           c->grad + (COUT[0] * CIN[0] * 9 + COUT[0]) +
                                               (COUT[1] * CIN[1] * 9 + COUT[1]));
    e = wgrad_tc<32, 32>(c->dh2, c->h1, c->partial, c->ny, c->nx, c->batch, c->derr, &np,
                         c->stream);
    if (e != cudaSuccess) return e;
    k_wgrad_sum<<<WGSUM_BLOCKS, 256, 0, c->stream>>>(c->partial, np, CIN[1], COUT[1], CINP[1], COUTP[1],
                                           c->grad + (COUT[0] * CIN[0] * 9 + COUT[0]));
    e = wgrad_tc<16, 32>(c->dh1, c->x16, c->partial, c->ny, c->nx, c->batch, c->derr, &np,
                         c->stream);
    if (e != cudaSuccess) return e;
    k_wgrad_sum<<<WGSUM_BLOCKS, 256, 0, c->stream>>>(c->partial, np, CIN[0], COUT[0], CINP[0], COUTP[0],
                                           c->grad);
    e = cudaGetLastError();
    if (e != cudaSuccess || !loss) return e;
    std::vector<double> lp(c->loss_blocks);
    e = cudaMemcpyAsync(lp.data(), c->lpart, sizeof(double) * c->loss_blocks,
                        cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    double s = 0.0;
    for (double v : lp) s += v;
    *loss = s / nel;
    return e;
}

// device error word: a bounded wait of a convolution gave up
acm_status check_err(acm_closure *c)
{
    unsigned f = 0;
    cudaError_t e = cudaMemcpyAsync(&f, c->derr, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cfail(c, ACM_ECUDA, cudaGetErrorString(e));
    if (f & ERR_TIMEOUT) return cfail(c, ACM_ETIMEOUT, "a tensor-core wait timed out");
    return ACM_OK;
}

void release(acm_closure *c)
{
    void *ptrs[] = {c->master, c->grad, c->adam_m, c->adam_v, c->x16, c->h1, c->h2, c->d16,
                    c->dh2, c->dh1, c->net, c->xbuf, c->partial, c->lpart, c->derr,
                    c->xnoisy};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < NL; ++l) {
        if (c->A[l]) cudaFree(c->A[l]);
        if (c->Bm[l]) cudaFree(c->Bm[l]);
        if (c->bias[l]) cudaFree(c->bias[l]);
    }
}

}  // namespace

extern "C" {

size_t acm_closure_num_params(void) { return n_params(); }

acm_status acm_closure_create(int nx, int ny, int batch, acm_closure **out)
{
    if (out) *out = nullptr;
    if (!out || nx < 16 || ny < 16 || nx % 16 || ny % 16 || batch < 1)
        return cfail(nullptr, ACM_EINVAL, "closure grid must be a multiple of 16 x 16, batch >= 1");
    acm_closure *c = new (std::nothrow) acm_closure();
    if (!c) return cfail(nullptr, ACM_ENOMEM, "host allocation failed");
    c->nx = nx;
    c->ny = ny;
    c->batch = batch;
    c->nparam = n_params();
    const size_t HW = (size_t)nx * ny, NB = HW * batch;
    const int tiles_img = (nx / FTW) * (ny / FTH);
    // weight-gradient partials: one per CTA, at most two CTAs per SM
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->wg_parts = std::min(tiles_img * batch, 2 * std::max(1, sms));
    c->loss_blocks = 512;
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    al((void **)&c->master, c->nparam * 4);
    al((void **)&c->grad, c->nparam * 4);
    al((void **)&c->adam_m, c->nparam * 4);
    al((void **)&c->adam_v, c->nparam * 4);
    for (int l = 0; l < NL; ++l) {
        al((void **)&c->A[l], (size_t)COUTP[l] * 9 * CINP[l] * 2);
        if (l > 0) al((void **)&c->Bm[l], (size_t)CINP[l] * 9 * COUTP[l] * 2);
        al((void **)&c->bias[l], (size_t)COUTP[l] * 4);
    }
    al((void **)&c->x16, NB * 16 * 2);
    al((void **)&c->h1, NB * 32 * 2);
    al((void **)&c->h2, NB * 32 * 2);
    al((void **)&c->d16, NB * 16 * 2);
    al((void **)&c->dh2, NB * 32 * 2);
    al((void **)&c->dh1, NB * 32 * 2);
    al((void **)&c->net, NB * 3 * 4);
    al((void **)&c->xbuf, NB * 3 * 4);
    al((void **)&c->partial, (size_t)c->wg_parts * (32 * 9 * 32 + 32) * 4);
    al((void **)&c->lpart, (size_t)c->loss_blocks * 8);
    al((void **)&c->derr, sizeof(unsigned));
    al((void **)&c->xnoisy, NB * 3 * 4);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // a failed allocation must not outlive this call
        release(c);
        delete c;
        return cfail(nullptr, e == cudaErrorMemoryAllocation ? ACM_ENOMEM : ACM_ECUDA,
                     std::string("closure allocation: ") + cudaGetErrorString(e));
    }
    *out = c;
    return ACM_OK;
}

acm_status acm_closure_set_stream(acm_closure *c, void *stream)
{
    if (!c) return cfail(nullptr, ACM_EINVAL, "null closure");
    const cudaStream_t next = static_cast<cudaStream_t>(stream);
    // the work already queued on the previous stream comes first
    CKC(c, acm::order_streams(c->stream, next));
    c->stream = next;
    return ACM_OK;
}

acm_status acm_closure_set_scales(acm_closure *c, const float *scales)
{
    if (!c || !scales) return cfail(c, ACM_EINVAL, "null argument");
    for (int i = 0; i < 3; ++i) {
        if (!(scales[i] > 0.f) || !std::isfinite(scales[i]))
            return cfail(c, ACM_EINVAL, "scales must be finite and > 0");
        c->scales[i] = scales[i];
    }
    if (c->scales[1] != c->scales[2]) return cfail(c, ACM_EINVAL, "u and v share one scale");
    return ACM_OK;
}

acm_status acm_closure_set_loss_weights(acm_closure *c, const float *w3)
{
    if (!c || !w3) return cfail(c, ACM_EINVAL, "null argument");
    for (int i = 0; i < 3; ++i) {
        if (!(w3[i] >= 0.f) || !std::isfinite(w3[i]))
            return cfail(c, ACM_EINVAL, "loss weights must be finite and >= 0");
        c->weights[i] = w3[i];
    }
    return ACM_OK;
}

acm_status acm_closure_set_input_noise(acm_closure *c, float sigma, uint64_t seed)
{
    if (!c) return cfail(nullptr, ACM_EINVAL, "null closure");
    if (!(sigma >= 0.f) || !std::isfinite(sigma)) return cfail(c, ACM_EINVAL, "sigma must be >= 0");
    c->noise = sigma;
    c->noise_seed = seed;
    c->noise_calls = 0;
    return ACM_OK;
}

acm_status acm_closure_set_weights(acm_closure *c, const float *w, size_t n)
{
    if (!c || !w) return cfail(c, ACM_EINVAL, "null argument");
    if (n != c->nparam) return cfail(c, ACM_EINVAL, "wrong number of parameters");
    CKC(c, cudaMemcpyAsync(c->master, w, n * 4, cudaMemcpyHostToDevice, c->stream));
    CKC(c, cudaMemsetAsync(c->adam_m, 0, n * 4, c->stream));
    CKC(c, cudaMemsetAsync(c->adam_v, 0, n * 4, c->stream));
    c->adam_t = 0;
    CKC(c, prep(c));
    CKC(c, cudaStreamSynchronize(c->stream));
    return ACM_OK;
}

acm_status acm_closure_get_weights(acm_closure *c, float *w, size_t n)
{
    if (!c || !w) return cfail(c, ACM_EINVAL, "null argument");
    if (n != c->nparam) return cfail(c, ACM_EINVAL, "wrong number of parameters");
    CKC(c, cudaMemcpyAsync(w, c->master, n * 4, cudaMemcpyDeviceToHost, c->stream));
    CKC(c, cudaStreamSynchronize(c->stream));
    return ACM_OK;
}

acm_status acm_closure_forward(acm_closure *c, const float *x_dev, float *net_dev)
{
    if (!c || !x_dev || !net_dev) return cfail(c, ACM_EINVAL, "null argument");
    CKC(c, forward(c, x_dev));
    CKC(c, cudaMemcpyAsync(net_dev, c->net, sizeof(float) * 3 * c->nx * c->ny * c->batch,
                           cudaMemcpyDeviceToDevice, c->stream));
    return ACM_OK;
}

acm_status acm_closure_loss_grad(acm_closure *c, const float *x_dev, const float *target_dev,
                                 double *loss, float *grad_host)
{
    if (!c || !x_dev || !target_dev) return cfail(c, ACM_EINVAL, "null argument");
    double l = 0.0;
    CKC(c, loss_grad(c, x_dev, target_dev, &l));
    if (acm_status st = check_err(c); st != ACM_OK) return st;
    if (loss) *loss = l;
    if (grad_host) {
        CKC(c, cudaMemcpyAsync(grad_host, c->grad, c->nparam * 4, cudaMemcpyDeviceToHost,
                               c->stream));
        CKC(c, cudaStreamSynchronize(c->stream));
    }
    return ACM_OK;
}

acm_status acm_closure_train_step(acm_closure *c, const float *x_dev, const float *target_dev,
                                  float lr, double *loss)
{
    if (!c || !x_dev || !target_dev) return cfail(c, ACM_EINVAL, "null argument");
    if (!(lr >= 0.f)) return cfail(c, ACM_EINVAL, "lr must be >= 0");
    CKC(c, loss_grad(c, x_dev, target_dev, loss));
    c->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)c->adam_t), c2 = 1.f - std::pow(b2, (float)c->adam_t);
    k_adam<<<32, 256, 0, c->stream>>>(c->master, c->grad, c->adam_m, c->adam_v, (int)c->nparam,
                                      lr, b1, b2, 1e-8f, c1, c2);
    CKC(c, cudaGetLastError());
    CKC(c, prep(c));
    return ACM_OK;
}

acm_status acm_closure_gather(acm_closure *c, acm_handle *h, float *x_dev)
{
    if (!c || !h || !x_dev) return cfail(c, ACM_EINVAL, "null argument");
    if (acm_sync(h) != ACM_OK) return cfail(c, ACM_ESTATE, "solver handle is not healthy");
    const int HW = c->nx * c->ny;
    for (int b = 0; b < c->batch; ++b) {
        float *r, *u, *v;
        int nx, ny;
        if (handle_fields_f32(h, b, &r, &u, &v, &nx, &ny) != ACM_OK || nx != c->nx || ny != c->ny)
            return cfail(c, ACM_EINVAL, "handle run is not an FP32 2D grid of the closure's size");
        k_gather_state<<<128, 256, 0, c->stream>>>(r, u, v, x_dev + (size_t)b * 3 * HW, HW,
                                                   c->scales[0], c->scales[1]);
    }
    CKC(c, cudaGetLastError());
    return ACM_OK;
}

acm_status acm_closure_apply(acm_closure *c, acm_handle *h)
{
    if (!c || !h) return cfail(c, ACM_EINVAL, "null argument");
    acm_status st = acm_closure_gather(c, h, c->xbuf);
    if (st != ACM_OK) return st;
    CKC(c, forward(c, c->xbuf));
    const int HW = c->nx * c->ny;
    for (int b = 0; b < c->batch; ++b) {
        float *r, *u, *v;
        int nx, ny;
        handle_fields_f32(h, b, &r, &u, &v, &nx, &ny);
        k_add_correction<<<128, 256, 0, c->stream>>>(r, u, v, c->net + (size_t)b * 3 * HW, HW,
                                                     c->scales[0], c->scales[1], c->weights[0]);
    }
    CKC(c, cudaGetLastError());
    // the handle's next step reads the fields: wait (and check the error word)
    return check_err(c);
}

acm_status acm_closure_destroy(acm_closure *c)
{
    if (!c) return ACM_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    release(c);
    delete c;
    return ACM_OK;
}

const char *acm_closure_last_error(const acm_closure *c)
{
    return c ? c->err.c_str() : g_cl_err.c_str();
}

}  // extern "C"
