// Node-pair arithmetic of the line-marching 2D kernels.  A lane's two nodes
// travel as P2<T>: float2 for FP32 storage, issued as packed two-lane FP32
// instructions (FFMA2/FADD2/FMUL2, sm_100 and later), double2 for FP64 (two
// scalar operations).  Every operation is an explicit round-to-nearest
// intrinsic, never contracted by the compiler, so a node's value does not
// depend on where its arithmetic was inlined.
#pragma once

#include <cuda_runtime.h>

namespace acm {
namespace pair {

template <typename T>
struct P2T;
template <>
struct P2T<float> {
    using type = float2;
};
template <>
struct P2T<double> {
    using type = double2;
};
template <typename T>
using P2 = typename P2T<T>::type;

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename T>
__device__ __forceinline__ P2<T> splat(T a)
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
// a - b
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ double2 sub2(double2 a, double2 b)
{
    return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}
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

// asynchronous global -> shared copy of N bytes (4, 8 or 16), grouped by
// commit; a wait leaves at most W newer groups pending
template <int N>
__device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(N)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int W>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(W) : "memory");
}

constexpr unsigned FULL = 0xffffffffu;

// x-neighbours of a lane's pair p = (a, b) from the adjacent lanes:
// W = (west of a, a), E = (b, east of b).  Lanes 0 and 31 get their own
// values in place of the missing neighbour.
template <typename T>
__device__ __forceinline__ void shuffle_we(P2<T> p, P2<T> &W, P2<T> &E)
{
    const T up = __shfl_up_sync(FULL, p.y, 1);
    const T dn = __shfl_down_sync(FULL, p.x, 1);
    W = mk(up, p.x);
    E = mk(p.y, dn);
}

}  // namespace pair
}  // namespace acm
