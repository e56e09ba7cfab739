// Internal declarations shared by the libacm translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/acm.h"

namespace acm {

// Field slots in every buffer (structure of arrays).
enum { F_R = 0, F_U = 1, F_V = 2, F_W = 3, F_PHI = 4, NFIELD = 5 };

// Device error word bits.
enum : unsigned { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u };

template <typename T>
struct Fields {
    T *f[NFIELD];
};

// Per-run coefficients, stored in both precisions so that kernels never
// convert (a double->float conversion runs on the FP64 pipe, which is narrow
// on GB300).
enum {
    C_RHO0 = 0, C_DT, C_CS2, C_NU,
    C_SATC,   // 1/2 c_s^2 dt^2 if the continuity SAT is on, else 0 (Eq. 2.10)
    C_SATM,   // nu + 1/2 c_s^2 dt if the momentum SAT is on, else 0 (Eq. 2.11)
    C_NUDT,   // nu dt
    C_GX, C_GY, C_GZ, C_LIDX, C_LIDY, C_LIDZ,
    C_A, C_KAPPA, C_M,
    C_WET,    // 2 (2/W) cos(theta): wetting term of the ghost order parameter
    C_BQA, C_BQB,  // body-force factor A + B phi^n: (1, 0), or the Boussinesq
                   // drop force (Section 3.5) beta/2 (1 + phi), beta = 2 (r-1)/(r+1)
    NCOEF
};

// Per-run description used by the 2D tile kernels and the reductions.
struct RunDesc {
    int nx, ny, nz;
    int bc[6];          // ACM_BC_* per face
    long long off;      // element offset of the run inside each field pool
    long long px, py;   // storage pitch (elements) in x and y (3D: padded)
    int pad;            // ghost layers in x and y (3D TMA layout), 0 in 2D
    int zg;             // ghost planes below (and above) the run: 2 for a 3D
                        // sub-domain (ACM_BC_HALO z faces), else 0
    double rho0, dt, cs2, nu;
    double g[3], lid[3];
    double a, kappa, M; // two-phase coefficients
    int sat_c, sat_m;
    int two_phase;
    float cf[NCOEF];
    double cd[NCOEF];
};

template <typename T>
__host__ __device__ __forceinline__ const T *coefs(const RunDesc &R);
template <>
__host__ __device__ __forceinline__ const float *coefs<float>(const RunDesc &R)
{
    return R.cf;
}
template <>
__host__ __device__ __forceinline__ const double *coefs<double>(const RunDesc &R)
{
    return R.cd;
}

// 2D tile geometry (outputs per tile).
constexpr int T2X = 32;
#ifndef ACM_T2Y
#define ACM_T2Y 32
#endif
constexpr int T2Y = ACM_T2Y;
constexpr int T2THREADS = 256;

// 3D z-marching kernel geometry.
constexpr int T3X = 32;
constexpr int T3PAD = 2;     // ghost layers in x and y of the 3D layout
constexpr int T3SLOTS = 5;   // input planes resident/in flight per CTA

struct Tuning {
    int zchunks = 0;       // 3D: z-chunks per column (0 = chunks of 16 planes)
    int t3y = 16;          // 3D: tile height (8 or 16)
    int graph_steps = 64;  // steps per captured CUDA graph (even)
    int blocks = 0;        // 2D: persistent CTAs (0 = occupancy x SMs)
    int line2d = 1;        // 2D single-phase periodic: line-marching kernel where it applies
};

// Launchers (defined in the kernel translation units).
template <typename T>
cudaError_t launch_step2d(const RunDesc *druns, const int4 *dwork, int nwork, int two_phase,
                          Fields<T> in, Fields<T> out, unsigned *derr, int blocks,
                          cudaStream_t s);
template <typename T>
int step2d_max_blocks_per_sm(int two_phase);

// 2D single-phase periodic runs whose width is a multiple of line2d_width():
// one warp per (run, x0, y0, rows) item of a strip of line2d_width() columns
// and at most line2d_rows() rows.
int line2d_rows();
int line2d_width();
template <typename T>
void line2d_prepare();  // launch attributes (before any capture)
// 2D two-phase runs periodic on all faces (nx >= 64, ny >= 16): one warp per
// (run, x0, y0, rows) item; a strip holds 64 columns from x0 (which may be
// -4) and writes the line2d_tp_stride() columns x0+4 .. of at most
// line2d_tp_rows() rows.
int line2d_tp_rows();
int line2d_tp_stride();
template <typename T>
void line2d_tp_prepare();
template <typename T>
cudaError_t launch_line2d_tp(const RunDesc *druns, const int4 *dwork, int nwork, bool gen,
                             Fields<T> in, Fields<T> out, unsigned *derr, cudaStream_t s);
template <typename T>
cudaError_t launch_line2d(const RunDesc *druns, const int4 *dwork, int nwork, bool gen,
                          Fields<T> in, Fields<T> out, unsigned *derr, cudaStream_t s);

template <typename T>
cudaError_t launch_step3d(const CUtensorMap *maps_in, Fields<T> out, const RunDesc &run,
                          unsigned *derr, int zchunks, int t3y, int sms, cudaStream_t s);
template <typename T>
int step3d_max_blocks_per_sm(int t3y);

template <typename T>
cudaError_t launch_reduce(const RunDesc *druns, int nruns, int dim, Fields<T> cur, const T *pu,
                          const T *pv, const T *pw, double *dpartials, int blocks_per_run,
                          double *dout, cudaStream_t s);

// 3D two-phase step (five launches: mu, Delta rho, momentum + phi*, mu*,
// phi^{n+1}); mu, phs, dr are scratch fields of the run's storage size.
template <typename T>
void tp3d_prepare();  // launch attributes of the 3D two-phase step (before any capture)
template <typename T>
cudaError_t launch_tp3d(const RunDesc &R, Fields<T> in, Fields<T> out, T *mu, T *phs, T *dr,
                        unsigned *err, int sms, cudaStream_t s);

// The MAMEs predictor-corrector (comparison scheme), periodic 2D runs over
// the same (run, tile) work list as launch_step2d.
template <typename T>
cudaError_t launch_mames2d(const RunDesc *druns, const int4 *dwork, int nwork, Fields<T> in,
                           Fields<T> out, unsigned *derr, int blocks, cudaStream_t s);
template <typename T>
int mames2d_max_blocks_per_sm();

// Halo exchange of 3D sub-domains (runs 0..nruns-1 form a ring along z):
// copies the two boundary planes of every run into the ghost planes of its
// neighbours, all four fields of f, one launch.
template <typename T>
cudaError_t launch_halo(const RunDesc *druns, int nruns, long long plane, Fields<T> f,
                        cudaStream_t s);

// Eq. (3.2) error sums of one field against an unpadded reference, and the
// Laplace-law diagnostics of two-phase runs (acm_diag.cu); partials hold 2
// (error) or 9 x nruns (Laplace) doubles per block.
constexpr int LAPLACE_PARTIALS = 9;
template <typename T>
cudaError_t launch_error_l2(const RunDesc &R, const T *f, const double *ref, double *partials,
                            int blocks, double *out, cudaStream_t s);
template <typename T>
cudaError_t launch_laplace(const RunDesc *druns, int nruns, int dim, const T *phi, const T *rho,
                           double *partials, int blocks, double *out, cudaStream_t s);


template <typename T>
cudaError_t launch_import(const double *src, T *dst, const RunDesc &run, int dim, double shift,
                          cudaStream_t s);
template <typename T>
cudaError_t launch_export(const T *src, double *dst, const RunDesc &run, int dim, double shift,
                          cudaStream_t s);

// FP32 2D fields of run `run` in the handle's current buffer (for the
// learned closure); ACM_EINVAL unless the handle is a 2D FP32 grid.
acm_status handle_fields_f32(acm_handle *h, int run, float **r, float **u, float **v, int *nx,
                             int *ny);

// Make stream `next` wait, on the device, for the work queued so far on
// stream `prev` (an event recorded on prev; no host wait).
cudaError_t order_streams(cudaStream_t prev, cudaStream_t next);

}  // namespace acm
