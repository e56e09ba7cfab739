/*
 * acm.h -- C ABI of libacm, a GB300 (sm_103a) solver for the simplified
 * "more actual macroscopic equations" (SMAMEs) of Huang, "Towards the simplest
 * simulation of incompressible viscous flows inspired by the lattice Boltzmann
 * method" (arXiv:2012.03525).
 *
 * One time step advances density (pressure p = rho c_s^2) and velocity on a
 * collocated uniform grid (Section 2):
 *   Eq. (2.10)  rho^{n+1} = rho^n - dt d_a(rho u_a)^n + 1/2 c_s^2 dt^2 d_aa rho^n
 *   Eq. (2.11)  (rho u_a)^{n+1} = (rho u_a)^n - dt d_b(rho u_a u_b + rho c_s^2 delta_ab)^n
 *               + nu dt d_bb(rho u_a)^n - (nu + 1/2 c_s^2 dt)(d_a rho^{n+1} - d_a rho^n)
 *               + dt rho^{n+1} g_a                 (body force, Section 2)
 *               + dt F_ST,a, F_ST = -phi d_a mu    (two-phase, Section 2)
 * with second-order centred differences (Eqs. 2.12-2.13).  The two-phase
 * order parameter phi follows the Cahn-Hilliard equation (Eq. 2.14) with
 * mu = 4 a phi (phi^2 - 1) - kappa d_aa phi, a = 3 sigma / (4W),
 * kappa = 3 sigma W / 8, discretised with lattice-weighted isotropic
 * (D2Q9) operators and advanced by a two-stage (Heun) Runge-Kutta step.
 *
 * Units: lattice units with delta_x = 1 and delta_t = params.dt, so the
 * lattice speed is c = 1/dt and c_s^2 = c^2/3 (Section 2, after Eq. 2.1).
 *
 * Conventions for every call:
 *   - every function returns an acm_status; nothing throws across the ABI;
 *   - host arrays are caller-owned, contiguous, [z][y][x] with x fastest,
 *     nx*ny*nz doubles per field; NULL is allowed for fields a run does not
 *     have (w in 2D, phi in single-phase runs) and, for acm_fields, for any
 *     field the caller does not want;
 *   - device memory belongs to the handle; the solver's arithmetic runs only
 *     on the GPU -- there is no CPU path;
 *   - acm_step is asynchronous on the handle's stream; a numerical blow-up
 *     (non-finite value) detected by the step kernels is reported as
 *     ACM_EUNSTABLE by the next synchronising call (acm_sync, acm_fields,
 *     acm_reduce_mass) and stays sticky until acm_set_fields;
 *   - a handle may be used by one host thread at a time.
 */
#ifndef ACM_H
#define ACM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct acm_handle acm_handle;

typedef enum {
    ACM_OK = 0,
    ACM_EINVAL = -1,    /* invalid argument or unsupported combination */
    ACM_ENOMEM = -2,    /* device or host allocation failed */
    ACM_ECUDA = -3,     /* a CUDA runtime/driver call failed */
    ACM_EUNSTABLE = -4, /* a non-finite value appeared in the fields */
    ACM_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
    ACM_ESTATE = -6     /* call out of order (e.g. step before set_fields) */
} acm_status;

/* boundary condition of one face.  ACM_BC_HALO marks the z faces of a 3D
 * sub-domain: the run is one z-slab of a larger periodic grid, and its two
 * neighbour planes beyond each z face are ghost planes copied from the
 * adjacent slabs (see acm_batch_create).  ACM_BC_SYMMETRY is a mirror plane
 * through the first/last node of the axis (the quarter domains of Sections
 * 3.6-3.7): the node beyond it is the image of the node one inside, rho,
 * phi, mu and the tangential velocity are even across it, the normal
 * velocity is odd and zero on it. */
enum {
    ACM_BC_PERIODIC = 0,
    ACM_BC_WALL = 1,
    ACM_BC_LID = 2,
    ACM_BC_HALO = 3,
    ACM_BC_SYMMETRY = 4
};

/* storage/arithmetic precision of the fields */
enum {
    ACM_FP64 = 0,     /* rho - rho0 and u stored and updated in FP64 */
    ACM_FP32_DEV = 1  /* rho - rho0 and u stored and updated in FP32 (deviation
                         form: the O(Ma^2) density signal keeps its digits) */
};

typedef struct {
    int dim;            /* 2 or 3 */
    int nx, ny, nz;     /* nodes per direction (nz = 1 in 2D); periodic faces
                           have no duplicated end node, wall faces put the
                           wall on the first/last node */
    double dt;          /* delta_t in lattice units (delta_x = 1); c_s^2 = 1/(3 dt^2) */
    double nu;          /* kinematic viscosity (lattice units) */
    double rho0;        /* reference density; fields are stored as rho - rho0 */
    int bc[6];          /* faces -x,+x,-y,+y,-z,+z: ACM_BC_*; a periodic face
                           must be paired with a periodic face */
    double lid_u[3];    /* wall velocity of ACM_BC_LID faces */
    double g[3];        /* body force per unit mass: + dt rho^{n+1} g in Eq. (2.11) */
    int two_phase;      /* 0 or 1: add phi, F_ST and the Cahn-Hilliard update */
    double sigma;       /* surface tension */
    double W;           /* interface width */
    double M;           /* mobility */
    int precision;      /* ACM_FP64 or ACM_FP32_DEV */
    int sat_mask;       /* bit0: continuity SAT of Eq. (2.10), bit1: momentum
                           SAT of Eq. (2.11); 3 = the paper's scheme, other
                           values reproduce the ablation of Section 3.1 */
    double theta_deg;   /* two-phase contact angle of wall faces (degrees):
                           d_n phi = -(2/W) cos(theta) (1 - phi_w^2), d_n mu = 0
                           (Section 2); 90 = neutral wetting */
    int scheme;         /* ACM_SCHEME_SMAMES: the one-step update, Eqs.
                           (2.10)-(2.11); ACM_SCHEME_MAMES: the predictor-
                           corrector of Eqs. (2.6)-(2.9) that it replaces
                           (comparison scheme: 2D, periodic, single-phase,
                           no body force; sat_mask is ignored) */
    double rho_ratio;   /* two-phase: 0 = the body force acts on both phases
                           (+ dt rho^{n+1} g); r > 0 = Boussinesq drop force
                           of Section 3.5 for a drop/ambient density ratio r:
                           the force acts on the drop (phi = +1) phase only,
                           scaled by 2 (r - 1)/(r + 1), i.e.
                           + dt rho^{n+1} g 2 (r - 1)/(r + 1) (1 + phi^n)/2 */
} acm_params;

/* time-stepping scheme */
enum { ACM_SCHEME_SMAMES = 0, ACM_SCHEME_MAMES = 1 };

/* Supported combinations (others return ACM_EINVAL):
 *   dim 2: periodic, wall or lid faces; single- or two-phase (walls of
 *          two-phase runs carry the wetting condition); FP64 or FP32_DEV;
 *   dim 3: single-phase: periodic x and y faces, z periodic or
 *          ACM_BC_HALO on both z faces; two-phase (D3Q19 isotropic
 *          operators) with z periodic or walls on both z faces (wetting
 *          condition, stationary) and x, y faces periodic or symmetry
 *          planes (both faces of an axis); FP64 or FP32_DEV.          */

/* Create a solver for ONE grid.  Validates the parameters, allocates the
 * double-buffered device fields on the current CUDA device and returns the
 * handle in *out (NULL on failure).  The handle creates its own non-blocking
 * CUDA stream (replace it with acm_set_stream).  Fields are undefined until
 * acm_set_fields.  A grid that does not fit in device memory returns
 * ACM_ENOMEM with everything it allocated released; the failed allocation is
 * not left behind as the CUDA runtime's last error, so the context stays
 * usable for other handles. */
acm_status acm_create(const acm_params *params, acm_handle **out);

/* Elements of the precision's type (double for ACM_FP64, float for
 * ACM_FP32_DEV) in ONE field buffer of a single-grid solver for PARAMS: the
 * storage acm_create_ext expects per field and buffer.  2D storage is the
 * grid itself ([y][x], unpadded); 3D storage is padded by two ghost layers
 * in x and y ([z][ny + 4][px], px = nx + 4 rounded up to a multiple of 8).
 * Host-only: needs no GPU.  ACM_EINVAL for invalid parameters. */
acm_status acm_storage_elems(const acm_params *params, size_t *elems);

/* Like acm_create, but the field storage is device memory the CALLER owns
 * (e.g. tensors of a framework's caching allocator), and the handle runs on
 * the caller's stream:
 *   dev_fields  10 device pointers, buffer-major: dev_fields[5 b + f] is
 *               field f of time-level buffer b (b = 0, 1; f = 0 rho - rho0,
 *               1 u, 2 v, 3 w, 4 phi).  Each holds acm_storage_elems(params)
 *               elements and starts on a 256-byte boundary (the 3D step
 *               stages planes by TMA).  Entries of fields the run does not
 *               have (w in 2D, phi in single-phase runs) must be NULL; the
 *               ten buffers must not overlap.
 *   stream      cudaStream_t every call of the handle uses (NULL = legacy
 *               default stream); the handle creates no stream of its own.
 * The library zero-fills the buffers at creation (on STREAM), never frees
 * them (acm_destroy leaves them to the caller, who must keep them alive
 * until then) and allocates only its small bookkeeping arrays (run
 * descriptor, error word, reduction partials, one host-transfer staging
 * field).  After acm_set_fields and acm_step, buffer acm_current_buffer(h)
 * holds the state in the storage layout above.  Scratch fields of the 3D
 * two-phase step are still allocated by the library.  ACM_EINVAL for a
 * missing, misaligned or superfluous pointer. */
acm_status acm_create_ext(const acm_params *params, void *const *dev_fields, void *stream,
                          acm_handle **out);

/* Index (0 or 1) of the buffer holding the current state. */
int acm_current_buffer(const acm_handle *h);

/* Stability pre-check (not in the paper, which reports blow-ups of
 * under-resolved runs in Sections 3.1 and 3.3).  A von Neumann analysis of
 * the forward-Euler step with centred advection and diffusion (the velocity
 * equation of Eq. 2.11 linearised about a uniform flow u) gives two
 * necessary conditions: |u|^2 dt <= 2 nu and 2 dim nu dt <= 1 (delta_x = 1).
 * *ratio receives max(max_nodes |u|^2 dt / (2 nu), 2 dim nu dt) over the N
 * nodes of the host arrays u, v, w (w may be NULL in 2D): a value above 1
 * means the run is expected to blow up.  acm_set_fields applies the same
 * check to every run's initial velocity and, when the ratio exceeds 1,
 * still returns ACM_OK but leaves a warning in acm_last_error.  Host-only:
 * needs no GPU. */
acm_status acm_stability_ratio(const acm_params *params, const double *u, const double *v,
                               const double *w, size_t n, double *ratio);

/* Create a solver for NRUNS grids (a batch).
 * dim 2: independent runs.  params[r] describes run r; all runs share
 *   precision and two_phase.  Grid sizes and physical parameters may differ
 *   per run.  One acm_step advances every run by one step with one
 *   persistent kernel launch over a (run, tile) work list.
 * dim 3: sub-domains of ONE periodic grid split along z (the slab
 *   decomposition a multi-GPU run would use, emulated on one GPU).  Every
 *   run has ACM_BC_HALO z faces, the same nx, ny and physical parameters;
 *   run r covers the next nz_r planes, and run r+1 (run 0 after the last)
 *   is its upper neighbour.  Each run stores two ghost planes beyond each z
 *   face.  One acm_step first copies, for every pair of neighbours, the two
 *   boundary planes of each into the ghost planes of the other (one
 *   halo-copy kernel launch: the exchange step of Eqs. 2.10-2.11, whose
 *   stencil reaches two planes through Delta rho), then advances each slab
 *   with its own step kernel launch.  The result is bitwise equal to the
 *   same grid run as one periodic handle. */
acm_status acm_batch_create(const acm_params *params, int nruns, acm_handle **out);

/* Use this CUDA stream (a cudaStream_t, may be NULL for the legacy default
 * stream) for every later call on the handle.  Invalidates captured graphs.
 * Work already queued on the previous stream runs first: the handle's own
 * stream is synchronised and destroyed; a caller's stream is ordered before
 * the new one on the device (an event, no host wait). */
acm_status acm_set_stream(acm_handle *h, void *stream);

/* Number of runs in the handle (1 for acm_create). */
int acm_nruns(const acm_handle *h);

/* Copy the initial state of run RUN from host memory: absolute density rho
 * and velocity components (w ignored in 2D; phi required iff two_phase).
 * Clears a sticky ACM_EUNSTABLE and resets the step counter of the handle.
 * Synchronous. */
acm_status acm_set_fields(acm_handle *h, int run, const double *rho, const double *u,
                          const double *v, const double *w, const double *phi);

/* Advance every run by NSTEPS time steps (asynchronous on the handle's
 * stream; long runs are replayed from a captured CUDA graph). */
acm_status acm_step(acm_handle *h, int64_t nsteps);

/* Wait for the handle's stream and report a blow-up or a device timeout. */
acm_status acm_sync(acm_handle *h);

/* Copy the current state of run RUN to host memory (absolute density).
 * Any pointer may be NULL.  Synchronous. */
acm_status acm_fields(acm_handle *h, int run, double *rho, double *u, double *v, double *w,
                      double *phi);

/* FP64 integral diagnostics of every run (Section 3: kinetic energy of the
 * Taylor-Green test, the steady-state criterion of the cavity test):
 *   out[8*r + 0] = sum rho
 *   out[8*r + 1..3] = sum rho u, sum rho v, sum rho w
 *   out[8*r + 4] = E_k = 1/2 sum |u|^2
 *   out[8*r + 5] = max over nodes of | |u^n| - |u^{n-1}| | (change made by
 *                  the last step; 0 before the first step)
 *   out[8*r + 6] = max |u|
 *   out[8*r + 7] = number of nodes holding a non-finite value of rho or u
 * OUT is a host array of 8 * acm_nruns(h) doubles.  Deterministic: the
 * summation order does not depend on timing.  FP64 storage: every operation
 * in FP64.  FP32 storage: per node FP32 arithmetic only (GB300's FP64 pipe
 * is narrow), with compensated FP32 sums carrying ~48 significant bits and
 * the products rho' u_a added exactly, combined in FP64 per thread; out[5]
 * has ~1e-7 relative precision (FP32 denominator |u| + |u_prev|).
 * Synchronous. */
acm_status acm_reduce_mass(acm_handle *h, double *out);

/* Velocity error of run RUN against a reference field (Eq. 3.2 of Section
 * 3.1, written there for u of the Taylor-Green vortex):
 *   out[a] = sqrt( sum (u_a - u_a,ref)^2 / sum u_a,ref^2 ),  a = 0, 1, 2,
 * summed over every node in FP64 on the GPU.  u_ref, v_ref, w_ref are host
 * arrays like acm_set_fields' (a NULL reference gives out[a] = 0; w_ref is
 * ignored in 2D).  A zero reference norm gives the absolute root-sum-square
 * error.  Synchronous. */
acm_status acm_reduce_error(acm_handle *h, int run, const double *u_ref, const double *v_ref,
                            const double *w_ref, double *out);

/* Laplace-law diagnostics of every run of a two-phase handle (FP64 on the
 * GPU), from phi and mu = 4 a phi (phi^2 - 1) - kappa Lap_iso(phi) of
 * Section 2 (Eq. 2.14's chemical potential, same isotropic Laplacian as the
 * step; wall nodes, whose Laplacian needs the wall's ghost values, are left
 * out):
 *   out[8 r + 0] = A = sum (1 + phi)/2: area (2D) or volume (3D) of the
 *                  phi > 0 phase
 *   out[8 r + 1] = R_eff = sqrt(A / pi) (2D) or (3 A / (4 pi))^(1/3) (3D)
 *   out[8 r + 2] = mu_G = sum mu (1 - phi^2) / sum (1 - phi^2), mu weighted
 *                  by the interface profile: for a tanh interface it is the
 *                  curvature term of mu, (dim - 1) sigma / (2 R), and at
 *                  equilibrium the uniform mu_0
 *   out[8 r + 3] = mean mu over nodes with phi > 0.95 (inside the drop)
 *   out[8 r + 4] = mean mu over nodes with phi < -0.95 (outside)
 *   out[8 r + 5] = p_in - p_out, p = c_s^2 rho averaged over the same sets
 *   out[8 r + 6] = the Laplace law's mu_0 = (dim - 1) sigma / (2 R_eff)
 *                  (2D: sigma / (2R), 3D: sigma / R; the jump of
 *                  p + phi mu - a (phi^2 - 1)^2 across the interface is
 *                  2 mu_0)
 *   out[8 r + 7] = number of nodes with phi > 0.95
 * Means over an empty set are 0.  ACM_EINVAL for single-phase handles.
 * Synchronous. */
acm_status acm_reduce_laplace(acm_handle *h, double *out);

/* Launch tuning knobs (the autotuner of the Python layer sweeps them).
 * Changing a knob drops captured graphs.  Returns ACM_EINVAL for an unknown
 * key or an out-of-range value. */
enum {
    ACM_TUNE_ZCHUNKS = 1,     /* 3D: z-chunks per x-y column (>= 1; 0 = chunks of 16 planes) */
    ACM_TUNE_T3Y = 2,         /* 3D: tile height in y, 8 or 16 */
    ACM_TUNE_GRAPH_STEPS = 3, /* steps per captured CUDA graph, even, >= 2; 0 disables graphs */
    ACM_TUNE_BLOCKS = 4,      /* 2D: persistent CTAs per launch (0 = fill the GPU) */
    ACM_TUNE_LINE2D = 5       /* 2D runs periodic on all faces (single-phase: width a
                                 multiple of 64; two-phase: nx >= 64, ny >= 16): 1 steps
                                 them with the line-marching kernels (the default for
                                 FP32_DEV storage), 0 with the tile kernel (the default
                                 for FP64) */
};
acm_status acm_set_tuning(acm_handle *h, int key, int value);

/* Current value of a tuning knob (-1 for an unknown key or a NULL handle). */
int acm_get_tuning(const acm_handle *h, int key);

/* Autotuner: time NSTEPS steps of every candidate launch shape (3D: tile
 * height x z-chunking; 2D: persistent CTA count of the tile kernel and,
 * where it applies, the line-marching kernel) with CUDA events on the
 * handle's stream, keep the fastest (readable with acm_get_tuning) and
 * restore the fields as they were (trial steps run on a device copy, which
 * this call allocates and frees).  *best_ms_per_step receives the winner's
 * time per step.  Synchronous; needs acm_set_fields first. */
acm_status acm_autotune(acm_handle *h, int nsteps, double *best_ms_per_step);

/* Step counter since acm_set_fields. */
int64_t acm_step_count(const acm_handle *h);

/* Free every resource of the handle (NULL is a no-op). */
acm_status acm_destroy(acm_handle *h);

/* Last error message of the handle, or of the calling thread when h is NULL
 * (e.g. after a failed create).  Never NULL. */
const char *acm_last_error(const acm_handle *h);

/* Box-filter restriction of every run of FINE (2D, single-phase, one grid
 * size) by FACTOR x FACTOR blocks, with a change of lattice units: the block
 * means of u, v are multiplied by U_SCALE and of rho - rho0 by RHO_SCALE
 * (same delta_t, delta_x times FACTOR: U_SCALE = 1/FACTOR, and the pressure
 * p = c_s^2 (rho - rho0) is kept when RHO_SCALE = 1/FACTOR^2).  The result
 * goes into the current fields of COARSE (same number of runs, grid =
 * fine / factor; resets its step counter like acm_set_fields) and/or into
 * OUT_DEV as normalised FP32 [nruns][3][ny/factor][nx/factor]
 * (s_rho (rho - rho0), s_u u, s_u v with scales3 = {s_rho, s_u, s_u}).  Used
 * to start coarse runs from, and to build training targets of the learned
 * closure from, fine runs.  Synchronous. */
acm_status acm_restrict(acm_handle *fine, acm_handle *coarse, int factor, double u_scale,
                        double rho_scale, float *out_dev, const float *scales3);

/* ---- learned closure ------------------------------------------------------
 * A small convolutional network that corrects a coarse-grid state after
 * solver steps: three periodic 3x3 convolutions, channels 3 -> 32 -> 32 -> 3,
 * ReLU after the first two; its output is added to the normalised state
 * (rho' s_rho, u s_u, v s_u).  BF16 weights and activations on the tensor
 * cores, FP32 accumulation, FP32 master weights trained with Adam.  This is
 * an addition to the method of the paper (a learned correction of the coarse
 * scheme); the plain scheme remains the reference its error is measured
 * against.
 *
 * Normalised state tensors are FP32 [batch][3][ny][nx] in device memory
 * (channel 0 = s_rho rho', 1 = s_u u, 2 = s_u v).  Weights are a flat FP32
 * vector: for each layer W[cout][cin][3][3] then b[cout]. */
typedef struct acm_closure acm_closure;

/* number of weights and biases (11011) */
size_t acm_closure_num_params(void);
/* grid nx x ny (both multiples of 16), BATCH states per call */
acm_status acm_closure_create(int nx, int ny, int batch, acm_closure **out);
/* later calls run on this stream (NULL: the legacy default stream, the
 * initial one); work already queued on the previous stream is ordered before
 * it on the device (an event, no host wait) */
acm_status acm_closure_set_stream(acm_closure *c, void *stream);
/* normalisation scales s_rho, s_u, s_u (s_u shared by u and v) */
acm_status acm_closure_set_scales(acm_closure *c, const float *scales3);
/* per-channel weights of the loss, default {1, 1, 1}; a channel of weight 0
 * is neither fitted nor corrected by acm_closure_apply (use {0, 1, 1} to
 * leave the density deviation, whose acoustic content differs between grids
 * of different lattice speed, to the scheme) */
acm_status acm_closure_set_loss_weights(acm_closure *c, const float *w3);
/* Training-input noise: acm_closure_loss_grad and acm_closure_train_step
 * add sigma * N(0, 1) (normalised units; counter-based normal variates from
 * SEED and the call count) to the channels of non-zero loss weight before the
 * forward pass, and fit x_noisy + net(x_noisy) to the target: the network
 * learns to pull perturbed states back toward the reference, which keeps
 * corrected free runs (whose inputs carry the closure's own past errors)
 * near the states it was trained on.  sigma = 0 (the default) turns it off.
 * Not part of the paper's method. */
acm_status acm_closure_set_input_noise(acm_closure *c, float sigma, uint64_t seed);
/* host FP32 weights in, resets the Adam state; or weights out */
acm_status acm_closure_set_weights(acm_closure *c, const float *w, size_t n);
acm_status acm_closure_get_weights(acm_closure *c, float *w, size_t n);
/* net(x) for normalised x -> net_dev (same layout), asynchronous */
acm_status acm_closure_forward(acm_closure *c, const float *x_dev, float *net_dev);
/* loss = mean((w_c (x + net(x) - target))^2) and its gradient (grad_host may be
 * NULL; n = acm_closure_num_params()); synchronous */
acm_status acm_closure_loss_grad(acm_closure *c, const float *x_dev, const float *target_dev,
                                 double *loss, float *grad_host);
/* one Adam step (beta 0.9/0.999, eps 1e-8) on that loss; *loss = the loss
 * before the step (loss may be NULL: then the step stays asynchronous) */
acm_status acm_closure_train_step(acm_closure *c, const float *x_dev, const float *target_dev,
                                  float lr, double *loss);
/* normalised state of runs 0..batch-1 of an FP32 2D handle -> x_dev */
acm_status acm_closure_gather(acm_closure *c, acm_handle *h, float *x_dev);
/* correct runs 0..batch-1 of the handle in place: state += net(state)/scale.
 * Waits for the handle's stream before and for the closure's stream after. */
acm_status acm_closure_apply(acm_closure *c, acm_handle *h);
acm_status acm_closure_destroy(acm_closure *c);
const char *acm_closure_last_error(const acm_closure *c);

/* ---- allocation-free diagnostics (the paper has no counterpart) ----------
 * The same FP64 diagnostics as acm_reduce_mass, computed from fields the
 * caller owns in device memory, for callers that cannot allocate device
 * memory where they need them: code whose device memory belongs entirely to
 * another runtime (a framework's caching allocator, a fixed pre-sized pool)
 * and loops with a hard latency budget that forbid allocation after start-up.
 * This call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.  Its scratch (the block partials of the reduction and a
 * run descriptor) lives in fixed file-scope device arrays inside libacm --
 * room for the partials of at most 4096 blocks (256 KiB) -- that every GPU
 * which loads the library holds until the process exits.
 *
 *   dim, nx, ny, nz  grid (nz = 1 in 2D); fields are contiguous [z][y][x],
 *                    x fastest, unpadded
 *   precision        ACM_FP64 (double arrays) or ACM_FP32_DEV (float arrays)
 *   rho0             reference density: the rho array holds rho - rho0 (the
 *                    deviation form the solver stores, which keeps the
 *                    O(Ma^2) density signal's digits in FP32); pass 0 for an
 *                    array of absolute density
 *   rho              density minus rho0 (device pointer)
 *   u, v, w          velocity (device pointers; w ignored in 2D)
 *   u_prev..w_prev   velocity before the last step for out[5], or all NULL
 *                    (then out[5] = 0)
 *   blocks           pass-1 blocks, 0 = default (min(ceil(n/256), 1024));
 *                    more than 4096 is rejected with ACM_EINVAL
 *   out_dev          DEVICE pointer to 8 doubles, same layout as one run of
 *                    acm_reduce_mass; written asynchronously on STREAM
 *   stream           cudaStream_t (NULL = legacy default stream)
 * The first call on a device resolves the device addresses of the scratch
 * arrays (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  Every call on a device shares the same
 * scratch and keeps the last call's contents: each call rewrites every
 * partial it later reads, so nothing needs clearing, but calls that overlap
 * on the GPU (different streams, no ordering between them) race on it and
 * must be serialised by the caller.  The call is asynchronous: it enqueues
 * three kernels on STREAM (the descriptor is written by a kernel from its
 * launch argument) and does not wait for the stream; errors found on the
 * host return before anything is enqueued.  Message of the last
 * failure on the calling thread: acm_noalloc_last_error(). */
acm_status acm_reduce_mass_noalloc(int dim, int nx, int ny, int nz, int precision, double rho0,
                                   const void *rho, const void *u, const void *v, const void *w,
                                   const void *u_prev, const void *v_prev, const void *w_prev,
                                   int blocks, double *out_dev, void *stream);
const char *acm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ACM_H */
