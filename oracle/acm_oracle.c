/*
 * acm_oracle.c -- plain FP64 CPU oracle for the simplified MAME scheme
 * (Huang, arXiv:2012.03525).  TEST INFRASTRUCTURE ONLY: nothing on the
 * product path may link, load or call this file; only the tests, the
 * smoke check and the benchmark's CPU-baseline leg use it.
 *
 * It is written to be read against the paper, not to be fast:
 *   - single thread, separate arrays for time levels n and n+1,
 *   - rho^{n+1} is computed for EVERY node before any momentum update
 *     (Section 2, the remark after Eq. 2.13: the step is fully explicit),
 *   - absolute density rho and momentum rho*u_alpha, exactly as in
 *     Eqs. (2.10)-(2.11), velocity recovered by one IEEE division,
 *   - build with -O2 -ffp-contract=off so no fused multiply-adds appear.
 *
 * Units: delta_x = 1, delta_t = p->dt, lattice speed c = 1/dt and
 * c_s^2 = c^2/3 (Section 2, text after Eq. 2.1).
 *
 * Readings of points the paper leaves open (the full list is kept with the
 * design notes):
 *   - advection flux d_beta(rho u_alpha u_beta) = centred difference of the
 *     nodal product (Eq. 2.12 applied to the product),
 *   - viscous term nu * Laplacian(rho u_alpha) as printed in Eq. (2.11),
 *   - walls: wall nodes sit on the first/last grid index; their velocity is
 *     Dirichlet and their density is the second-order zero-normal-gradient
 *     extrapolation (4 rho_1 - rho_2)/3, applied to rho^{n+1} before the
 *     momentum update so that d_alpha rho^{n+1} next to a wall uses it;
 *     corner/edge nodes shared by a stationary wall and a lid are stationary,
 *   - two-phase walls: ghost nodes mirror the first interior node (zero normal
 *     derivative of mu) plus the wetting correction for phi (Section 2);
 *   - two-phase: "second order isotropic" operators are the lattice-weighted
 *     D2Q9 (2D) / D3Q19 (3D) gradient and Laplacian; the Cahn-Hilliard
 *     equation (Eq. 2.14) is advanced by Heun's two-stage RK2 with u^n frozen;
 *     F_ST = -phi^n grad mu^n enters the momentum update (Section 2, the
 *     two-phase paragraph), mu = 4 a phi (phi^2-1) - kappa Lap(phi),
 *     a = 3 sigma/(4W), kappa = 3 sigma W/8.
 *   - the MAMEs predictor-corrector (Eqs. 2.6-2.9, oracle_step_mames), kept
 *     as the comparison scheme: centred first differences, compact second
 *     differences for d_aa, the centred four-point mixed difference for
 *     d_ab (a != b), periodic grids only.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PERIODIC 0
#define OR_WALL 1
#define OR_LID 2
#define OR_SYMMETRY 4

typedef struct {
    int dim, nx, ny, nz;   /* nodes per direction; nz = 1 in 2D */
    double dt;             /* delta_t in lattice units (delta_x = 1) */
    double nu;             /* kinematic viscosity */
    double rho0;           /* reference density (two-phase: physical density) */
    int bc[6];             /* faces -x,+x,-y,+y,-z,+z: 0 periodic, 1 wall, 2 lid,
                              4 symmetry (mirror) plane */
    double lid_u[3];       /* velocity of faces marked as lid */
    double g[3];           /* body force per unit mass */
    int two_phase;         /* 0 or 1 */
    double sigma, W, M;    /* surface tension, interface width, mobility */
    int sat_mask;          /* bit0: continuity SAT, bit1: momentum SAT */
    double theta_deg;      /* contact angle of wall faces (two-phase) */
    double rho_ratio;      /* two-phase: 0 = body force on both phases; r > 0 =
                              Boussinesq drop force (Section 3.5) */
} oracle_params;

typedef struct {
    const oracle_params *p;
    int n[3];
    int periodic[3];
    int mirror[3];  /* both faces of the axis are symmetry planes */
} grid_t;

/* Symmetry (mirror) planes (the quarter domains of Sections 3.6-3.7): the
   plane passes through the first/last node of the axis, which stay unknowns
   of the scheme; a node one beyond the plane is the mirror image of the node
   one inside, c(-1) = c(1), c(n) = c(n-2).  Scalars (rho, phi, mu) and the
   tangential velocity are even across the plane, the normal velocity (and
   momentum) component is odd: its image changes sign, and it is zero on the
   plane. */
static inline int wrap(int c, int n, int periodic, int mirror)
{
    if (periodic) {
        if (c < 0) return c + n;
        if (c >= n) return c - n;
    }
    if (mirror) {
        if (c < 0) return -c;
        if (c >= n) return 2 * (n - 1) - c;
    }
    return c;
}

/* linear index of node (i,j,k); periodic directions wrap (stencils reach at
   most one node past an edge); wall directions are only ever asked for
   indices inside the grid (interior stencils reach at most the wall) */
static inline long gidx(const grid_t *G, int i, int j, int k)
{
    i = wrap(i, G->n[0], G->periodic[0], G->mirror[0]);
    j = wrap(j, G->n[1], G->periodic[1], G->mirror[1]);
    k = wrap(k, G->n[2], G->periodic[2], G->mirror[2]);
    return ((long)k * G->n[1] + j) * G->n[0] + i;
}

/* a node is a wall node if it lies on a wall or lid face (not on a periodic
   or a symmetry face) */
static int on_wall(const grid_t *G, int i, int j, int k)
{
    int c[3] = {i, j, k};
    for (int d = 0; d < G->p->dim; ++d)
        if (!G->periodic[d] && !G->mirror[d] && (c[d] == 0 || c[d] == G->n[d] - 1)) return 1;
    return 0;
}

/* linear index of a node and of its +/- neighbours along each axis, and
   whether that neighbour is a mirror image (beyond a symmetry plane) */
typedef struct { long c, p[3], m[3]; int rp[3], rm[3]; } nbr_t;

static nbr_t neighbours(const grid_t *G, int i, int j, int k)
{
    nbr_t nb;
    int cc[3] = {i, j, k};
    nb.c = gidx(G, i, j, k);
    for (int d = 0; d < 3; ++d) {
        int e[3] = {0, 0, 0};
        e[d] = 1;
        nb.p[d] = (d < G->p->dim) ? gidx(G, i + e[0], j + e[1], k + e[2]) : nb.c;
        nb.m[d] = (d < G->p->dim) ? gidx(G, i - e[0], j - e[1], k - e[2]) : nb.c;
        nb.rp[d] = d < G->p->dim && G->mirror[d] && cc[d] + 1 >= G->n[d];
        nb.rm[d] = d < G->p->dim && G->mirror[d] && cc[d] - 1 < 0;
    }
    return nb;
}

/* value at the + (plus = 1) or - neighbour along d of component field f;
   odd = the axis whose component f is (-1 for a scalar): across a symmetry
   plane normal to that axis the image changes sign */
static double nbv(const double *f, const nbr_t *nb, int d, int plus, int odd)
{
    double v = f[plus ? nb->p[d] : nb->m[d]];
    int refl = plus ? nb->rp[d] : nb->rm[d];
    return (refl && d == odd) ? -v : v;
}

/* centred first difference, Eq. (2.12), delta_x = 1, of a scalar field */
static double dcen(const double *f, const nbr_t *nb, int d)
{
    return (f[nb->p[d]] - f[nb->m[d]]) / 2.0;
}

/* the same for component `odd` of a vector field */
static double dcen_c(const double *f, const nbr_t *nb, int d, int odd)
{
    return (nbv(f, nb, d, 1, odd) - nbv(f, nb, d, 0, odd)) / 2.0;
}

/* 5-point (2D) / 7-point (3D) Laplacian, Eq. (2.13) and its 3D extension;
   odd: as for nbv (-1 for a scalar) */
static double lap(const grid_t *G, const double *f, const nbr_t *nb, int odd)
{
    double s = 0.0;
    for (int d = 0; d < G->p->dim; ++d) s += nbv(f, nb, d, 1, odd) + nbv(f, nb, d, 0, odd);
    return s - 2.0 * G->p->dim * f[nb->c];
}

/* ---- lattice-weighted isotropic operators for the two-phase part ---- */
typedef struct { int e[3]; double w; } vel_t;
static const vel_t D2Q9[9] = {
    {{0, 0, 0}, 4.0 / 9.0},
    {{1, 0, 0}, 1.0 / 9.0}, {{-1, 0, 0}, 1.0 / 9.0},
    {{0, 1, 0}, 1.0 / 9.0}, {{0, -1, 0}, 1.0 / 9.0},
    {{1, 1, 0}, 1.0 / 36.0}, {{-1, 1, 0}, 1.0 / 36.0},
    {{1, -1, 0}, 1.0 / 36.0}, {{-1, -1, 0}, 1.0 / 36.0}};
static const vel_t D3Q19[19] = {
    {{0, 0, 0}, 1.0 / 3.0},
    {{1, 0, 0}, 1.0 / 18.0}, {{-1, 0, 0}, 1.0 / 18.0},
    {{0, 1, 0}, 1.0 / 18.0}, {{0, -1, 0}, 1.0 / 18.0},
    {{0, 0, 1}, 1.0 / 18.0}, {{0, 0, -1}, 1.0 / 18.0},
    {{1, 1, 0}, 1.0 / 36.0}, {{-1, 1, 0}, 1.0 / 36.0},
    {{1, -1, 0}, 1.0 / 36.0}, {{-1, -1, 0}, 1.0 / 36.0},
    {{1, 0, 1}, 1.0 / 36.0}, {{-1, 0, 1}, 1.0 / 36.0},
    {{1, 0, -1}, 1.0 / 36.0}, {{-1, 0, -1}, 1.0 / 36.0},
    {{0, 1, 1}, 1.0 / 36.0}, {{0, -1, 1}, 1.0 / 36.0},
    {{0, 1, -1}, 1.0 / 36.0}, {{0, -1, -1}, 1.0 / 36.0}};
#define CS2_LAT (1.0 / 3.0) /* lattice sound speed squared of the weights */

static const vel_t *vset(const grid_t *G, int *q)
{
    if (G->p->dim == 2) { *q = 9; return D2Q9; }
    *q = 19;
    return D3Q19;
}

/* Value of a two-phase field at node (i,j,k), where a coordinate may lie one
   node beyond a wall face.  Wall faces carry the boundary conditions of the
   two-phase paragraph of Section 2: the ghost node beyond a wall mirrors the
   node one inside, f(-1) = f(1) (zero normal derivative, used for mu), and
   for the order parameter the wetting condition d_n phi = -(2/W) cos(theta)
   (1 - phi_w^2), with n the wall normal pointing into the fluid and the
   centred difference d_n phi = (phi(1) - phi(-1)) / 2, gives
   phi(-1) = phi(1) + 2 (2/W) cos(theta) (1 - phi_w^2). */
enum { F_MIRROR = 0, F_WETTING = 1 };

static double field_at(const grid_t *G, const double *f, int kind, int i, int j, int k)
{
    /* images across symmetry planes first (scalar fields: even), so that a
       ghost beyond a wall and a mirror plane takes its image's wall term */
    for (int d = 0; d < G->p->dim; ++d)
        if (G->mirror[d]) {
            int *cd = d == 0 ? &i : (d == 1 ? &j : &k);
            *cd = wrap(*cd, G->n[d], 0, 1);
        }
    int c[3] = {i, j, k};
    double add = 0.0;
    for (int d = 0; d < G->p->dim; ++d) {
        if (G->periodic[d] || G->mirror[d]) continue;
        int mirror;
        if (c[d] == -1) mirror = 1;
        else if (c[d] == G->n[d]) mirror = G->n[d] - 2;
        else continue;
        if (kind == F_WETTING) {
            /* phi_w: the boundary node nearest the ghost node (the ghost's
               own coordinates clamped into the box in every walled
               direction), so that at an edge or corner every wall's term
               takes the same edge/corner node */
            int cw[3] = {i, j, k};
            for (int e = 0; e < G->p->dim; ++e)
                if (!G->periodic[e] && !G->mirror[e])
                    cw[e] = cw[e] < 0 ? 0 : (cw[e] >= G->n[e] ? G->n[e] - 1 : cw[e]);
            double pw = f[gidx(G, cw[0], cw[1], cw[2])];
            double ct = cos(G->p->theta_deg * 3.14159265358979323846 / 180.0);
            add += 2.0 * (2.0 / G->p->W) * ct * (1.0 - pw * pw);
        }
        c[d] = mirror;
    }
    return f[gidx(G, c[0], c[1], c[2])] + add;
}

/* G_iso,d f = (1/c_sL^2) sum_i w_i e_id f(x + e_i) */
static double grad_iso(const grid_t *G, const double *f, int kind, int i, int j, int k, int d)
{
    int q;
    const vel_t *V = vset(G, &q);
    double s = 0.0;
    for (int a = 0; a < q; ++a) {
        if (V[a].e[d] == 0) continue;
        s += V[a].w * V[a].e[d] *
             field_at(G, f, kind, i + V[a].e[0], j + V[a].e[1], k + V[a].e[2]);
    }
    return s / CS2_LAT;
}

/* L_iso f = (2/c_sL^2) sum_i w_i (f(x + e_i) - f(x)) */
static double lap_iso(const grid_t *G, const double *f, int kind, int i, int j, int k)
{
    int q;
    const vel_t *V = vset(G, &q);
    double f0 = f[gidx(G, i, j, k)];
    double s = 0.0;
    for (int a = 1; a < q; ++a)
        s += V[a].w * (field_at(G, f, kind, i + V[a].e[0], j + V[a].e[1], k + V[a].e[2]) - f0);
    return 2.0 * s / CS2_LAT;
}

/* chemical potential, Section 2 two-phase paragraph:
   mu = 4 a phi (phi^2 - 1) - kappa Lap_iso(phi) */
static void chem_pot(const grid_t *G, const double *phi, double *mu)
{
    const oracle_params *p = G->p;
    double a = 3.0 * p->sigma / (4.0 * p->W);
    double kappa = 3.0 * p->sigma * p->W / 8.0;
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                long c = gidx(G, i, j, k);
                double f = phi[c];
                mu[c] = 4.0 * a * f * (f * f - 1.0) - kappa * lap_iso(G, phi, F_WETTING, i, j, k);
            }
}

/* right-hand side of the Cahn-Hilliard equation (Eq. 2.14):
   R = -u_alpha G_iso,alpha(phi) + M Lap_iso(mu) */
static void che_rhs(const grid_t *G, const double *phi, const double *mu,
                    const double *const *uvw, double *R)
{
    const oracle_params *p = G->p;
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                long c = gidx(G, i, j, k);
                double adv = 0.0;
                for (int d = 0; d < p->dim; ++d)
                    adv += uvw[d][c] * grad_iso(G, phi, F_WETTING, i, j, k, d);
                R[c] = -adv + p->M * lap_iso(G, mu, F_MIRROR, i, j, k);
            }
}

static int setup_grid(const oracle_params *p, grid_t *G)
{
    if (p->dim != 2 && p->dim != 3) return -1;
    G->p = p;
    G->n[0] = p->nx;
    G->n[1] = p->ny;
    G->n[2] = (p->dim == 3) ? p->nz : 1;
    for (int d = 0; d < 3; ++d) {
        G->mirror[d] = 0;
        if (d >= p->dim) { G->periodic[d] = 1; continue; }
        int lo = p->bc[2 * d], hi = p->bc[2 * d + 1];
        if ((lo == OR_PERIODIC) != (hi == OR_PERIODIC)) return -1;
        if ((lo == OR_SYMMETRY) != (hi == OR_SYMMETRY)) return -1;
        G->periodic[d] = (lo == OR_PERIODIC);
        G->mirror[d] = (lo == OR_SYMMETRY);
        if (G->n[d] < (G->periodic[d] ? 1 : 3)) return -1;
    }
    return 0;
}

/* One time step of Eqs. (2.10)-(2.11) (+ body force, + surface tension and
   the Cahn-Hilliard update when two_phase).  Arrays are [z][y][x], x fastest.
   Returns 0 on success, -1 on invalid parameters, -2 on allocation failure. */
int oracle_step(const oracle_params *p, double *rho, double *u, double *v,
                double *w, double *phi, long nsteps)
{
    grid_t G;
    if (setup_grid(p, &G) != 0) return -1;
    const int dim = p->dim;
    const long N = (long)G.n[0] * G.n[1] * G.n[2];
    const double dt = p->dt;
    const double c = 1.0 / dt;
    const double cs2 = c * c / 3.0;
    const int sat_c = p->sat_mask & 1;
    const int sat_m = (p->sat_mask >> 1) & 1;

    double *vel[3] = {u, v, w};
    double *m[3], *rho1, *mnew[3], *mu = NULL, *mus = NULL, *phis = NULL, *R = NULL;
    int ok = 1;
    rho1 = malloc(sizeof(double) * N);
    ok &= rho1 != NULL;
    for (int d = 0; d < 3; ++d) {
        m[d] = malloc(sizeof(double) * N);
        mnew[d] = malloc(sizeof(double) * N);
        ok &= m[d] != NULL && mnew[d] != NULL;
    }
    if (p->two_phase) {
        mu = malloc(sizeof(double) * N);
        mus = malloc(sizeof(double) * N);
        phis = malloc(sizeof(double) * N);
        R = malloc(sizeof(double) * N);
        ok &= mu && mus && phis && R;
    }
    if (!ok) {
        free(rho1);
        for (int d = 0; d < 3; ++d) { free(m[d]); free(mnew[d]); }
        free(mu); free(mus); free(phis); free(R);
        return -2;
    }

    for (long step = 0; step < nsteps; ++step) {
        /* momentum rho u_alpha at time n */
        for (int d = 0; d < dim; ++d)
            for (long c0 = 0; c0 < N; ++c0) m[d][c0] = rho[c0] * vel[d][c0];

        if (p->two_phase) chem_pot(&G, phi, mu);

        /* ---- continuity, Eq. (2.10), every non-wall node ---- */
        for (long c0 = 0; c0 < N; ++c0) rho1[c0] = rho[c0];
        for (int k = 0; k < G.n[2]; ++k)
            for (int j = 0; j < G.n[1]; ++j)
                for (int i = 0; i < G.n[0]; ++i) {
                    if (on_wall(&G, i, j, k)) continue;
                    nbr_t nb = neighbours(&G, i, j, k);
                    long c0 = nb.c;
                    double div = 0.0;
                    for (int d = 0; d < dim; ++d) div += dcen_c(m[d], &nb, d, d);
                    double r = rho[c0] - dt * div;
                    if (sat_c) r += 0.5 * cs2 * dt * dt * lap(&G, rho, &nb, -1);
                    rho1[c0] = r;
                }
        /* wall density: second-order zero normal gradient, face by face */
        for (int d = 0; d < dim; ++d) {
            if (G.periodic[d] || G.mirror[d]) continue;
            for (int k = 0; k < G.n[2]; ++k)
                for (int j = 0; j < G.n[1]; ++j)
                    for (int i = 0; i < G.n[0]; ++i) {
                        int cc[3] = {i, j, k};
                        int s;
                        if (cc[d] == 0) s = 1;
                        else if (cc[d] == G.n[d] - 1) s = -1;
                        else continue;
                        int c1[3] = {i, j, k}, c2[3] = {i, j, k};
                        c1[d] += s;
                        c2[d] += 2 * s;
                        rho1[gidx(&G, i, j, k)] =
                            (4.0 * rho1[gidx(&G, c1[0], c1[1], c1[2])] -
                             rho1[gidx(&G, c2[0], c2[1], c2[2])]) / 3.0;
                    }
        }

        /* ---- momentum, Eq. (2.11) (+ dt rho^{n+1} g, + dt F_ST) ---- */
        for (int k = 0; k < G.n[2]; ++k)
            for (int j = 0; j < G.n[1]; ++j)
                for (int i = 0; i < G.n[0]; ++i) {
                    nbr_t nb = neighbours(&G, i, j, k);
                    long c0 = nb.c;
                    if (on_wall(&G, i, j, k)) {
                        for (int d = 0; d < dim; ++d) mnew[d][c0] = 0.0;
                        continue;
                    }
                    for (int a = 0; a < dim; ++a) {
                        /* flux d_beta(rho u_a u_beta + rho cs2 delta_ab) */
                        double flux = 0.0;
                        for (int b = 0; b < dim; ++b)
                            flux += (nbv(m[a], &nb, b, 1, a) * nbv(vel[b], &nb, b, 1, b) -
                                     nbv(m[a], &nb, b, 0, a) * nbv(vel[b], &nb, b, 0, b)) / 2.0;
                        flux += cs2 * dcen(rho, &nb, a);
                        double mn = m[a][c0] - dt * flux + p->nu * dt * lap(&G, m[a], &nb, a);
                        if (sat_m)
                            mn -= (p->nu + 0.5 * cs2 * dt) *
                                  (dcen(rho1, &nb, a) - dcen(rho, &nb, a));
                        /* body force; with the Boussinesq approximation of
                           Section 3.5 it acts on the drop only, times
                           (rho_L - rho_G) / ((rho_L + rho_G)/2) =
                           2 (r - 1)/(r + 1), the drop's share of a node
                           being its volume fraction (1 + phi)/2 */
                        double ga = p->g[a];
                        if (p->two_phase && p->rho_ratio > 0.0)
                            ga *= 2.0 * (p->rho_ratio - 1.0) / (p->rho_ratio + 1.0) *
                                  (0.5 * (1.0 + phi[c0]));
                        mn += dt * rho1[c0] * ga;
                        if (p->two_phase)
                            mn += dt * (-phi[c0] * grad_iso(&G, mu, F_MIRROR, i, j, k, a));
                        mnew[a][c0] = mn;
                    }
                }

        /* ---- Cahn-Hilliard, Eq. (2.14), Heun RK2 with u^n frozen ---- */
        if (p->two_phase) {
            const double *uvw[3] = {u, v, w};
            che_rhs(&G, phi, mu, uvw, R);
            for (long c0 = 0; c0 < N; ++c0) phis[c0] = phi[c0] + dt * R[c0];
            chem_pot(&G, phis, mus);
            double *R2 = mu; /* mu^n no longer needed */
            che_rhs(&G, phis, mus, uvw, R2);
            for (long c0 = 0; c0 < N; ++c0)
                phi[c0] = 0.5 * (phi[c0] + phis[c0] + dt * R2[c0]);
        }

        /* ---- new state: u = (rho u)^{n+1} / rho^{n+1}, wall velocities ---- */
        for (int k = 0; k < G.n[2]; ++k)
            for (int j = 0; j < G.n[1]; ++j)
                for (int i = 0; i < G.n[0]; ++i) {
                    long c0 = gidx(&G, i, j, k);
                    rho[c0] = rho1[c0];
                    if (!on_wall(&G, i, j, k)) {
                        int cc[3] = {i, j, k};
                        for (int d = 0; d < dim; ++d)
                            vel[d][c0] = (G.mirror[d] && (cc[d] == 0 || cc[d] == G.n[d] - 1))
                                             ? 0.0 /* normal velocity on a symmetry plane */
                                             : mnew[d][c0] / rho1[c0];
                        continue;
                    }
                    /* a node on any stationary wall is at rest; otherwise it
                       is on a lid face and moves with the lid */
                    int cc[3] = {i, j, k}, stationary = 0;
                    for (int d = 0; d < dim; ++d) {
                        if (G.periodic[d] || G.mirror[d]) continue;
                        if (cc[d] == 0 && p->bc[2 * d] == OR_WALL) stationary = 1;
                        if (cc[d] == G.n[d] - 1 && p->bc[2 * d + 1] == OR_WALL) stationary = 1;
                    }
                    for (int d = 0; d < dim; ++d) vel[d][c0] = stationary ? 0.0 : p->lid_u[d];
                }
    }

    free(rho1);
    for (int d = 0; d < 3; ++d) { free(m[d]); free(mnew[d]); }
    free(mu); free(mus); free(phis); free(R);
    return 0;
}

/* ---- MAMEs predictor-corrector (Section 2, Eqs. 2.6-2.9): the scheme the
   simplified one-step update replaces, kept as a comparison scheme ----

   Spatial operators (the paper does not print them for this scheme; these
   are the second-order centred forms on the same grid):
     D_a f      centred first difference (Eq. 2.12),
     D_aa f     compact second difference f(+a) - 2 f + f(-a),
     D_ab f     (a != b) centred mixed difference
                (f(+a+b) - f(+a-b) - f(-a+b) + f(-a-b)) / 4,
     L f        sum_a D_aa f (Eq. 2.13).
   Pi_ab = rho u_a u_b + p delta_ab with p = c_s^2 rho.  Periodic grids only. */
static double dmix(const grid_t *G, const double *f, int i, int j, int k, int a, int b)
{
    int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
    ea[a] = 1;
    eb[b] = 1;
    if (a == b)
        return f[gidx(G, i + ea[0], j + ea[1], k + ea[2])] - 2.0 * f[gidx(G, i, j, k)] +
               f[gidx(G, i - ea[0], j - ea[1], k - ea[2])];
    double pp = f[gidx(G, i + ea[0] + eb[0], j + ea[1] + eb[1], k + ea[2] + eb[2])];
    double pm = f[gidx(G, i + ea[0] - eb[0], j + ea[1] - eb[1], k + ea[2] - eb[2])];
    double mp = f[gidx(G, i - ea[0] + eb[0], j - ea[1] + eb[1], k - ea[2] + eb[2])];
    double mm = f[gidx(G, i - ea[0] - eb[0], j - ea[1] - eb[1], k - ea[2] - eb[2])];
    return (pp - pm - mp + mm) / 4.0;
}

/* Pi_ab of a state (rho, m) at every node; P[a*3+b] */
static void momentum_flux(const grid_t *G, const double *rho, double *const *m, double cs2,
                          double **P)
{
    const int dim = G->p->dim;
    const long N = (long)G->n[0] * G->n[1] * G->n[2];
    for (long c = 0; c < N; ++c)
        for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b)
                P[a * 3 + b][c] = m[a][c] * (m[b][c] / rho[c]) + (a == b ? cs2 * rho[c] : 0.0);
}

/* sum_b D_b Pi_ab at node (i,j,k) */
static double div_flux(const grid_t *G, double **P, const nbr_t *nb, int a)
{
    double s = 0.0;
    for (int b = 0; b < G->p->dim; ++b) s += dcen(P[a * 3 + b], nb, b);
    return s;
}

int oracle_step_mames(const oracle_params *p, double *rho, double *u, double *v, double *w,
                      long nsteps)
{
    grid_t G;
    if (setup_grid(p, &G) != 0) return -1;
    for (int d = 0; d < p->dim; ++d)
        if (!G.periodic[d]) return -1;
    if (p->two_phase) return -1;
    const int dim = p->dim;
    const long N = (long)G.n[0] * G.n[1] * G.n[2];
    const double dt = p->dt, nu = p->nu;
    const double cs2 = (1.0 / dt) * (1.0 / dt) / 3.0;
    double *vel[3] = {u, v, w};
    double *m[3] = {0}, *ms[3] = {0}, *P[9] = {0}, *Ps[9] = {0}, *rhos;
    int ok = (rhos = malloc(sizeof(double) * N)) != NULL;
    for (int a = 0; a < 3; ++a) {
        ok &= (m[a] = malloc(sizeof(double) * N)) != NULL;
        ok &= (ms[a] = malloc(sizeof(double) * N)) != NULL;
    }
    for (int q = 0; q < 9; ++q) {
        ok &= (P[q] = malloc(sizeof(double) * N)) != NULL;
        ok &= (Ps[q] = malloc(sizeof(double) * N)) != NULL;
    }
    if (ok) {
        for (long step = 0; step < nsteps; ++step) {
            for (long c = 0; c < N; ++c)
                for (int a = 0; a < dim; ++a) m[a][c] = rho[c] * vel[a][c];
            momentum_flux(&G, rho, m, cs2, P);
            /* predictor, Eqs. (2.6) and (2.7) */
            for (int k = 0; k < G.n[2]; ++k)
                for (int j = 0; j < G.n[1]; ++j)
                    for (int i = 0; i < G.n[0]; ++i) {
                        nbr_t nb = neighbours(&G, i, j, k);
                        double div_m = 0.0, ddPi = 0.0;
                        for (int a = 0; a < dim; ++a) {
                            div_m += dcen(m[a], &nb, a);
                            for (int b = 0; b < dim; ++b) ddPi += dmix(&G, P[a * 3 + b], i, j, k, a, b);
                        }
                        rhos[nb.c] = rho[nb.c] - dt * div_m + 0.5 * dt * dt * ddPi;
                        for (int a = 0; a < dim; ++a) {
                            double grad_div = 0.0;
                            for (int g = 0; g < dim; ++g) grad_div += dmix(&G, m[g], i, j, k, a, g);
                            ms[a][nb.c] = m[a][nb.c] - dt * div_flux(&G, P, &nb, a) +
                                          nu * dt * lap(&G, m[a], &nb, a) + 2.0 * nu * dt * grad_div;
                        }
                    }
            /* corrector, Eqs. (2.8) and (2.9) */
            momentum_flux(&G, rhos, ms, cs2, Ps);
            const double cc = nu / cs2 - 0.5 * dt;
            for (int k = 0; k < G.n[2]; ++k)
                for (int j = 0; j < G.n[1]; ++j)
                    for (int i = 0; i < G.n[0]; ++i) {
                        nbr_t nb = neighbours(&G, i, j, k);
                        for (int a = 0; a < dim; ++a) {
                            double mn = ms[a][nb.c] +
                                        cc * (div_flux(&G, Ps, &nb, a) - div_flux(&G, P, &nb, a));
                            vel[a][nb.c] = mn / rhos[nb.c];
                        }
                    }
            memcpy(rho, rhos, sizeof(double) * N);
        }
    }
    free(rhos);
    for (int a = 0; a < 3; ++a) { free(m[a]); free(ms[a]); }
    for (int q = 0; q < 9; ++q) { free(P[q]); free(Ps[q]); }
    return ok ? 0 : -2;
}

/* Chemical potential field of phi (exposed for the equilibrium pins). */
int oracle_chem_pot(const oracle_params *p, const double *phi, double *mu)
{
    grid_t G;
    if (setup_grid(p, &G) != 0) return -1;
    chem_pot(&G, phi, mu);
    return 0;
}

/* Isotropic gradient (component d) and Laplacian of a field. */
int oracle_grad_lap_iso(const oracle_params *p, const double *f, int d,
                        double *grad, double *lapl)
{
    grid_t G;
    if (setup_grid(p, &G) != 0) return -1;
    for (int k = 0; k < G.n[2]; ++k)
        for (int j = 0; j < G.n[1]; ++j)
            for (int i = 0; i < G.n[0]; ++i) {
                long c = gidx(&G, i, j, k);
                if (grad) grad[c] = grad_iso(&G, f, F_MIRROR, i, j, k, d);
                if (lapl) lapl[c] = lap_iso(&G, f, F_MIRROR, i, j, k);
            }
    return 0;
}

/* Integral diagnostics (Section 3: kinetic energy of the Taylor-Green test,
   steady-state criterion of the cavity test), summed in index order:
   out[0] = sum rho, out[1..3] = sum rho u_alpha, out[4] = 1/2 sum |u|^2,
   out[5] = max | |u| - |u_prev| | (0 if u_prev is NULL), out[6] = max |u|,
   out[7] = number of non-finite values among rho, u, v, w. */
int oracle_reduce(const oracle_params *p, const double *rho, const double *u,
                  const double *v, const double *w, const double *up,
                  const double *vp, const double *wp, double out[8])
{
    grid_t G;
    if (setup_grid(p, &G) != 0) return -1;
    const long N = (long)G.n[0] * G.n[1] * G.n[2];
    const double *vel[3] = {u, v, w};
    const double *velp[3] = {up, vp, wp};
    for (int q = 0; q < 8; ++q) out[q] = 0.0;
    for (long c = 0; c < N; ++c) {
        double s2 = 0.0, sp2 = 0.0;
        out[0] += rho[c];
        int bad = !isfinite(rho[c]);
        for (int d = 0; d < p->dim; ++d) {
            out[1 + d] += rho[c] * vel[d][c];
            s2 += vel[d][c] * vel[d][c];
            bad |= !isfinite(vel[d][c]);
            if (up) sp2 += velp[d][c] * velp[d][c];
        }
        out[4] += 0.5 * s2;
        if (up) {
            double dm = fabs(sqrt(s2) - sqrt(sp2));
            if (dm > out[5]) out[5] = dm;
        }
        if (sqrt(s2) > out[6]) out[6] = sqrt(s2);
        out[7] += bad;
    }
    return 0;
}
