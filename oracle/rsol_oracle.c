/*
 * FP64 oracle for the reduced-speed-of-light (RSOL) MHD-PIC cosmic-ray step
 * of Ji & Hopkins, "A Reduced-Speed-of-Light Formulation of the
 * Magnetohydrodynamic-Particle-in-Cell Method" (arXiv:2111.14704).
 *
 * TEST INFRASTRUCTURE.  This file is a plain, slow, obviously-checkable
 * restatement of what the GPU library computes.  Only the test-suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or helper with the CUDA library, and the CUDA
 * library never calls it.  Build: gcc -O2 -ffp-contract=off (no FMA
 * contraction, so every product is rounded as written).
 *
 * What it follows, step by step (all in double precision):
 *
 *   packet ansatz (Sec. 2): f = sum_j N_j W(x - <x>_j) delta(p - <p>_j);
 *     here W is the CIC (linear) or TSC (quadratic) B-spline on a periodic
 *     grid with nodes at integer coordinates.  The same W gathers E, B to a
 *     packet and scatters its moments back.
 *   Eq. momentum.alt (Sec. 2): d(gamma beta)/dt = (c~/c) (q/(m c)) [E + beta x B],
 *     integrated by the Boris kick-rotate-kick (the paper gives no integrator;
 *     this is the textbook Boris scheme), u = gamma beta at half steps.
 *   effective velocity (Sec. 2): d<x>/dt = v_eff = c~ beta.
 *   back-reaction (Sec. 2, force on the gas): -sum_j n_j q_j [E + beta_j x B]
 *     = -sum_j n_j (c/c~) d<p>_j/dt; the energy source is the same (c/c~) rule
 *     applied to the packet energy E_j = N_j gamma m c^2.
 *   packet totals (Sec. 2): N_j, M_j = N_j m, E_j = N_j gamma m c^2,
 *     P_j = N_j gamma beta m c.
 *
 * Parity pins: every exported function here is checked in tests/ against
 * closed forms (discrete gyro-orbit, E x B drift, |u| conservation, pure-E
 * kick), the textbook B-spline definitions by brute force, partition of unity,
 * the (c/c~) momentum-exchange identity, c~-independence in static fields,
 * and numpy's stable argsort.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz; /* periodic grid: nodes (= cells) per axis */
    int32_t shape;      /* 1 = CIC, 2 = TSC */
    double dx;          /* cell size */
    double c;           /* true speed of light */
    double c_tilde;     /* reduced speed of light */
    double q_over_m;    /* q / m of the species */
    double q;           /* charge of one CR (m = q / q_over_m) */
    double dt;          /* timestep */
} orc_params;

typedef struct {
    int64_t n;
    int32_t *ix, *iy, *iz;      /* cell per axis, 0 <= i < n_axis */
    double *ox, *oy, *oz;       /* offset in the cell, [0, 1) */
    double *ux, *uy, *uz;       /* u = gamma beta (at the half step) */
    double *w;                  /* N_j, packet weight */
} orc_particles;

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/*
 * One-axis factors of the shape function W for a packet at x = i + f,
 * f in [0, 1).  Returns the node offset (relative to i) of w[0]; the nodes are
 * i + off, i + off + 1, (i + off + 2 for TSC).
 *   CIC: linear B-spline, nodes i, i+1 with weights 1 - f, f.
 *   TSC: quadratic B-spline around the nearest node j (j = i if f < 1/2,
 *        else i + 1; f = 1/2 goes to i + 1), d = x - j in [-1/2, 1/2):
 *        W(j-1) = (1/2 - d)^2 / 2, W(j) = 3/4 - d^2, W(j+1) = (1/2 + d)^2 / 2.
 */
int orc_weights_1d(int shape, double f, double w[3])
{
    if (shape == 1) {
        w[0] = 1.0 - f;
        w[1] = f;
        w[2] = 0.0;
        return 0;
    }
    int off;
    double d;
    if (f < 0.5) {
        d = f;
        off = -1;
    } else {
        d = f - 1.0;
        off = 0;
    }
    w[0] = 0.5 * (0.5 - d) * (0.5 - d);
    w[1] = 0.75 - d * d;
    w[2] = 0.5 * (0.5 + d) * (0.5 + d);
    return off;
}

static int npts(int shape) { return shape == 1 ? 2 : 3; }

/*
 * Gather: E(x_j), B(x_j) = sum over nodes W(x_j - x_node) {E, B}(node).
 * F holds 6 planes [Ex, Ey, Ez, Bx, By, Bz], each nz*ny*nx, x fastest.
 */
void orc_gather(const orc_params *p, const double *F, int ix, int iy, int iz,
                double fx, double fy, double fz, double E[3], double B[3])
{
    double wx[3], wy[3], wz[3];
    int ox = orc_weights_1d(p->shape, fx, wx);
    int oy = orc_weights_1d(p->shape, fy, wy);
    int oz = orc_weights_1d(p->shape, fz, wz);
    int64_t ncell = (int64_t)p->nx * p->ny * p->nz;
    int np_ = npts(p->shape);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int c = 0; c < np_; ++c) {
        int kz = wrap(iz + oz + c, p->nz);
        for (int b = 0; b < np_; ++b) {
            int ky = wrap(iy + oy + b, p->ny);
            for (int a = 0; a < np_; ++a) {
                int kx = wrap(ix + ox + a, p->nx);
                double W = wx[a] * wy[b] * wz[c];
                int64_t node = ((int64_t)kz * p->ny + ky) * p->nx + kx;
                for (int q = 0; q < 6; ++q)
                    acc[q] += W * F[q * ncell + node];
            }
        }
    }
    for (int q = 0; q < 3; ++q) {
        E[q] = acc[q];
        B[q] = acc[q + 3];
    }
}

/* Scatter: G[q](node) += W(x - x_node) * Q[q], for nq quantities (planes of G). */
static void scatter(const orc_params *p, double *G, int nq, const double *Q, int ix,
                    int iy, int iz, double fx, double fy, double fz)
{
    double wx[3], wy[3], wz[3];
    int ox = orc_weights_1d(p->shape, fx, wx);
    int oy = orc_weights_1d(p->shape, fy, wy);
    int oz = orc_weights_1d(p->shape, fz, wz);
    int64_t ncell = (int64_t)p->nx * p->ny * p->nz;
    int np_ = npts(p->shape);
    for (int c = 0; c < np_; ++c) {
        int kz = wrap(iz + oz + c, p->nz);
        for (int b = 0; b < np_; ++b) {
            int ky = wrap(iy + oy + b, p->ny);
            for (int a = 0; a < np_; ++a) {
                int kx = wrap(ix + ox + a, p->nx);
                double W = wx[a] * wy[b] * wz[c];
                int64_t node = ((int64_t)kz * p->ny + ky) * p->nx + kx;
                for (int q = 0; q < nq; ++q)
                    G[q * ncell + node] += W * Q[q];
            }
        }
    }
}

static void cross(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * Boris kick-rotate-kick for Eq. momentum.alt with h = (c~/c)(q/(m c)) dt / 2:
 *   u- = u0 + h E,  g- = sqrt(1 + |u-|^2),  t = h B / g-,  s = 2 t / (1 + |t|^2),
 *   u' = u- + u- x t,  u+ = u- + u' x s,  u1 = u+ + h E.
 * The rotation gives u+ - u- = (u+ + u-) x t, i.e. the magnetic term is taken at
 * beta_bar = (u+ + u-) / (2 g-).
 */
void orc_boris(double h, const double E[3], const double B[3], const double u0[3],
               double um[3], double up[3], double u1[3], double *gm)
{
    double t[3], s[3], uprime[3], cr[3];
    for (int q = 0; q < 3; ++q)
        um[q] = u0[q] + h * E[q];
    *gm = sqrt(1.0 + dot(um, um));
    for (int q = 0; q < 3; ++q)
        t[q] = h * B[q] / *gm;
    double t2 = dot(t, t);
    for (int q = 0; q < 3; ++q)
        s[q] = 2.0 * t[q] / (1.0 + t2);
    cross(um, t, cr);
    for (int q = 0; q < 3; ++q)
        uprime[q] = um[q] + cr[q];
    cross(uprime, s, cr);
    for (int q = 0; q < 3; ++q)
        up[q] = um[q] + cr[q];
    for (int q = 0; q < 3; ++q)
        u1[q] = up[q] + h * E[q];
}

/* Boris half-step factor h = (c~/c) (q/m) / c * dt / 2 of Eq. momentum.alt. */
double orc_boris_h(const orc_params *p)
{
    double K = (p->c_tilde / p->c) * (p->q_over_m / p->c);
    return K * p->dt / 2.0;
}

/*
 * Drift x += dt c~ beta / dx on one axis (Sec. 2, v_eff = c~ beta), carried into
 * the integer cell: off += delta; k = floor(off); cell = (cell + k) mod n;
 * off -= k; an offset that rounds up to 1 moves to the next cell at 0.
 */
static void drift_axis(int32_t *cell, double *off, double delta, int n)
{
    double o = *off + delta;
    double k = floor(o);
    o = o - k;
    int ci = *cell + (int)k;
    if (o >= 1.0) {
        o = 0.0;
        ci += 1;
    }
    *cell = wrap(ci, n);
    *off = o;
}

/*
 * The eight feedback quantities of one packet per unit volume, deposited with
 * the gather weights at x^n:
 *   Q0 = N q                         charge
 *   Q1..3 = N q c u1 / g1            current, beta at n+1/2
 *   Q4..6 = -N q [E + beta_bar x B]  momentum source on the gas,
 *                                    beta_bar = (u+ + u-) / (2 g-)
 *                                    (= -(c/c~) N m c (u1 - u0) / dt)
 *   Q7 = -N q c E . (u+ + u-) / (g1 + g0)
 *                                    energy source on the gas
 *                                    (= -(c/c~) N m c^2 (g1 - g0) / dt)
 */
void orc_feedback(const orc_params *p, double N, const double E[3], const double B[3],
                  const double um[3], const double up[3], double gm, const double u1[3],
                  double g0, double g1, double Q[8])
{
    double inv_vol = 1.0 / (p->dx * p->dx * p->dx);
    double Nq = N * p->q * inv_vol;
    double bbar[3], bxB[3], sum[3];
    for (int q = 0; q < 3; ++q) {
        bbar[q] = (up[q] + um[q]) / (2.0 * gm);
        sum[q] = up[q] + um[q];
    }
    cross(bbar, B, bxB);
    Q[0] = Nq;
    for (int q = 0; q < 3; ++q)
        Q[1 + q] = Nq * p->c * u1[q] / g1;
    for (int q = 0; q < 3; ++q)
        Q[4 + q] = -Nq * (E[q] + bxB[q]);
    Q[7] = -Nq * p->c * dot(E, sum) / (g1 + g0);
}

/*
 * One timestep for every packet, in index order: gather E, B at x^n; Boris
 * (u^{n-1/2} -> u^{n+1/2}); deposit the eight feedback quantities into G
 * (8 planes, accumulated; may be NULL) with the x^n weights; drift x^n -> x^{n+1}.
 * F: 6 field planes for time t^n.
 */
void orc_step(const orc_params *p, const double *F, orc_particles *P, double *G)
{
    double h = orc_boris_h(p);
    double adv = p->dt * p->c_tilde / p->dx;
    for (int64_t j = 0; j < P->n; ++j) {
        int ix = P->ix[j], iy = P->iy[j], iz = P->iz[j];
        double fx = P->ox[j], fy = P->oy[j], fz = P->oz[j];
        double E[3], B[3];
        orc_gather(p, F, ix, iy, iz, fx, fy, fz, E, B);
        double u0[3] = {P->ux[j], P->uy[j], P->uz[j]};
        double um[3], up[3], u1[3], gm;
        orc_boris(h, E, B, u0, um, up, u1, &gm);
        double g0 = sqrt(1.0 + dot(u0, u0));
        double g1 = sqrt(1.0 + dot(u1, u1));
        if (G) {
            double Q[8];
            orc_feedback(p, P->w[j], E, B, um, up, gm, u1, g0, g1, Q);
            scatter(p, G, 8, Q, ix, iy, iz, fx, fy, fz);
        }
        int32_t cx = ix, cy = iy, cz = iz;
        drift_axis(&cx, &P->ox[j], adv * u1[0] / g1, p->nx);
        drift_axis(&cy, &P->oy[j], adv * u1[1] / g1, p->ny);
        drift_axis(&cz, &P->oz[j], adv * u1[2] / g1, p->nz);
        P->ix[j] = cx;
        P->iy[j] = cy;
        P->iz[j] = cz;
        P->ux[j] = u1[0];
        P->uy[j] = u1[1];
        P->uz[j] = u1[2];
    }
}

/*
 * State moments at the current positions and momenta (Sec. 2 packet totals
 * per unit volume), 8 planes of G, accumulated:
 *   0 number density N;  1..3 momentum density N m c u;  4 energy density
 *   N gamma m c^2;  5..7 current density N q c u / gamma.
 */
void orc_state_moments(const orc_params *p, const orc_particles *P, double *G)
{
    double m = p->q / p->q_over_m;
    double inv_vol = 1.0 / (p->dx * p->dx * p->dx);
    for (int64_t j = 0; j < P->n; ++j) {
        double u[3] = {P->ux[j], P->uy[j], P->uz[j]};
        double g = sqrt(1.0 + dot(u, u));
        double N = P->w[j] * inv_vol;
        double Q[8];
        Q[0] = N;
        for (int q = 0; q < 3; ++q)
            Q[1 + q] = N * m * p->c * u[q];
        Q[4] = N * g * m * p->c * p->c;
        for (int q = 0; q < 3; ++q)
            Q[5 + q] = N * p->q * p->c * u[q] / g;
        scatter(p, G, 8, Q, P->ix[j], P->iy[j], P->iz[j], P->ox[j], P->oy[j], P->oz[j]);
    }
}

/*
 * Global packet totals (Sec. 2): out[0] = sum N_j, out[1..3] = sum P_j =
 * sum N_j m c u_j, out[4] = sum E_j = sum N_j gamma_j m c^2,
 * out[5..7] = sum N_j q c beta_j.
 */
void orc_totals(const orc_params *p, const orc_particles *P, double out[8])
{
    double m = p->q / p->q_over_m;
    for (int q = 0; q < 8; ++q)
        out[q] = 0.0;
    for (int64_t j = 0; j < P->n; ++j) {
        double u[3] = {P->ux[j], P->uy[j], P->uz[j]};
        double g = sqrt(1.0 + dot(u, u));
        double N = P->w[j];
        out[0] += N;
        for (int q = 0; q < 3; ++q)
            out[1 + q] += N * m * p->c * u[q];
        out[4] += N * g * m * p->c * p->c;
        for (int q = 0; q < 3; ++q)
            out[5 + q] += N * p->q * p->c * u[q] / g;
    }
}

/*
 * Node that anchors a packet's stencil on one axis, the sort coordinate:
 * CIC: the cell's lower node i; TSC: the nearest node, i + 1 when f >= 1/2
 * (periodic), so packets with equal anchors share all 27 stencil nodes.
 */
int32_t orc_anchor_node(int32_t shape, int32_t i, double f, int32_t n)
{
    if (shape == 2 && f >= 0.5)
        return (i + 1) % n;
    return i;
}

/*
 * Sort key of a cell: cells are grouped into cubic bins of edge `bin` cells
 * (partial bins at the high faces when bin does not divide n); the key is the
 * bin's linear index (x fastest) times bin^3 plus the cell's linear index
 * inside the bin (x fastest).  bin = 1 gives the plain linear cell index.
 */
int64_t orc_cell_key(int32_t nx, int32_t ny, int32_t nz, int32_t bin, int32_t ix,
                     int32_t iy, int32_t iz)
{
    int64_t nbx = (nx + bin - 1) / bin, nby = (ny + bin - 1) / bin;
    (void)nz;
    int64_t bx = ix / bin, by = iy / bin, bz = iz / bin;
    int64_t lx = ix % bin, ly = iy % bin, lz = iz % bin;
    int64_t b3 = (int64_t)bin * bin * bin;
    return ((bz * nby + by) * nbx + bx) * b3 + (lz * bin + ly) * bin + lx;
}

/*
 * Stable counting sort of n keys in [0, nkeys): perm[r] = index of the r-th
 * element in the sorted order, equal keys in their original order.  Returns 0,
 * or -1 for a key out of range or no memory.
 */
int orc_stable_sort(const int64_t *key, int64_t n, int64_t nkeys, int64_t *perm)
{
    int64_t *count = (int64_t *)calloc((size_t)nkeys + 1, sizeof(int64_t));
    if (!count)
        return -1;
    for (int64_t j = 0; j < n; ++j) {
        if (key[j] < 0 || key[j] >= nkeys) {
            free(count);
            return -1;
        }
        count[key[j] + 1] += 1;
    }
    for (int64_t k = 0; k < nkeys; ++k)
        count[k + 1] += count[k];
    for (int64_t j = 0; j < n; ++j)
        perm[count[key[j]]++] = j;
    free(count);
    return 0;
}

/*
 * Catastrophic losses (Sec. 2, collisional terms): a packet loses CRs at the
 * true rate <sigma v> n_n, slowed by c~/c like every CR time derivative, so
 * over one step N_j <- N_j exp(-(c~/c) sigma c beta_j n_n(x_j) dt), with beta_j
 * at the packet's current momentum and n_n gathered with W (or uniform when nn
 * is NULL).  M_j, E_j and P_j are proportional to N_j and decay with it.
 */
void orc_losses(const orc_params *p, orc_particles *P, const double *nn, double nn_uniform,
                double sigma)
{
    int64_t ncell = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t j = 0; j < P->n; ++j) {
        double u[3] = {P->ux[j], P->uy[j], P->uz[j]};
        double g = sqrt(1.0 + dot(u, u));
        double beta = sqrt(dot(u, u)) / g;
        double n_n = nn_uniform;
        if (nn) {
            double wx[3], wy[3], wz[3];
            int ox = orc_weights_1d(p->shape, P->ox[j], wx);
            int oy = orc_weights_1d(p->shape, P->oy[j], wy);
            int oz = orc_weights_1d(p->shape, P->oz[j], wz);
            int np_ = npts(p->shape);
            n_n = 0.0;
            for (int c = 0; c < np_; ++c)
                for (int b = 0; b < np_; ++b)
                    for (int a = 0; a < np_; ++a) {
                        int kx = wrap(P->ix[j] + ox + a, p->nx);
                        int ky = wrap(P->iy[j] + oy + b, p->ny);
                        int kz = wrap(P->iz[j] + oz + c, p->nz);
                        n_n += wx[a] * wy[b] * wz[c] * nn[((int64_t)kz * p->ny + ky) * p->nx + kx];
                    }
            (void)ncell;
        }
        double rate = (p->c_tilde / p->c) * sigma * p->c * beta * n_n;
        P->w[j] *= exp(-rate * p->dt);
    }
}

/*
 * Forward-mode tangent of the packet step (used to check the library's
 * reverse-mode gradients by an independent method).  Loss of a run of
 * n_steps steps: L = || sum_n S^n ||_2 over every node and the three
 * components of the momentum source S (the deposited back-reaction of Sec. 2).
 * Given a direction dF of the fields (per step, or one static grid when
 * f_stride == 0), propagates d(x, u) packet by packet alongside the step and
 * returns out[0] = L, out[1] = dL/d(eps) along dF.  Fields F and dF hold
 * n_steps blocks of 6 planes (stride f_stride doubles between steps).
 */
static void dweights_1d(int shape, double f, double w[3], double dw[3], int *first)
{
    *first = orc_weights_1d(shape, f, w);
    if (shape == 1) {
        dw[0] = -1.0;
        dw[1] = 1.0;
        dw[2] = 0.0;
        return;
    }
    double d = f < 0.5 ? f : f - 1.0;
    dw[0] = -(0.5 - d);
    dw[1] = -2.0 * d;
    dw[2] = 0.5 + d;
}

void orc_tangent_run(const orc_params *p, int n_steps, const double *F, const double *dF,
                     int64_t f_stride, orc_particles *P, double out[2])
{
    int64_t ncell = (int64_t)p->nx * p->ny * p->nz;
    double *G = (double *)calloc((size_t)(3 * ncell), sizeof(double));
    double *dG = (double *)calloc((size_t)(3 * ncell), sizeof(double));
    double *dx = (double *)calloc((size_t)(3 * P->n), sizeof(double));
    double *du = (double *)calloc((size_t)(3 * P->n), sizeof(double));
    double h = orc_boris_h(p);
    double adv = p->c_tilde * p->dt / p->dx;
    double inv_vol = 1.0 / (p->dx * p->dx * p->dx);
    int np_ = npts(p->shape);
    for (int n = 0; n < n_steps; ++n) {
        const double *Fn = F + n * f_stride;
        const double *dFn = dF + n * f_stride;
        for (int64_t j = 0; j < P->n; ++j) {
            int32_t ci[3] = {P->ix[j], P->iy[j], P->iz[j]};
            double f[3] = {P->ox[j], P->oy[j], P->oz[j]};
            int nn[3] = {p->nx, p->ny, p->nz};
            double w[3][3], dw[3][3];
            int first[3];
            for (int a = 0; a < 3; ++a)
                dweights_1d(p->shape, f[a], w[a], dw[a], &first[a]);
            double E[3] = {0, 0, 0}, B[3] = {0, 0, 0}, dE[3] = {0, 0, 0}, dB[3] = {0, 0, 0};
            double *dxj = dx + 3 * j, *duj = du + 3 * j;
            int64_t nodes[27];
            double Wk[27], dWk[27];
            int K = 0;
            for (int c = 0; c < np_; ++c)
                for (int b = 0; b < np_; ++b)
                    for (int a = 0; a < np_; ++a) {
                        int kx = wrap(ci[0] + first[0] + a, nn[0]);
                        int ky = wrap(ci[1] + first[1] + b, nn[1]);
                        int kz = wrap(ci[2] + first[2] + c, nn[2]);
                        nodes[K] = ((int64_t)kz * p->ny + ky) * p->nx + kx;
                        Wk[K] = w[0][a] * w[1][b] * w[2][c];
                        dWk[K] = dw[0][a] * w[1][b] * w[2][c] * dxj[0] +
                                 w[0][a] * dw[1][b] * w[2][c] * dxj[1] +
                                 w[0][a] * w[1][b] * dw[2][c] * dxj[2];
                        for (int q = 0; q < 3; ++q) {
                            E[q] += Wk[K] * Fn[q * ncell + nodes[K]];
                            B[q] += Wk[K] * Fn[(3 + q) * ncell + nodes[K]];
                            dE[q] += dWk[K] * Fn[q * ncell + nodes[K]] + Wk[K] * dFn[q * ncell + nodes[K]];
                            dB[q] += dWk[K] * Fn[(3 + q) * ncell + nodes[K]] +
                                     Wk[K] * dFn[(3 + q) * ncell + nodes[K]];
                        }
                        ++K;
                    }
            /* Boris with tangents */
            double u0[3] = {P->ux[j], P->uy[j], P->uz[j]};
            double um[3], dum[3], t[3], dtt[3], s[3], ds[3], up_[3], dup[3], upr[3], dupr[3];
            double cr[3], cr2[3], cr3[3];
            for (int q = 0; q < 3; ++q) {
                um[q] = u0[q] + h * E[q];
                dum[q] = duj[q] + h * dE[q];
            }
            double gm = sqrt(1.0 + dot(um, um));
            double dgm = dot(um, dum) / gm;
            for (int q = 0; q < 3; ++q) {
                t[q] = h * B[q] / gm;
                dtt[q] = h * dB[q] / gm - h * B[q] * dgm / (gm * gm);
            }
            double t2 = dot(t, t), dt2 = 2.0 * dot(t, dtt);
            for (int q = 0; q < 3; ++q) {
                s[q] = 2.0 * t[q] / (1.0 + t2);
                ds[q] = 2.0 * dtt[q] / (1.0 + t2) - 2.0 * t[q] * dt2 / ((1.0 + t2) * (1.0 + t2));
            }
            cross(um, t, cr);
            cross(dum, t, cr2);
            cross(um, dtt, cr3);
            for (int q = 0; q < 3; ++q) {
                upr[q] = um[q] + cr[q];
                dupr[q] = dum[q] + cr2[q] + cr3[q];
            }
            cross(upr, s, cr);
            cross(dupr, s, cr2);
            cross(upr, ds, cr3);
            for (int q = 0; q < 3; ++q) {
                up_[q] = um[q] + cr[q];
                dup[q] = dum[q] + cr2[q] + cr3[q];
            }
            double u1[3], du1[3];
            for (int q = 0; q < 3; ++q) {
                u1[q] = up_[q] + h * E[q];
                du1[q] = dup[q] + h * dE[q];
            }
            /* momentum source and its tangent */
            double Nq = P->w[j] * p->q * inv_vol;
            double bb[3], dbb[3], S[3], dS[3];
            for (int q = 0; q < 3; ++q) {
                bb[q] = (up_[q] + um[q]) / (2.0 * gm);
                dbb[q] = (dup[q] + dum[q]) / (2.0 * gm) - (up_[q] + um[q]) * dgm / (2.0 * gm * gm);
            }
            cross(bb, B, cr);
            cross(dbb, B, cr2);
            cross(bb, dB, cr3);
            for (int q = 0; q < 3; ++q) {
                S[q] = -Nq * (E[q] + cr[q]);
                dS[q] = -Nq * (dE[q] + cr2[q] + cr3[q]);
            }
            for (int k = 0; k < K; ++k)
                for (int q = 0; q < 3; ++q) {
                    G[q * ncell + nodes[k]] += Wk[k] * S[q];
                    dG[q * ncell + nodes[k]] += dWk[k] * S[q] + Wk[k] * dS[q];
                }
            /* drift and its tangent (the carry does not change the position) */
            double g1 = sqrt(1.0 + dot(u1, u1));
            double dg1 = dot(u1, du1) / g1;
            for (int q = 0; q < 3; ++q)
                dxj[q] += adv * (du1[q] / g1 - u1[q] * dg1 / (g1 * g1));
            int32_t cx = ci[0], cy = ci[1], cz = ci[2];
            double beta[3] = {u1[0] / g1, u1[1] / g1, u1[2] / g1};
            drift_axis(&cx, &P->ox[j], adv * beta[0], p->nx);
            drift_axis(&cy, &P->oy[j], adv * beta[1], p->ny);
            drift_axis(&cz, &P->oz[j], adv * beta[2], p->nz);
            P->ix[j] = cx;
            P->iy[j] = cy;
            P->iz[j] = cz;
            P->ux[j] = u1[0];
            P->uy[j] = u1[1];
            P->uz[j] = u1[2];
            for (int q = 0; q < 3; ++q)
                duj[q] = du1[q];
        }
    }
    double L2 = 0.0, dL = 0.0;
    for (int64_t i = 0; i < 3 * ncell; ++i) {
        L2 += G[i] * G[i];
        dL += G[i] * dG[i];
    }
    out[0] = sqrt(L2);
    out[1] = out[0] > 0 ? dL / out[0] : 0.0;
    free(G);
    free(dG);
    free(dx);
    free(du);
}

/*
 * Per-packet timestep limit (Sec. 3, timestep constraints).  Every CR time
 * derivative carries c~/c, so every CR constraint is c/c~ times its usual
 * value:
 *   gyration     dt_j < C / Omega~_j,  Omega~_j = (c~/c) |q/m| |B(x_j)| / (gamma_j c)
 *   CR Courant   dt_j < C dx / |v_eff|, |v_eff| = c~ beta_j
 *   losses       dt_j < C N_j / |dN_j/dt| = C / ((c~/c) sigma n_n c beta_j)
 * (sigma_nn = sigma n_n, uniform; 0 = no losses).  B is gathered at x_j with
 * W, gamma and beta are those of u_j.  Returns C times the smallest bound
 * that applies (HUGE_VAL when none does).
 */
double orc_dt_limit(const orc_params *p, const double *F, const orc_particles *P, int64_t j,
                    double courant, double sigma_nn)
{
    double E[3], B[3];
    orc_gather(p, F, P->ix[j], P->iy[j], P->iz[j], P->ox[j], P->oy[j], P->oz[j], E, B);
    double u[3] = {P->ux[j], P->uy[j], P->uz[j]};
    double u2 = dot(u, u);
    double g = sqrt(1.0 + u2);
    double beta = sqrt(u2) / g;
    double bmag = sqrt(dot(B, B));
    double lim = HUGE_VAL;
    double omega = ((p->c_tilde / p->c) * fabs(p->q_over_m) / p->c) * bmag / g;
    if (omega > 0.0)
        lim = 1.0 / omega;
    if (beta > 0.0) {
        double t_cross = (p->dx / p->c_tilde) / beta;
        if (t_cross < lim)
            lim = t_cross;
        if (sigma_nn > 0.0) {
            double t_loss = (1.0 / ((p->c_tilde / p->c) * sigma_nn * p->c)) / beta;
            if (t_loss < lim)
                lim = t_loss;
        }
    }
    return courant * lim;
}

/* Sub-cycling level: the smallest k in [0, max_level] with dt / 2^k <= limit. */
int orc_subcycle_level(double dt, double limit, int max_level)
{
    int k = 0;
    double dts = dt;
    while (k < max_level && dts > limit) {
        dts *= 0.5;
        ++k;
    }
    return k;
}

/*
 * One global step dt with per-packet sub-cycling: packet j takes 2^k_j
 * sub-steps of dt / 2^k_j in the fields F (held over the step), k_j from its
 * limit at the start of the step.  Each sub-step is the packet's own orc_step
 * with the sub-step's dt and, for the deposit, its weight times 2^-k_j, so G
 * receives the time average over dt of the eight densities.  levels (may be
 * NULL) receives k_j.
 */
void orc_step_subcycled(const orc_params *p, const double *F, orc_particles *P, double *G,
                        double courant, double sigma_nn, int max_level, int32_t *levels)
{
    for (int64_t j = 0; j < P->n; ++j) {
        double lim = orc_dt_limit(p, F, P, j, courant, sigma_nn);
        int k = orc_subcycle_level(p->dt, lim, max_level);
        if (levels)
            levels[j] = k;
        orc_params ps = *p;
        ps.dt = ldexp(p->dt, -k);
        double wsub = ldexp(P->w[j], -k);
        orc_particles one;
        one.n = 1;
        one.ix = &P->ix[j];
        one.iy = &P->iy[j];
        one.iz = &P->iz[j];
        one.ox = &P->ox[j];
        one.oy = &P->oy[j];
        one.oz = &P->oz[j];
        one.ux = &P->ux[j];
        one.uy = &P->uy[j];
        one.uz = &P->uz[j];
        one.w = &wsub;
        for (long s = 0; s < (1L << k); ++s)
            orc_step(&ps, F, &one, G);
    }
}
