/*
 * rsol.h -- C ABI of librsol, the GB300 (sm_103a) implementation of the
 * cosmic-ray packet step of the reduced-speed-of-light (RSOL) MHD-PIC method
 * (Ji & Hopkins, arXiv:2111.14704).
 *
 * The method (Sec. 2 of the paper): every CR packet j carries a weight N_j,
 * a position <x>_j and a dimensionless momentum u = gamma beta.  With the true
 * speed of light c and the reduced one c~ both explicit,
 *     d<x>_j/dt      = v_eff = c~ beta                         (Sec. 2, v_eff)
 *     d(gamma beta)/dt = (c~/c) (q/(m c)) [E + beta x B]        (Eq. momentum.alt)
 * and the back-reaction on the gas is -sum_j n_j q [E + beta_j x B]
 * = -sum_j n_j (c/c~) d<p>_j/dt (Sec. 2, force on the gas).
 *
 * One step of this library, per packet: gather E, B at x^n from the node grid
 * with the packet kernel W (CIC or TSC B-spline, nodes at integer
 * coordinates, periodic); Boris kick-rotate-kick u^{n-1/2} -> u^{n+1/2};
 * deposit, with the same x^n weights, the eight feedback densities
 *     rho = N q,  J = N q c beta^{n+1/2},
 *     S = -N q [E + beta_bar x B]     (= -(c/c~) N m c du/dt),
 *     H = -N q c E.(u+ + u-)/(g^{n+1/2} + g^{n-1/2})  (= -(c/c~) N m c^2 dgamma/dt);
 * drift x += dt c~ beta^{n+1/2}, carried into an integer cell.
 *
 * Conventions common to every call
 *   - Units: positions in cells (dx multiplies lengths only in the densities),
 *     u dimensionless, fields in the caller's Gaussian units.
 *   - Device pointers: every array argument named "d_*" or held in
 *     rsol_particles is a CUDA device pointer of the current device; host
 *     pointers are named "h_*".  The caller owns every buffer; the library
 *     borrows them for the duration of the call (which is asynchronous on the
 *     stream given).  The context owns only its scratch.
 *   - Element type: float when params.precision == 32, double when 64, for
 *     every floating array (particles, fields, feedback, moments).
 *   - Grids are node-major, x fastest: element (iz, iy, ix, k) of a grid with
 *     K components per node is at ((iz*ny + iy)*nx + ix)*K + k.
 *       fields   K = 8: Ex Ey Ez Bx By Bz, then two ignored slots;
 *       feedback K = 8: rho Jx Jy Jz Sx Sy Sz H  (accumulated into: zero it);
 *       moments  K = 8: n  Px Py Pz  e  jx jy jz (accumulated into: zero it).
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Calls on one context (rsol_ctx or rsol_batch_ctx) share its scratch
 *     (sort buffers, bin ranges, claim counters): order them on one stream, or
 *     across streams with events.  Distinct contexts may run concurrently.
 *   - Errors: every call returns an rsol_status and never aborts; the message
 *     of the last failure is rsol_last_error(ctx).  Kernel-detected problems
 *     (non-finite momentum, a drift beyond one cell) set a device status word
 *     that rsol_check() reads (it synchronises the stream).
 */
#ifndef RSOL_H
#define RSOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rsol_status {
    RSOL_OK = 0,
    RSOL_ERR_INVALID_ARG = 1, /* a size, pointer, alignment or parameter is invalid   */
    RSOL_ERR_CUDA = 2,        /* a CUDA runtime call or a launch failed               */
    RSOL_ERR_OOM = 3,         /* context scratch could not be allocated               */
    RSOL_ERR_NONFINITE = 4,   /* a packet's momentum became NaN or infinite           */
    RSOL_ERR_COURANT = 5,     /* a packet moved more than one cell in a step          */
    RSOL_ERR_UNSORTED = 6,    /* a sorted-only call got a set rsol_sort did not write */
    RSOL_ERR_TIMEOUT = 7      /* a bounded device wait ran out                        */
} rsol_status;

/* Problem parameters (Sec. 2: grid, species q and q/m, c and c~). */
typedef struct rsol_params {
    int32_t nx, ny, nz;    /* periodic grid, nodes = cells per axis, 2..1024 each      */
    int32_t shape;         /* packet kernel W: 1 = CIC (linear), 2 = TSC (quadratic)   */
    int32_t precision;     /* 32 = float arrays, 64 = double arrays                   */
    int32_t deterministic; /* 1 = order-independent (bit-reproducible) deposits        */
    int32_t bin;           /* sort bin edge in nodes: 1, 2, 4, 8 or 16; 0 = 8 (FP32)   */
                           /* or 4 (FP64); the binned kernel runs for 4 and 8          */
    int32_t warps;         /* CTA width of the binned push, in warps: 8 or 16; 0 =     */
                           /* the widest that fits shared memory (16 for FP32).  The   */
                           /* Python package's autotuner picks bin and warps per GPU   */
                           /* and workload; results do not depend on either.           */
    double dx;             /* cell size (> 0)                                          */
    double c;              /* true speed of light (> 0)                                */
    double c_tilde;        /* reduced speed of light, 0 < c~ <= c                      */
    double q_over_m;       /* charge-to-mass ratio of the species (!= 0)               */
    double q;              /* charge of one CR (!= 0); m = q / q_over_m                */
} rsol_params;

/*
 * Structure-of-arrays packets (Sec. 2 ansatz: weight N_j, position, momentum).
 * cell[j] packs the integer cell of packet j as ix | iy << 10 | iz << 20;
 * off[a][j] in [0, 1) is the offset inside that cell along axis a, so the
 * position is (ix + off[0][j]) * dx, ...; u[a][j] = gamma beta_a; w[j] = N_j.
 * All eight arrays hold n elements, 16-byte aligned.
 */
typedef struct rsol_particles {
    int64_t n;
    uint32_t *cell;
    void *off[3];
    void *u[3];
    void *w;
} rsol_particles;

typedef struct rsol_ctx rsol_ctx;

/* Validate params and create a context on the current device.  *out is set
 * to NULL on failure.  The context allocates its scratch lazily. */
rsol_status rsol_init(const rsol_params *params, rsol_ctx **out);

/* Release the context and its scratch (after the device has finished using
 * it).  Accepts NULL. */
rsol_status rsol_destroy(rsol_ctx *ctx);

/* Human-readable description of the last failure on ctx ("" if none). */
const char *rsol_last_error(const rsol_ctx *ctx);

/*
 * The fused hot step (Sec. 2: Eq. momentum.alt, v_eff, force on the gas):
 * gather E, B from d_fields (time t^n) at x^n, Boris-advance u, deposit the
 * eight feedback densities into d_feedback when it is not NULL, drift x.
 * Updates parts->cell, off and u in place; w is read only.  dt > 0.  When
 * parts is the set the last rsol_sort wrote, the binned shared-memory kernel
 * runs; otherwise a kernel that needs no ordering runs (same results up to
 * the order of floating-point additions; deterministic mode makes each of
 * them bitwise reproducible from run to run).  "The set the last rsol_sort
 * wrote" is decided by buffer identity: parts->cell and parts->n equal the
 * output of this context's last rsol_sort.  If the caller frees that output
 * and a new set happens to reuse the address, the binned kernel runs on it
 * with the old bin ranges: results stay correct (the ranges still partition
 * the packets, and packets outside their bin's tile take the order-free
 * path inside the kernel) but slower, until the next rsol_sort.
 */
rsol_status rsol_push_gather(rsol_ctx *ctx, const rsol_particles *parts,
                             const void *d_fields, double dt, void *d_feedback,
                             void *stream);

/*
 * State moments at the current positions and momenta (Sec. 2 packet totals
 * N_j, P_j = N_j m c u, E_j = N_j gamma m c^2, per unit volume, plus the
 * current N_j q c beta), deposited with W into d_moments (accumulated).
 */
rsol_status rsol_deposit(rsol_ctx *ctx, const rsol_particles *parts, void *d_moments,
                         void *stream);

/*
 * Stable sort of the packets by cell key (bin-major: the bin's linear index,
 * x fastest, times bin^3 plus the cell's linear index inside its bin), from
 * in to out (distinct buffers of the same n).  Equal keys keep their input
 * order, so the permutation is unique and reproducible.  Also records the
 * per-bin ranges that rsol_push_gather's binned kernel uses.  Not in the
 * paper: it orders packets so that gathers and deposits stay on chip.
 * Where the key space (bins x bin^3) is at most 2^26 and at most twice n, a
 * counting sort by key runs (count, scan, place with one atomic per run of
 * equal keys, then each key's packets ordered by input position); otherwise
 * an LSD radix sort.  Both give the same permutation.  The first counting
 * sort of a context allocates 4 bytes per key of scratch.  Cells must lie
 * inside the grid (rsol_push_gather keeps them there); a packet whose cell
 * does not is neither lost nor duplicated, but its place in the order is
 * unspecified, and the next push flags it and leaves it where it is.
 */
rsol_status rsol_sort(rsol_ctx *ctx, const rsol_particles *in, rsol_particles *out,
                      void *stream);

/*
 * Global FP64 totals (Sec. 2 packet totals; the conserved momentum
 * rho u + (c/c~) P of Sec. 2 needs sum P_j).  Writes to h_totals[16] (host):
 *   [0] sum N_j   [1..3] sum N_j m c u   [4] sum N_j gamma m c^2
 *   [5..7] sum N_j q c beta
 *   [8..15] sum over nodes of d_feedback's 8 components times dx^3
 *           (0 when d_feedback is NULL).
 * The reduction order is fixed, so repeated calls give identical bits.
 * Synchronises the stream.
 */
rsol_status rsol_moments(rsol_ctx *ctx, const rsol_particles *parts,
                         const void *d_feedback, double *h_totals, void *stream);

/*
 * Field source standing in for the MHD solver (out of scope in the paper's
 * hot path): B = B0 x + sum_m A_m e_m cos(2 pi n_m . r / L - omega_m t + phi_m),
 * omega_m = sigma_m k_x vA, gas velocity u = u_gas - sum_m sigma_m vA dB_m / B0,
 * E = -(u/c) x B (Sec. 2, ideal-MHD electric field), written to d_fields.
 * h_modes: n_modes records of 8 doubles (host): n_x n_y n_z (integers, as
 * doubles) e_x e_y e_z A_m phi_m; h_sigma: n_modes doubles (+1 or -1).
 * n_modes <= 256.  Node r = (ix, iy, iz) * dx, L = (nx, ny, nz) * dx.
 */
rsol_status rsol_alfven_fields(rsol_ctx *ctx, const double *h_modes, const double *h_sigma,
                               int32_t n_modes, double t, double B0, double vA,
                               const double *h_u_gas, void *d_fields, void *stream);

/*
 * Catastrophic losses over one step (Sec. 2, collisional terms): every CR
 * time derivative is slowed by c~/c, so a packet that loses CRs at the true
 * rate <sigma v> n_n = sigma c beta n_n keeps
 *     w_j <- w_j exp(-(c~/c) sigma c beta_j n_n(x_j) dt),
 * with beta_j at its current momentum and n_n gathered with W from d_nn (one
 * value per node, node-major, the context's element type) or, when d_nn is
 * NULL, the uniform nn_uniform.  The loss per distance travelled on the grid
 * is then independent of c~.  M_j, E_j and P_j are proportional to N_j and
 * decay with it.  sigma >= 0, n_n >= 0, dt > 0.  Only w is written.
 */
rsol_status rsol_losses(rsol_ctx *ctx, const rsol_particles *parts, const void *d_nn,
                        double nn_uniform, double sigma, double dt, void *stream);

/* Synchronise the stream and return (and clear) the device status word. */
rsol_status rsol_check(rsol_ctx *ctx, void *stream);

/*
 * rsol_sort_static: the same stable sort as rsol_sort (same permutation, same
 * output arrays) for callers that cannot allocate device memory -- code whose
 * device memory is owned by another component's allocator, or host threads
 * that must not wait on the device synchronisation that cudaMalloc/cudaFree
 * can imply.  It takes the parameters directly (no rsol_ctx, whose creation
 * allocates) and never calls cudaMalloc, cudaFree or any allocating routine.
 * The paper has no counterpart: this is a deployment variant of rsol_sort.
 *
 * Scratch: a static device array of 5 MiB inside the library, present on every
 * device that loads it until the process exits.  Problems whose sort buffers
 * do not fit are rejected with RSOL_ERR_INVALID_ARG; the limit covers at least
 * 262,144 packets on grids of up to 65,536 bins (4 + 4 bytes per packet twice,
 * 1 KiB per 4096 packets, 4 bytes per bin).  Every call looks up the array's
 * device address on the current device (no allocation); the first call on a
 * device also loads the library's module there, so make that first call
 * before any stream capture.  All calls share the array: calls that overlap on the device race
 * and must be serialised by the caller.  The bin ranges it computes are not
 * used by rsol_push_gather (which keeps the order-free kernel for this set).
 * Returns RSOL_ERR_CUDA when a launch fails.
 */
rsol_status rsol_sort_static(const rsol_params *params, const rsol_particles *in,
                             rsol_particles *out, void *stream);

/*
 * Batches of independent periodic boxes (each with its own grid, c~ and dt)
 * advanced together by two launches per step (sparse bins, dense bins).  The paper's method
 * is applied to every box unchanged; batching is a systems layer.
 *
 * Packets of all boxes share one rsol_particles: box b owns packets
 * h_offsets[b] .. h_offsets[b+1]-1 (h_offsets[0] = 0, non-decreasing), with
 * cells in its own grid.  Grids (fields, feedback) of all boxes are
 * concatenated node-major: box b's nodes start at node sum_{b'<b} nx*ny*nz;
 * rsol_batch_total_nodes gives the total (each grid holds 8 components per
 * node).  common supplies shape, precision, deterministic, bin (4 or 8, 0 =
 * default), dx, c, q_over_m and q; its nx, ny, nz, c_tilde are ignored.
 * warps: CTA width of the batched kernel, 8 or 16 (0 = 16), chosen by the
 * autotuner of the Python package.
 */
typedef struct rsol_batch_desc {
    int32_t n_boxes;
    int32_t warps;
    const int32_t *h_dims;     /* host, 3 per box: nx, ny, nz (2..1024)              */
    const double *h_c_tilde;   /* host, per box: 0 < c~ <= c                        */
    const double *h_dt;        /* host, per box: dt > 0 with dt c~ / dx <= 1        */
    const int64_t *h_offsets;  /* host, n_boxes + 1 packet offsets                  */
} rsol_batch_desc;

typedef struct rsol_batch_ctx rsol_batch_ctx;

rsol_status rsol_batch_init(const rsol_params *common, const rsol_batch_desc *desc,
                            rsol_batch_ctx **out);
rsol_status rsol_batch_destroy(rsol_batch_ctx *ctx);
const char *rsol_batch_last_error(const rsol_batch_ctx *ctx);
int64_t rsol_batch_total_nodes(const rsol_batch_ctx *ctx);

/* Stable sort of every box's packets by its own bin-major anchor key (as
 * rsol_sort per box), in one pass over the whole set; in and out distinct.
 * Where the batch's box-major key space is at most 2^26 keys and twice the
 * packets, the counting sort of rsol_sort runs, its scratch (4 bytes per key)
 * allocated by rsol_batch_init, so that sorts captured in a CUDA graph
 * allocate nothing; otherwise the radix sort. */
rsol_status rsol_batch_sort(rsol_batch_ctx *ctx, const rsol_particles *in, rsol_particles *out,
                            void *stream);

/* One fused step (as rsol_push_gather) for every box, each with its own c~ and
 * dt, in two launches: one warp per sparse bin (at most 768 packets per 8^3
 * bin, 256 per 4^3 bin; global gathers and atomics), then a persistent kernel
 * running the binned tiles over the dense bins.  parts must be the set
 * rsol_batch_sort last wrote (RSOL_ERR_UNSORTED otherwise).  d_feedback is
 * accumulated into. */
rsol_status rsol_batch_push_gather(rsol_batch_ctx *ctx, const rsol_particles *parts,
                                   const void *d_fields, void *d_feedback, void *stream);

/* The field source of rsol_alfven_fields for box `box`, written into that
 * box's slice of the concatenated field grid. */
rsol_status rsol_batch_alfven_fields(rsol_batch_ctx *ctx, int32_t box, const double *h_modes,
                                     const double *h_sigma, int32_t n_modes, double t, double B0,
                                     double vA, const double *h_u_gas, void *d_fields,
                                     void *stream);

/* Synchronise the stream and return (and clear) the batch's device status word. */
rsol_status rsol_batch_check(rsol_batch_ctx *ctx, void *stream);

/* Number of CUDA kernels this context has launched since rsol_init (a
 * diagnostic for benchmarks; no device work).  Returns -1 for NULL. */
int64_t rsol_kernel_launches(const rsol_ctx *ctx);

/*
 * Per-packet adaptive timestep with sub-cycling (Sec. 3, timestep
 * constraints).  Every CR time derivative carries c~/c, so every CR timestep
 * constraint is c/c~ times its usual value; packet j's limit is
 *     dt_j = C min( 1 / Omega~_j,  dx / (c~ beta_j),  1 / ((c~/c) sigma n_n c beta_j) ),
 *     Omega~_j = (c~/c) |q/m| |B(x_j)| / (gamma_j c),
 * with B gathered with W at x_j and gamma_j, beta_j from u_j at the start of
 * the step (a term is left out when its rate is 0; the loss term when
 * sigma_nn = 0).  The packet takes 2^k_j sub-steps of dt / 2^k_j, k_j the
 * smallest level in [0, max_level] with dt / 2^k_j <= dt_j, each the full
 * step of rsol_push_gather (gather, Boris, feedback, drift) in the fields
 * d_fields held over dt, its deposit carrying 2^-k_j: d_feedback receives the
 * time average over dt of the eight densities (accumulated; may be NULL).
 * Levels are decided in the context's precision.  d_levels (device, n bytes;
 * may be NULL) receives k_j.  Packets keep their order in `parts`; the kernel
 * visits them level by level, so that a warp's lanes take the same number of
 * sub-steps.  Requires c~ dt / dx / 2^max_level <= 1 (no sub-step moves a
 * packet more than one cell); c~ dt / dx itself may exceed 1.
 */
typedef struct rsol_subcycle_desc {
    double courant;     /* C, 0 < C <= 1                                  */
    double sigma_nn;    /* sigma n_n of the loss limit (uniform), >= 0    */
    int32_t max_level;  /* 0 .. 16                                        */
    int32_t reserved;   /* must be 0                                      */
} rsol_subcycle_desc;

rsol_status rsol_push_subcycled(rsol_ctx *ctx, const rsol_particles *parts, const void *d_fields,
                                double dt, const rsol_subcycle_desc *desc, void *d_feedback,
                                uint8_t *d_levels, void *stream);

/*
 * The same sub-cycled step (same levels, same sub-steps, same time-averaged
 * deposit into d_feedback, which is required here) on the shared-memory
 * tiled kernel: the packets of `in` are first sorted into `out` by level
 * (highest first) and, within a level, by the bin-major anchor key of
 * rsol_sort; then, for each sub-step s = 0 .. 2^top - 1 of the highest level
 * present, every level k whose step ends there (s a multiple of 2^(top - k))
 * advances by one binned launch over its own bins, with h, c~ dt/dx and the
 * deposit scaled by 2^-k.  `out` holds the advanced packets in that order; in and out
 * must not share arrays.  Needs the context's bin to be 4 or 8, c~ dt/dx <= 1
 * (the tiles' 2-node halo covers one cell of drift over the step) and
 * (max_level + 1) x bins x bin^3 < 2^31.  h_level_counts (host, max_level + 1
 * int64, may be NULL) receives the packets per level.  Synchronises the stream
 * once, after the sort, to read the level counts.
 */
rsol_status rsol_sort_push_subcycled(rsol_ctx *ctx, const rsol_particles *in, rsol_particles *out,
                                     const void *d_fields, double dt, const rsol_subcycle_desc *desc,
                                     void *d_feedback, int64_t *h_level_counts, void *stream);

/* ------------------------------------------------------------------------
 * Differentiable run (reverse mode).
 *
 * Loss of a run of N steps: L = || sum_{n} S^n ||_2, the Euclidean norm over
 * every node and the three components of the momentum source S (the force
 * density the CRs exert on the gas, Sec. 2) deposited in step n, i.e. of
 * components 4..6 of a feedback grid accumulated over the run.  Gradients
 * are taken with respect to the E, B field grid (a perturbation held fixed
 * over the run, added to every step's fields) and to the amplitudes A_m of
 * the field source of rsol_alfven_fields.  Positions enter in cell units.
 * ------------------------------------------------------------------------ */

/* L and 1/L (0 when L = 0) of the accumulated feedback grid d_feedback
 * (node-major [node][8], the context's type), written to d_loss[0..1]
 * (device doubles).  FP64 sums in a fixed order; no synchronisation. */
rsol_status rsol_loss_norm(rsol_ctx *ctx, const void *d_feedback, double *d_loss, void *stream);

/*
 * Reverse of one rsol_push_gather step n (Sec. 2: gather, Boris push of
 * Eq. momentum.alt, momentum source, drift at c~ beta) for the loss above.
 * parts: the packets' state at the start of step n (x^n, u^n); not modified.
 * d_fields: the fields F^n of that step.  d_feedback, d_loss: the run's
 * accumulated feedback and its rsol_loss_norm.
 * d_xbar, d_ubar: 3 device arrays each (x, y, z) of parts->n elements of the
 * context's type, 16-byte aligned: on entry dL/dx^{n+1} and dL/du^{n+1}, on
 * return dL/dx^n and dL/du^n (zero before the last step).
 * d_field_bar: node-major [node][8] grid of the context's type; dL/dF^n is
 * ADDED to components 0..5 (E, B); 6..7 are not touched.  Uses float or
 * double atomics: the sum order, and so the last bits, vary between runs.
 */
rsol_status rsol_adjoint_step(rsol_ctx *ctx, const rsol_particles *parts, const void *d_fields,
                              double dt, const void *d_feedback, const double *d_loss,
                              void *const d_xbar[3], void *const d_ubar[3], void *d_field_bar,
                              void *stream);

/*
 * Reverse of rsol_alfven_fields at time t with respect to the amplitudes:
 * given d_field_bar = dL/dF (node-major, components 0..5) of the fields it
 * wrote, ADDS sum over nodes of dL/dF . dF/dA_m to d_amp_bar[m] (device
 * doubles, m < n_modes), in a fixed order (bit-reproducible).  B is linear
 * in A and E = -(u/c) x B bilinear in (u, B), so the derivative is exact.
 * When d_field_bar_total is not NULL, d_field_bar is also added into it and
 * then zeroed (components 0..5).  Mode arguments as rsol_alfven_fields;
 * n_modes >= 1.
 */
rsol_status rsol_alfven_adjoint(rsol_ctx *ctx, const double *h_modes, const double *h_sigma,
                                int32_t n_modes, double t, double B0, double vA,
                                const double *h_u_gas, void *d_field_bar, void *d_field_bar_total,
                                double *d_amp_bar, void *stream);

/* Field source of a differentiable run: a static grid, or the Alfven modes
 * evaluated at t0 + n dt in step n (exactly one of the two). */
typedef struct rsol_grad_desc {
    int32_t steps;              /* push + deposit steps, >= 1                         */
    int32_t checkpoint_every;   /* k >= 1: packet states kept every k steps; the     */
                                /* reverse sweep recomputes the k - 1 between         */
    double dt;                  /* step, 0 < c~ dt / dx <= 1                          */
    const void *d_fields;       /* static node-major field grid, or NULL             */
    const double *h_modes;      /* host, as rsol_alfven_fields (when d_fields NULL)  */
    const double *h_sigma;
    int32_t n_modes;
    int32_t reserved;           /* must be 0                                         */
    double t0, B0, vA;
    const double *h_u_gas;      /* host, 3 doubles                                   */
} rsol_grad_desc;

/*
 * Whole differentiable run: sorts a copy of parts (rsol_sort), runs
 * desc->steps forward steps (rsol_push_gather, accumulating d_feedback, which
 * is zeroed first) keeping the packet state every checkpoint_every steps,
 * computes L (rsol_loss_norm into d_loss[0..1]), then sweeps the steps in
 * reverse, recomputing each segment's states from its checkpoint with the
 * forward step (bitwise the same states) and applying rsol_adjoint_step and,
 * for mode fields, rsol_alfven_adjoint.  On return d_field_bar (zeroed first)
 * holds dL/dF for a field perturbation held fixed over the run, and
 * d_amp_bar (mode fields only, n_modes doubles, zeroed first; may be NULL)
 * dL/dA.  parts is not modified.  Scratch: about
 * (steps / k + k) * n * (4 + 6 * elem) + n * (4 + 13 * elem) bytes, plus for
 * mode fields one node-major grid per step (the forward sweep keeps every
 * step's fields for the reverse sweep while they fit in 16 GiB, else they are
 * evaluated again), kept by the context for later calls.  Everything runs on
 * `stream`; the call returns without synchronising.  Once a first call with the
 * same sizes has grown the scratch, a call allocates nothing and never waits on
 * the host, so it can be captured in a CUDA graph and replayed.
 */
rsol_status rsol_gradient(rsol_ctx *ctx, const rsol_particles *parts, const rsol_grad_desc *desc,
                          void *d_feedback, double *d_loss, void *d_field_bar, double *d_amp_bar,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RSOL_H */
