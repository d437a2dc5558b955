// C-ABI layer of the differentiable run: loss, reverse step, field-source
// adjoint and the checkpointed driver (contracts in include/rsol.h).
#include <cmath>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "../../include/rsol.h"
#include "rsol_ctx.h"
#include "rsol_internal.h"

using namespace rsol_api;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Upper bound on the per-step field grids rsol_gradient keeps for mode fields.
constexpr size_t kFieldCacheBytes = size_t(16) << 30;

// One packet state (no weights): cell, offsets, momenta.
struct State {
    uint32_t *cell;
    void *off[3];
    void *u[3];
};

size_t state_bytes(int64_t n, int es) { return align256(size_t(n) * 4) + 6 * align256(size_t(n) * es); }

State carve_state(char *&p, int64_t n, int es)
{
    State s;
    s.cell = reinterpret_cast<uint32_t *>(p);
    p += align256(size_t(n) * 4);
    for (int a = 0; a < 3; ++a) {
        s.off[a] = p;
        p += align256(size_t(n) * es);
    }
    for (int a = 0; a < 3; ++a) {
        s.u[a] = p;
        p += align256(size_t(n) * es);
    }
    return s;
}

rsol_particles as_particles(const State &s, int64_t n, void *w)
{
    rsol_particles P;
    P.n = n;
    P.cell = s.cell;
    for (int a = 0; a < 3; ++a) {
        P.off[a] = s.off[a];
        P.u[a] = s.u[a];
    }
    P.w = w;
    return P;
}

cudaError_t copy_state(const State &dst, const State &src, int64_t n, int es, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(dst.cell, src.cell, size_t(n) * 4, cudaMemcpyDeviceToDevice, st);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        e = cudaMemcpyAsync(dst.off[a], src.off[a], size_t(n) * es, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst.u[a], src.u[a], size_t(n) * es, cudaMemcpyDeviceToDevice, st);
    }
    return e;
}

bool modes_ok(const double *h_modes, const double *h_sigma, int n_modes, const double *u_gas)
{
    return n_modes >= 1 && n_modes <= 256 && h_modes && h_sigma && u_gas;
}

} // namespace

extern "C" {

rsol_status rsol_loss_norm(rsol_ctx *ctx, const void *d_feedback, double *d_loss, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    if (!d_feedback || !aligned16(d_feedback) || !d_loss)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_loss_norm: feedback (16-byte aligned) and loss required");
    cudaError_t e = rsol::loss_norm(d_feedback, n_nodes(ctx), ctx->p.precision, ctx->d_partials,
                                    TOTALS_BLOCKS, d_loss, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_loss_norm launch");
    ctx->launches += 2;
    return RSOL_OK;
}

} // extern "C"

namespace {

// The reverse step on `P`; bin_start (or null) the bin ranges of the sort
// that produced P's order, for the tiled kernel.
rsol_status adjoint_launch(rsol_ctx *ctx, const rsol_particles *P, const void *d_fields, double dt,
                           const void *d_feedback, const double *d_loss, void *const d_xbar[3],
                           void *const d_ubar[3], void *d_field_bar, const uint32_t *bin_start,
                           void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, P, "rsol_adjoint_step");
    if (st != RSOL_OK)
        return st;
    if (!(std::isfinite(dt) && dt > 0))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_adjoint_step: dt must be finite and > 0");
    const double adv = dt * ctx->p.c_tilde / ctx->p.dx;
    if (adv > 1.0)
        return fail(ctx, RSOL_ERR_COURANT, "rsol_adjoint_step: c~ dt / dx = %g > 1", adv);
    if (!d_fields || !aligned16(d_fields) || !d_feedback || !aligned16(d_feedback) || !d_loss ||
        !d_field_bar || !aligned16(d_field_bar) || !d_xbar || !d_ubar)
        return fail(ctx, RSOL_ERR_INVALID_ARG,
                    "rsol_adjoint_step: fields, feedback, field_bar (16-byte aligned), loss, xbar, ubar required");
    for (int a = 0; a < 3; ++a)
        if (!d_xbar[a] || !d_ubar[a] || !aligned16(d_xbar[a]) || !aligned16(d_ubar[a]))
            return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_adjoint_step: xbar/ubar arrays NULL or not aligned");
    if (P->n == 0)
        return RSOL_OK;
    rsol::AdjDesc d{};
    d.n = P->n;
    d.cell = P->cell;
    for (int a = 0; a < 3; ++a) {
        d.off[a] = P->off[a];
        d.u[a] = P->u[a];
        d.xb[a] = d_xbar[a];
        d.ub[a] = d_ubar[a];
    }
    d.w = P->w;
    d.fields = d_fields;
    d.fb = d_feedback;
    d.loss = d_loss;
    d.fbar = d_field_bar;
    d.nx = ctx->p.nx;
    d.ny = ctx->p.ny;
    d.nz = ctx->p.nz;
    d.shape = ctx->p.shape;
    d.h = (ctx->p.c_tilde / ctx->p.c) * (ctx->p.q_over_m / ctx->p.c) * dt / 2.0;
    d.adv = adv;
    d.qv = ctx->p.q / (ctx->p.dx * ctx->p.dx * ctx->p.dx);
    d.c = ctx->p.c;
    d.status = ctx->d_status;
    d.sm_count = ctx->sm_count;
    d.bin_start = bin_start;
    d.bin = ctx->bin;
    d.nbx = ctx->nbx;
    d.nby = ctx->nby;
    d.nbz = ctx->nbz;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = ctx->p.precision == 32 ? rsol::adjoint_step_f32(d, s) : rsol::adjoint_step_f64(d, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_adjoint_step launch");
    ctx->launches += 1;
    return RSOL_OK;
}

} // namespace

extern "C" {

rsol_status rsol_adjoint_step(rsol_ctx *ctx, const rsol_particles *P, const void *d_fields,
                              double dt, const void *d_feedback, const double *d_loss,
                              void *const d_xbar[3], void *const d_ubar[3], void *d_field_bar,
                              void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    const bool sorted = P && ctx->sorted_cell == P->cell && ctx->sorted_n == P->n;
    return adjoint_launch(ctx, P, d_fields, dt, d_feedback, d_loss, d_xbar, d_ubar, d_field_bar,
                          sorted ? ctx->sort.bin_start : nullptr, stream);
}

rsol_status rsol_alfven_adjoint(rsol_ctx *ctx, const double *h_modes, const double *h_sigma,
                                int32_t n_modes, double t, double B0, double vA,
                                const double *h_u_gas, void *d_field_bar, void *d_field_bar_total,
                                double *d_amp_bar, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    if (!modes_ok(h_modes, h_sigma, n_modes, h_u_gas))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_alfven_adjoint: bad mode arrays (1 <= n_modes <= 256)");
    if (!(std::isfinite(B0) && B0 != 0 && std::isfinite(vA) && std::isfinite(t)))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_alfven_adjoint: B0, vA, t must be finite, B0 != 0");
    if (!d_field_bar || !aligned16(d_field_bar) || !d_amp_bar ||
        (d_field_bar_total && !aligned16(d_field_bar_total)))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_alfven_adjoint: field_bar (aligned) and amp_bar required");
    const size_t need = rsol::alfven_adjoint_scratch_bytes(ctx->p.nx, ctx->p.ny, ctx->p.nz, n_modes);
    rsol_status st = ensure_buffer(ctx, &ctx->field_mem, &ctx->field_bytes, need, "field scratch");
    if (st != RSOL_OK)
        return st;
    cudaError_t e = rsol::alfven_adjoint(h_modes, h_sigma, n_modes, t, B0, vA, h_u_gas, ctx->p.c,
                                         ctx->p.dx, ctx->p.nx, ctx->p.ny, ctx->p.nz, ctx->p.precision,
                                         d_field_bar, d_field_bar_total, d_amp_bar, ctx->field_mem,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_alfven_adjoint launch");
    ctx->launches += 4;
    return RSOL_OK;
}

rsol_status rsol_gradient(rsol_ctx *ctx, const rsol_particles *parts, const rsol_grad_desc *g,
                          void *d_feedback, double *d_loss, void *d_field_bar, double *d_amp_bar,
                          void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, parts, "rsol_gradient");
    if (st != RSOL_OK)
        return st;
    if (!g || g->steps < 1 || g->checkpoint_every < 1 || g->reserved != 0 ||
        !(std::isfinite(g->dt) && g->dt > 0))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_gradient: steps >= 1, checkpoint_every >= 1, dt > 0 required");
    const bool use_modes = g->d_fields == nullptr;
    if (use_modes) {
        if (!modes_ok(g->h_modes, g->h_sigma, g->n_modes, g->h_u_gas))
            return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_gradient: no static fields and bad mode arrays");
        if (!(std::isfinite(g->B0) && g->B0 != 0 && std::isfinite(g->vA) && std::isfinite(g->t0)))
            return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_gradient: B0, vA, t0 must be finite, B0 != 0");
    } else if (!aligned16(g->d_fields)) {
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_gradient: fields not 16-byte aligned");
    }
    if (!d_feedback || !aligned16(d_feedback) || !d_loss || !d_field_bar || !aligned16(d_field_bar))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_gradient: feedback, loss and field_bar required");
    if (g->dt * ctx->p.c_tilde / ctx->p.dx > 1.0)
        return fail(ctx, RSOL_ERR_COURANT, "rsol_gradient: c~ dt / dx > 1");
    const int64_t n = parts->n;
    const int es = elem_bytes(ctx);
    const int k = g->checkpoint_every < g->steps ? g->checkpoint_every : g->steps;
    const int nseg = (g->steps + k - 1) / k;
    const size_t grid_bytes = size_t(n_nodes(ctx)) * 8 * es;
    const size_t n_modes = use_modes ? size_t(g->n_modes) : 0;
    const size_t wbytes = align256(size_t(n) * es);
    const size_t bs_bytes = align256(size_t(ctx->nbins + 1) * 4);

    // scratch: two work sets (the forward sweep re-sorts the packets at every
    // checkpoint), per segment a checkpoint with its weights, the sort's
    // permutation and bin ranges, the segment's rebuilt states, two sets of
    // adjoints, and for mode fields the field grids, the per-step field
    // adjoint and a spare amplitude accumulator
    const size_t sb = state_bytes(n, es);
    size_t need = 2 * (sb + wbytes) + size_t(nseg) * (sb + wbytes + align256(size_t(n) * 4) + bs_bytes) +
                  size_t(k - 1) * sb + 12 * wbytes;
    // mode fields: every step's grid is kept from the forward sweep (the
    // reverse sweep then reads it back instead of evaluating the modes again)
    // unless that would take more than kFieldCacheBytes
    const bool cache_fields = use_modes && double(g->steps) * double(grid_bytes) <= double(kFieldCacheBytes);
    const int n_field_bufs = use_modes ? (cache_fields ? g->steps : 1) : 0;
    if (use_modes)
        need += size_t(n_field_bufs) * align256(grid_bytes) + align256(grid_bytes) +
                align256(n_modes * sizeof(double));
    if ((st = ensure_buffer(ctx, &ctx->grad_mem, &ctx->grad_bytes, need, "gradient scratch")) != RSOL_OK)
        return st;
    if (use_modes) {
        const size_t fneed = rsol::alfven_adjoint_scratch_bytes(ctx->p.nx, ctx->p.ny, ctx->p.nz, g->n_modes);
        if ((st = ensure_buffer(ctx, &ctx->field_mem, &ctx->field_bytes, fneed, "field scratch")) != RSOL_OK)
            return st;
    }
    char *p = static_cast<char *>(ctx->grad_mem);
    State work[2];
    void *work_w[2];
    for (int i = 0; i < 2; ++i) {
        work[i] = carve_state(p, n, es);
        work_w[i] = p;
        p += wbytes;
    }
    State *ck = new (std::nothrow) State[size_t(nseg) + size_t(k)];
    void **ck_w = new (std::nothrow) void *[size_t(nseg)];
    uint32_t **perm = new (std::nothrow) uint32_t *[size_t(nseg)];
    uint32_t **bstart = new (std::nothrow) uint32_t *[size_t(nseg)];
    auto release = [&]() {
        delete[] ck;
        delete[] ck_w;
        delete[] perm;
        delete[] bstart;
    };
    if (!ck || !ck_w || !perm || !bstart) {
        release();
        return fail(ctx, RSOL_ERR_OOM, "rsol_gradient: host state tables");
    }
    State *seg = ck + nseg;
    for (int i = 0; i < nseg; ++i) {
        ck[i] = carve_state(p, n, es);
        ck_w[i] = p;
        p += wbytes;
        perm[i] = reinterpret_cast<uint32_t *>(p);
        p += align256(size_t(n) * 4);
        bstart[i] = reinterpret_cast<uint32_t *>(p);
        p += bs_bytes;
    }
    for (int i = 1; i < k; ++i)
        seg[i] = carve_state(p, n, es);
    void *xb[2][3], *ub[2][3];
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 3; ++a) {
            xb[b][a] = p;
            p += wbytes;
            ub[b][a] = p;
            p += wbytes;
        }
    void *F = const_cast<void *>(g->d_fields);
    char *field_cache = nullptr;
    void *fbar_step = nullptr;
    double *amp = d_amp_bar;
    if (use_modes) {
        field_cache = p;
        F = p;
        p += size_t(n_field_bufs) * align256(grid_bytes);
        fbar_step = p;
        p += align256(grid_bytes);
        if (!amp)
            amp = reinterpret_cast<double *>(p);
        p += align256(n_modes * sizeof(double));
    }

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    // fields of step `step` into F: evaluated in the forward sweep (into the
    // step's cache slot when caching), read back from the cache afterwards
    auto fields_at = [&](int step, bool forward) -> rsol_status {
        if (!use_modes)
            return RSOL_OK;
        if (cache_fields) {
            F = field_cache + size_t(step) * align256(grid_bytes);
            if (!forward)
                return RSOL_OK;
        }
        return rsol_alfven_fields(ctx, g->h_modes, g->h_sigma, g->n_modes, g->t0 + step * g->dt, g->B0,
                                  g->vA, g->h_u_gas, F, stream);
    };
#define RSOL_TRY(expr)                  \
    do {                                \
        if ((st = (expr)) != RSOL_OK) { \
            release();                  \
            return st;                  \
        }                               \
    } while (0)
#define RSOL_TRY_CUDA(expr, what)              \
    do {                                       \
        if ((e = (expr)) != cudaSuccess) {     \
            release();                         \
            return cuda_fail(ctx, e, what);    \
        }                                      \
    } while (0)

    // the sort's final permutation (sorted position -> source position) lies in
    // the index buffer its last radix pass wrote
    const int passes = (ctx->key_bits + 7) / 8;

    // forward sweep: a sort at every checkpoint keeps each segment's packets
    // within their bins' tiles for the segment's k steps
    int cur = 0;
    for (int step = 0; step < g->steps; ++step) {
        if (step % k == 0) {
            const int sg = step / k;
            rsol_particles Wc = as_particles(work[cur], n, work_w[cur]);
            rsol_particles Wn = as_particles(work[cur ^ 1], n, work_w[cur ^ 1]);
            RSOL_TRY(rsol_sort(ctx, step == 0 ? parts : &Wc, &Wn, stream));
            cur ^= 1;
            if (step == 0)
                RSOL_TRY_CUDA(cudaMemsetAsync(d_feedback, 0, grid_bytes, s), "rsol_gradient: zero feedback");
            else
                RSOL_TRY_CUDA(cudaMemcpyAsync(perm[sg], ctx->sort.idx[passes & 1], size_t(n) * 4,
                                              cudaMemcpyDeviceToDevice, s),
                              "rsol_gradient: permutation");
            RSOL_TRY_CUDA(cudaMemcpyAsync(bstart[sg], ctx->sort.bin_start, size_t(ctx->nbins + 1) * 4,
                                          cudaMemcpyDeviceToDevice, s),
                          "rsol_gradient: bin ranges");
            RSOL_TRY_CUDA(copy_state(ck[sg], work[cur], n, es, s), "rsol_gradient: checkpoint");
            RSOL_TRY_CUDA(cudaMemcpyAsync(ck_w[sg], work_w[cur], size_t(n) * es, cudaMemcpyDeviceToDevice, s),
                          "rsol_gradient: checkpoint weights");
        }
        RSOL_TRY(fields_at(step, true));
        rsol_particles W = as_particles(work[cur], n, work_w[cur]);
        RSOL_TRY(rsol_push_gather(ctx, &W, F, g->dt, d_feedback, stream));
    }
    RSOL_TRY(rsol_loss_norm(ctx, d_feedback, d_loss, stream));

    // reverse sweep
    int ab = 0;  // which adjoint set holds the current segment's order
    for (int a = 0; a < 3; ++a) {
        RSOL_TRY_CUDA(cudaMemsetAsync(xb[ab][a], 0, size_t(n) * es, s), "rsol_gradient: zero xbar");
        RSOL_TRY_CUDA(cudaMemsetAsync(ub[ab][a], 0, size_t(n) * es, s), "rsol_gradient: zero ubar");
    }
    RSOL_TRY_CUDA(cudaMemsetAsync(d_field_bar, 0, grid_bytes, s), "rsol_gradient: zero field_bar");
    if (use_modes) {
        RSOL_TRY_CUDA(cudaMemsetAsync(fbar_step, 0, grid_bytes, s), "rsol_gradient: zero step field_bar");
        RSOL_TRY_CUDA(cudaMemsetAsync(amp, 0, n_modes * sizeof(double), s), "rsol_gradient: zero amp_bar");
    }
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int n0 = sg * k;
        const int len = (g->steps - n0) < k ? (g->steps - n0) : k;
        seg[0] = ck[sg];
        for (int i = 1; i < len; ++i) {
            RSOL_TRY_CUDA(copy_state(seg[i], seg[i - 1], n, es, s), "rsol_gradient: segment copy");
            RSOL_TRY(fields_at(n0 + i - 1, false));
            rsol_particles Q = as_particles(seg[i], n, ck_w[sg]);
            RSOL_TRY(rsol_push_gather(ctx, &Q, F, g->dt, nullptr, stream));
        }
        for (int i = len - 1; i >= 0; --i) {
            RSOL_TRY(fields_at(n0 + i, false));
            rsol_particles Q = as_particles(seg[i], n, ck_w[sg]);
            RSOL_TRY(adjoint_launch(ctx, &Q, F, g->dt, d_feedback, d_loss, xb[ab], ub[ab],
                                    use_modes ? fbar_step : d_field_bar, bstart[sg], stream));
            if (use_modes)
                RSOL_TRY(rsol_alfven_adjoint(ctx, g->h_modes, g->h_sigma, g->n_modes,
                                             g->t0 + (n0 + i) * g->dt, g->B0, g->vA, g->h_u_gas,
                                             fbar_step, d_field_bar, amp, stream));
        }
        if (sg > 0) {
            // into the previous segment's packet order
            RSOL_TRY_CUDA(rsol::unpermute6(n, es, perm[sg], xb[ab], ub[ab], xb[ab ^ 1], ub[ab ^ 1], ctx->sm_count, s),
                          "rsol_gradient: unpermute adjoints");
            ctx->launches += 1;
            ab ^= 1;
        }
    }
#undef RSOL_TRY
#undef RSOL_TRY_CUDA
    release();
    return RSOL_OK;
}

} // extern "C"
