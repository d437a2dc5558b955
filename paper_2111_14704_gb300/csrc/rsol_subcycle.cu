// C-ABI layer of the sub-cycled push (contract in include/rsol.h).
#include <cmath>

#include <cuda_runtime.h>

#include "../../include/rsol.h"
#include "rsol_ctx.h"
#include "rsol_internal.h"

using namespace rsol_api;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kMaxLevels = 16;

} // namespace

extern "C" {

rsol_status rsol_push_subcycled(rsol_ctx *ctx, const rsol_particles *P, const void *d_fields,
                                double dt, const rsol_subcycle_desc *sd, void *d_feedback,
                                uint8_t *d_levels, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, P, "rsol_push_subcycled");
    if (st != RSOL_OK)
        return st;
    if (!sd || !(std::isfinite(sd->courant) && sd->courant > 0 && sd->courant <= 1) ||
        !(std::isfinite(sd->sigma_nn) && sd->sigma_nn >= 0) || sd->max_level < 0 ||
        sd->max_level > kMaxLevels || sd->reserved != 0)
        return fail(ctx, RSOL_ERR_INVALID_ARG,
                    "rsol_push_subcycled: need 0 < courant <= 1, sigma_nn >= 0, 0 <= max_level <= 16");
    if (!(std::isfinite(dt) && dt > 0))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_push_subcycled: dt must be finite and > 0");
    if (!d_fields || !aligned16(d_fields) || (d_feedback && !aligned16(d_feedback)))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_push_subcycled: fields / feedback not 16-byte aligned");
    const double adv = dt * ctx->p.c_tilde / ctx->p.dx;
    if (std::ldexp(adv, -sd->max_level) > 1.0)
        return fail(ctx, RSOL_ERR_COURANT,
                    "rsol_push_subcycled: c~ dt / dx / 2^max_level = %g > 1", std::ldexp(adv, -sd->max_level));
    if (P->n == 0)
        return RSOL_OK;
    const size_t n = size_t(P->n);
    const size_t need = align256(n) + align256(n * 4) + align256(sizeof(uint32_t) * (kMaxLevels + 1));
    if ((st = ensure_buffer(ctx, &ctx->sub_mem, &ctx->sub_bytes, need, "sub-cycling scratch")) != RSOL_OK)
        return st;
    const bool det = ctx->p.deterministic && d_feedback;
    if (det) {
        const size_t fneed = size_t(n_nodes(ctx)) * 8 * sizeof(long long);
        if (ctx->fx_bytes < fneed) {
            void *mem = ctx->fx;
            size_t bytes = ctx->fx_bytes;
            if ((st = ensure_buffer(ctx, &mem, &bytes, fneed, "deterministic accumulators")) != RSOL_OK)
                return st;
            ctx->fx = static_cast<long long *>(mem);
            ctx->fx_bytes = bytes;
            cudaError_t e = cudaMemset(ctx->fx, 0, fneed);
            if (e != cudaSuccess)
                return cuda_fail(ctx, e, "cudaMemset");
        }
    }
    char *base = static_cast<char *>(ctx->sub_mem);
    rsol::SubDesc s{};
    s.level = d_levels ? d_levels : reinterpret_cast<uint8_t *>(base);
    s.order = reinterpret_cast<uint32_t *>(base + align256(n));
    s.counts = reinterpret_cast<uint32_t *>(base + align256(n) + align256(n * 4));
    s.courant = sd->courant;
    s.k_gyro = (ctx->p.c_tilde / ctx->p.c) * std::fabs(ctx->p.q_over_m) / ctx->p.c;
    s.k_cross = ctx->p.dx / ctx->p.c_tilde;
    s.k_loss = sd->sigma_nn > 0 ? 1.0 / ((ctx->p.c_tilde / ctx->p.c) * sd->sigma_nn * ctx->p.c) : 0.0;
    s.dt = dt;
    s.max_level = sd->max_level;

    rsol::PushDesc d{};
    d.n = P->n;
    d.cell = P->cell;
    for (int a = 0; a < 3; ++a) {
        d.off[a] = P->off[a];
        d.u[a] = P->u[a];
    }
    d.w = P->w;
    d.fields = d_fields;
    d.fb = d_feedback;
    d.fx = det ? ctx->fx : nullptr;
    d.nx = ctx->p.nx;
    d.ny = ctx->p.ny;
    d.nz = ctx->p.nz;
    d.shape = ctx->p.shape;
    d.det = det ? 1 : 0;
    d.h = (ctx->p.c_tilde / ctx->p.c) * (ctx->p.q_over_m / ctx->p.c) * dt / 2.0;
    d.adv = adv;
    d.qv = ctx->p.q / (ctx->p.dx * ctx->p.dx * ctx->p.dx);
    d.c = ctx->p.c;
    d.fx_scale = ctx->fx_scale;
    d.status = ctx->d_status;
    d.sm_count = ctx->sm_count;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = ctx->p.precision == 32 ? rsol::push_subcycled_f32(d, s, cs) : rsol::push_subcycled_f64(d, s, cs);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_push_subcycled launch");
    ctx->launches += 4;
    if (det) {
        e = ctx->p.precision == 32
                ? rsol::fixed_to_grid_f32(ctx->fx, d_feedback, n_nodes(ctx) * 8, 1.0 / ctx->fx_scale,
                                          ctx->sm_count, cs)
                : rsol::fixed_to_grid_f64(ctx->fx, d_feedback, n_nodes(ctx) * 8, 1.0 / ctx->fx_scale,
                                          ctx->sm_count, cs);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "rsol_push_subcycled fixed-point flush");
        ctx->launches += 1;
    }
    return RSOL_OK;
}

} // extern "C"
