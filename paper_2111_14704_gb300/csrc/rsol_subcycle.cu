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

rsol_status rsol_sort_push_subcycled(rsol_ctx *ctx, const rsol_particles *in, rsol_particles *out,
                                     const void *d_fields, double dt, const rsol_subcycle_desc *sd,
                                     void *d_feedback, int64_t *h_level_counts, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, in, "rsol_sort_push_subcycled(in)");
    if (st != RSOL_OK || (st = check_particles(ctx, out, "rsol_sort_push_subcycled(out)")) != RSOL_OK)
        return st;
    if (in->n != out->n)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_sort_push_subcycled: in.n != out.n");
    {
        const void *a[8] = {in->cell, in->off[0], in->off[1], in->off[2], in->u[0], in->u[1], in->u[2], in->w};
        const void *b[8] = {out->cell, out->off[0], out->off[1], out->off[2], out->u[0], out->u[1], out->u[2], out->w};
        if (in->n > 0)
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j)
                    if (a[i] == b[j])
                        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_sort_push_subcycled: in and out share an array");
    }
    if (!sd || !(std::isfinite(sd->courant) && sd->courant > 0 && sd->courant <= 1) ||
        !(std::isfinite(sd->sigma_nn) && sd->sigma_nn >= 0) || sd->max_level < 0 ||
        sd->max_level > kMaxLevels || sd->reserved != 0)
        return fail(ctx, RSOL_ERR_INVALID_ARG,
                    "rsol_sort_push_subcycled: need 0 < courant <= 1, sigma_nn >= 0, 0 <= max_level <= 16");
    if (!(std::isfinite(dt) && dt > 0))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_sort_push_subcycled: dt must be finite and > 0");
    if (!d_fields || !aligned16(d_fields) || !d_feedback || !aligned16(d_feedback))
        return fail(ctx, RSOL_ERR_INVALID_ARG,
                    "rsol_sort_push_subcycled: fields and feedback required, 16-byte aligned");
    if (ctx->bin != 4 && ctx->bin != 8)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_sort_push_subcycled: the context's bin must be 4 or 8");
    const double adv = dt * ctx->p.c_tilde / ctx->p.dx;
    if (adv > 1.0)
        return fail(ctx, RSOL_ERR_COURANT,
                    "rsol_sort_push_subcycled: c~ dt / dx = %g > 1 (the tiles' halo covers one cell of drift)", adv);
    int lb = 0;
    while ((1 << lb) < ctx->bin)
        ++lb;
    const int64_t nbins = ctx->nbins;
    const int64_t nbins_total = nbins * (sd->max_level + 1);
    int key_bits = 0;
    while ((int64_t(1) << key_bits) < (nbins_total << (3 * lb)))
        ++key_bits;
    if (key_bits > 31)
        return fail(ctx, RSOL_ERR_INVALID_ARG,
                    "rsol_sort_push_subcycled: %d levels x %lld bins do not fit a 31-bit key",
                    sd->max_level + 1, (long long)nbins);
    if (in->n == 0) {
        if (h_level_counts)
            for (int k = 0; k <= sd->max_level; ++k)
                h_level_counts[k] = 0;
        return RSOL_OK;
    }
    const int64_t n = in->n;
    const int es = elem_bytes(ctx);
    const size_t need = rsol::sort_scratch_bytes(n, nbins_total);
    if ((st = ensure_buffer(ctx, &ctx->sub_mem, &ctx->sub_bytes, need, "sub-cycling scratch")) != RSOL_OK)
        return st;
    const bool det = ctx->p.deterministic != 0;
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
    rsol::SortScratch ss;
    rsol::sort_scratch_carve(base, n, nbins_total, &ss);
    if (ctx->sorted_cell == out->cell)
        ctx->sorted_cell = nullptr;  // out is about to hold a different order

    rsol::SubDesc s{};
    s.courant = sd->courant;
    s.k_gyro = (ctx->p.c_tilde / ctx->p.c) * std::fabs(ctx->p.q_over_m) / ctx->p.c;
    s.k_cross = ctx->p.dx / ctx->p.c_tilde;
    s.k_loss = sd->sigma_nn > 0 ? 1.0 / ((ctx->p.c_tilde / ctx->p.c) * sd->sigma_nn * ctx->p.c) : 0.0;
    s.dt = dt;
    s.max_level = sd->max_level;
    rsol::PushDesc d{};
    d.n = n;
    d.cell = in->cell;
    for (int a = 0; a < 3; ++a) {
        d.off[a] = in->off[a];
        d.u[a] = in->u[a];
    }
    d.w = in->w;
    d.fields = d_fields;
    d.nx = ctx->p.nx;
    d.ny = ctx->p.ny;
    d.nz = ctx->p.nz;
    d.shape = ctx->p.shape;
    d.status = ctx->d_status;
    d.sm_count = ctx->sm_count;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = ctx->p.precision == 32
                        ? rsol::level_keys_f32(d, s, lb, ctx->nbx, ctx->nby, uint32_t(nbins), ss.keys[0], cs)
                        : rsol::level_keys_f64(d, s, lb, ctx->nbx, ctx->nby, uint32_t(nbins), ss.keys[0], cs);
    if (e == cudaSuccess)
        e = rsol::sort_from_keys(ss, n, es, in->cell, in->off, in->u, in->w, out->cell, out->off, out->u,
                                 out->w, lb, key_bits, nbins_total, cs);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_sort_push_subcycled: level sort");
    ctx->launches += 2 + 4 * ((key_bits + 7) / 8);

    // packets per level: the level ranks' first bins, read back once
    uint32_t starts[kMaxLevels + 2];
    e = cudaMemcpy2DAsync(starts, sizeof(uint32_t), ss.bin_start, size_t(nbins) * sizeof(uint32_t),
                          sizeof(uint32_t), size_t(sd->max_level + 2), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_sort_push_subcycled: level counts");
    int64_t count[kMaxLevels + 1];
    int top = -1;  // highest level present
    for (int k = 0; k <= sd->max_level; ++k) {
        const int r = sd->max_level - k;
        count[k] = int64_t(starts[r + 1]) - int64_t(starts[r]);
        if (count[k] > 0 && k > top)
            top = k;
        if (h_level_counts)
            h_level_counts[k] = count[k];
    }
    if (top < 0)
        return RSOL_OK;

    // level k's packets are the bins of rank r0 + (top - k), r0 = max_level - top
    const double h = (ctx->p.c_tilde / ctx->p.c) * (ctx->p.q_over_m / ctx->p.c) * dt / 2.0;
    const double qv = ctx->p.q / (ctx->p.dx * ctx->p.dx * ctx->p.dx);
    const int r0 = sd->max_level - top;

    rsol::PushDesc b{};
    b.n = n;
    b.cell = out->cell;
    for (int a = 0; a < 3; ++a) {
        b.off[a] = out->off[a];
        b.u[a] = out->u[a];
    }
    b.w = out->w;
    b.fields = d_fields;
    b.fb = d_feedback;
    b.fx = det ? ctx->fx : nullptr;
    b.nx = ctx->p.nx;
    b.ny = ctx->p.ny;
    b.nz = ctx->p.nz;
    b.shape = ctx->p.shape;
    b.det = det ? 1 : 0;
    b.h = h;
    b.adv = adv;
    b.qv = qv;
    b.c = ctx->p.c;
    b.fx_scale = ctx->fx_scale;
    b.status = ctx->d_status;
    b.sm_count = ctx->sm_count;
    b.bin = ctx->bin;
    b.nbx = ctx->nbx;
    b.nby = ctx->nby;
    b.nbz = ctx->nbz;
    b.tile_mode = 1;
    b.warps = ctx->p.warps;
    b.perm = ss.keys[0];  // free once the level sort has gathered the packets
    // sub-step s of the finest level: level k moves when s is a multiple of
    // 2^(top - k), i.e. the levels top .. top - ctz(s) (all at s = 0).  Each
    // moving level is one binned push over its own bins, with h, adv and the
    // deposit scaled by 2^-k; the levels are disjoint packet sets sharing the
    // grids, so their launches commute.
    const long n_sub = 1L << top;
    for (long sub = 0; sub < n_sub; ++sub) {
        int kmin = 0;
        if (sub > 0) {
            int z = 0;
            while (((sub >> z) & 1L) == 0)
                ++z;
            kmin = top - z > 0 ? top - z : 0;
        }
        for (int k = top; k >= kmin; --k) {
            if (count[k] == 0)
                continue;
            const double sc = std::ldexp(1.0, -k);
            rsol::PushDesc dk = b;
            dk.h = h * sc;
            dk.adv = adv * sc;
            dk.qv = qv * sc;
            dk.bin_start = ss.bin_start + int64_t(r0 + (top - k)) * nbins;
            e = ctx->p.precision == 32 ? rsol::push_f32(dk, cs) : rsol::push_f64(dk, cs);
            if (e != cudaSuccess)
                return cuda_fail(ctx, e, "rsol_sort_push_subcycled: sub-step launch");
            ctx->launches += 1;
        }
    }
    if (det) {
        e = ctx->p.precision == 32
                ? rsol::fixed_to_grid_f32(ctx->fx, d_feedback, n_nodes(ctx) * 8, 1.0 / ctx->fx_scale,
                                          ctx->sm_count, cs)
                : rsol::fixed_to_grid_f64(ctx->fx, d_feedback, n_nodes(ctx) * 8, 1.0 / ctx->fx_scale,
                                          ctx->sm_count, cs);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "rsol_sort_push_subcycled fixed-point flush");
        ctx->launches += 1;
    }
    return RSOL_OK;
}

} // extern "C"
