// C-ABI layer of librsol: argument validation, context scratch, launches.
// Declarations and the contract of every entry point are in include/rsol.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "../../include/rsol.h"
#include "rsol_device.cuh"
#include "rsol_internal.h"

#include "rsol_ctx.h"

using namespace rsol_api;

namespace {

rsol_status ensure_fx(rsol_ctx *ctx)
{
    const size_t need = size_t(ctx->p.nx) * ctx->p.ny * ctx->p.nz * 8 * sizeof(long long);
    if (ctx->fx_bytes >= need)
        return RSOL_OK;
    if (ctx->fx)
        cudaFree(ctx->fx);
    ctx->fx = nullptr;
    ctx->fx_bytes = 0;
    if (cudaMalloc(&ctx->fx, need) != cudaSuccess)
        return fail(ctx, RSOL_ERR_OOM, "deterministic accumulators: cudaMalloc(%zu) failed", need);
    cudaError_t e = cudaMemset(ctx->fx, 0, need);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMemset");
    ctx->fx_bytes = need;
    return RSOL_OK;
}

rsol_status ensure_sort(rsol_ctx *ctx, int64_t n)
{
    if (ctx->sort_mem && ctx->sort.capacity >= n)
        return RSOL_OK;
    const size_t need = rsol::sort_scratch_bytes(n, ctx->nbins);
    if (ctx->sort_mem)
        cudaFree(ctx->sort_mem);
    ctx->sort_mem = nullptr;
    ctx->sort_bytes = 0;
    if (cudaMalloc(&ctx->sort_mem, need) != cudaSuccess)
        return fail(ctx, RSOL_ERR_OOM, "sort scratch: cudaMalloc(%zu) failed", need);
    ctx->sort_bytes = need;
    rsol::sort_scratch_carve(ctx->sort_mem, n, ctx->nbins, &ctx->sort);
    return RSOL_OK;
}

} // namespace

extern "C" {

rsol_status rsol_init(const rsol_params *p, rsol_ctx **out)
{
    if (!out)
        return RSOL_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p)
        return RSOL_ERR_INVALID_ARG;
    const bool grid_ok = p->nx >= 2 && p->ny >= 2 && p->nz >= 2 && p->nx <= 1024 &&
                         p->ny <= 1024 && p->nz <= 1024;
    const int bin = p->bin == 0 ? (p->precision == 32 ? 8 : 4) : p->bin;
    const bool bin_ok = bin == 1 || bin == 2 || bin == 4 || bin == 8 || bin == 16;
    const bool phys_ok = std::isfinite(p->dx) && p->dx > 0 && std::isfinite(p->c) && p->c > 0 &&
                         std::isfinite(p->c_tilde) && p->c_tilde > 0 && p->c_tilde <= p->c &&
                         std::isfinite(p->q_over_m) && p->q_over_m != 0 && std::isfinite(p->q) &&
                         p->q != 0;
    if (!grid_ok || !(p->shape == 1 || p->shape == 2) ||
        !(p->precision == 32 || p->precision == 64) || !(p->deterministic == 0 || p->deterministic == 1) ||
        !bin_ok || !(p->warps == 0 || p->warps == 8 || p->warps == 16) || !phys_ok)
        return RSOL_ERR_INVALID_ARG;
    rsol_ctx *ctx = new (std::nothrow) rsol_ctx();
    if (!ctx)
        return RSOL_ERR_OOM;
    ctx->p = *p;
    ctx->bin = bin;
    ctx->nbx = (p->nx + bin - 1) / bin;
    ctx->nby = (p->ny + bin - 1) / bin;
    ctx->nbz = (p->nz + bin - 1) / bin;
    ctx->nbins = int64_t(ctx->nbx) * ctx->nby * ctx->nbz;
    const int64_t nkeys = ctx->nbins * bin * bin * bin;
    int bits = 0;
    while ((int64_t(1) << bits) < nkeys)
        ++bits;
    ctx->key_bits = bits;
    ctx->fx_scale = std::ldexp(1.0, p->precision == 32 ? 32 : 40);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->d_status, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->d_totals, sizeof(double) * (16 + 16 * TOTALS_BLOCKS));
    if (e != cudaSuccess) {
        rsol_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? RSOL_ERR_OOM : RSOL_ERR_CUDA;
    }
    ctx->d_partials = ctx->d_totals + 16;
    *out = ctx;
    return RSOL_OK;
}

rsol_status rsol_destroy(rsol_ctx *ctx)
{
    if (!ctx)
        return RSOL_OK;
    if (ctx->d_status)
        cudaFree(ctx->d_status);
    if (ctx->d_totals)
        cudaFree(ctx->d_totals);
    if (ctx->sort_mem)
        cudaFree(ctx->sort_mem);
    if (ctx->fx)
        cudaFree(ctx->fx);
    if (ctx->field_mem)
        cudaFree(ctx->field_mem);
    if (ctx->grad_mem)
        cudaFree(ctx->grad_mem);
    if (ctx->sub_mem)
        cudaFree(ctx->sub_mem);
    if (ctx->count_mem)
        cudaFree(ctx->count_mem);
    delete ctx;
    return RSOL_OK;
}

const char *rsol_last_error(const rsol_ctx *ctx) { return ctx ? ctx->err : "no context"; }

rsol_status rsol_push_gather(rsol_ctx *ctx, const rsol_particles *P, const void *d_fields,
                             double dt, void *d_feedback, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, P, "rsol_push_gather");
    if (st != RSOL_OK)
        return st;
    if (!(std::isfinite(dt) && dt > 0))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_push_gather: dt must be finite and > 0");
    if (!d_fields || !aligned16(d_fields))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_push_gather: fields NULL or not 16-byte aligned");
    if (d_feedback && !aligned16(d_feedback))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_push_gather: feedback not 16-byte aligned");
    const double adv = dt * ctx->p.c_tilde / ctx->p.dx;
    if (adv > 1.0)
        return fail(ctx, RSOL_ERR_COURANT,
                    "rsol_push_gather: c~ dt / dx = %g > 1 (a packet could cross more than one cell)", adv);
    if (P->n == 0)
        return RSOL_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool det = ctx->p.deterministic && d_feedback;
    if (det && (st = ensure_fx(ctx)) != RSOL_OK)
        return st;
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
    d.tile_mode = 0;
    d.bin_start = nullptr;
    d.bin = ctx->bin;
    d.warps = ctx->p.warps;
    d.nbx = ctx->nbx;
    d.nby = ctx->nby;
    d.nbz = ctx->nbz;
    if (ctx->sorted_cell == P->cell && ctx->sorted_n == P->n) {
        d.bin_start = ctx->sort.bin_start;
        d.tile_mode = 1;
        d.perm = ctx->sort.keys[0];  // the sort's key buffer is free until the next sort
    }
    cudaError_t e = ctx->p.precision == 32 ? rsol::push_f32(d, s) : rsol::push_f64(d, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_push_gather launch");
    ctx->launches += 1 + (det ? 1 : 0);
    if (det) {
        e = ctx->p.precision == 32
                ? rsol::fixed_to_grid_f32(ctx->fx, d_feedback, n_nodes(ctx) * 8, 1.0 / ctx->fx_scale,
                                          ctx->sm_count, s)
                : rsol::fixed_to_grid_f64(ctx->fx, d_feedback, n_nodes(ctx) * 8, 1.0 / ctx->fx_scale,
                                          ctx->sm_count, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "rsol_push_gather fixed-point flush");
    }
    return RSOL_OK;
}

rsol_status rsol_deposit(rsol_ctx *ctx, const rsol_particles *P, void *d_moments, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, P, "rsol_deposit");
    if (st != RSOL_OK)
        return st;
    if (!d_moments || !aligned16(d_moments))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_deposit: moments NULL or not 16-byte aligned");
    if (P->n == 0)
        return RSOL_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool det = ctx->p.deterministic != 0;
    if (det && (st = ensure_fx(ctx)) != RSOL_OK)
        return st;
    const double m = ctx->p.q / ctx->p.q_over_m;
    rsol::MomentsDesc d{};
    d.n = P->n;
    d.cell = P->cell;
    for (int a = 0; a < 3; ++a) {
        d.off[a] = P->off[a];
        d.u[a] = P->u[a];
    }
    d.w = P->w;
    d.grid = d_moments;
    d.fx = det ? ctx->fx : nullptr;
    d.nx = ctx->p.nx;
    d.ny = ctx->p.ny;
    d.nz = ctx->p.nz;
    d.shape = ctx->p.shape;
    d.det = det ? 1 : 0;
    d.inv_vol = 1.0 / (ctx->p.dx * ctx->p.dx * ctx->p.dx);
    d.mc = m * ctx->p.c;
    d.mc2 = m * ctx->p.c * ctx->p.c;
    d.qc = ctx->p.q * ctx->p.c;
    d.fx_scale = ctx->fx_scale;
    d.sm_count = ctx->sm_count;
    if (ctx->sorted_cell == P->cell && ctx->sorted_n == P->n) {
        d.bin_start = ctx->sort.bin_start;  // tiles per sort bin
        d.bin = ctx->bin;
        d.nbx = ctx->nbx;
        d.nby = ctx->nby;
        d.nbz = ctx->nbz;
    }
    cudaError_t e = ctx->p.precision == 32 ? rsol::moments_grid_f32(d, s) : rsol::moments_grid_f64(d, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_deposit launch");
    ctx->launches += 1 + (det ? 1 : 0);
    if (det) {
        e = ctx->p.precision == 32
                ? rsol::fixed_to_grid_f32(ctx->fx, d_moments, n_nodes(ctx) * 8, 1.0 / ctx->fx_scale,
                                          ctx->sm_count, s)
                : rsol::fixed_to_grid_f64(ctx->fx, d_moments, n_nodes(ctx) * 8, 1.0 / ctx->fx_scale,
                                          ctx->sm_count, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "rsol_deposit fixed-point flush");
    }
    return RSOL_OK;
}

rsol_status rsol_sort(rsol_ctx *ctx, const rsol_particles *in, rsol_particles *out, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, in, "rsol_sort(in)");
    if (st != RSOL_OK)
        return st;
    if ((st = check_particles(ctx, out, "rsol_sort(out)")) != RSOL_OK)
        return st;
    if (in->n != out->n)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_sort: in.n != out.n");
    const void *a[8] = {in->cell, in->off[0], in->off[1], in->off[2], in->u[0], in->u[1], in->u[2], in->w};
    const void *b[8] = {out->cell, out->off[0], out->off[1], out->off[2], out->u[0], out->u[1], out->u[2], out->w};
    if (in->n > 0)
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j)
                if (a[i] == b[j])
                    return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_sort: in and out share an array");
    if ((st = ensure_sort(ctx, in->n > 0 ? in->n : 1)) != RSOL_OK)
        return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nkeys = ctx->nbins * ctx->bin * ctx->bin * ctx->bin;
    const bool counting = rsol::count_sort_applies(in->n, nkeys);
    if (counting) {
        const size_t need = rsol::count_scratch_bytes(in->n, nkeys);
        if ((st = ensure_buffer(ctx, &ctx->count_mem, &ctx->count_bytes, need, "rsol_sort")) != RSOL_OK)
            return st;
        rsol::count_scratch_carve(ctx->count_mem, in->n, nkeys, &ctx->count);
    }
    const int passes = (ctx->key_bits + 7) / 8;
    cudaError_t e =
        counting ? rsol::count_sort_particles(ctx->sort, ctx->count, in->n, elem_bytes(ctx), in->cell,
                                              in->off, in->u, in->w, out->cell, out->off, out->u,
                                              out->w, ctx->p.nx, ctx->p.ny, ctx->p.nz, ctx->bin,
                                              ctx->p.shape, ctx->key_bits, ctx->nbins, s)
                 : rsol::sort_particles(ctx->sort, in->n, elem_bytes(ctx), in->cell, in->off, in->u,
                                        in->w, out->cell, out->off, out->u, out->w, ctx->p.nx,
                                        ctx->p.ny, ctx->p.nz, ctx->bin, ctx->p.shape, ctx->key_bits,
                                        ctx->nbins, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_sort launch");
    ctx->launches += in->n > 0 ? (counting ? rsol::count_sort_launches(nkeys) : 2 + 4 * passes) : 0;
    ctx->sorted_cell = out->cell;
    ctx->sorted_n = out->n;
    return RSOL_OK;
}

rsol_status rsol_moments(rsol_ctx *ctx, const rsol_particles *P, const void *d_feedback,
                         double *h_totals, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, P, "rsol_moments");
    if (st != RSOL_OK)
        return st;
    if (!h_totals)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_moments: h_totals is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double m = ctx->p.q / ctx->p.q_over_m;
    rsol::TotalsDesc d{};
    d.n = P->n;
    for (int a = 0; a < 3; ++a)
        d.u[a] = P->u[a];
    d.w = P->w;
    d.fb = d_feedback;
    d.n_nodes = n_nodes(ctx);
    d.mc = m * ctx->p.c;
    d.mc2 = m * ctx->p.c * ctx->p.c;
    d.qc = ctx->p.q * ctx->p.c;
    d.vol = ctx->p.dx * ctx->p.dx * ctx->p.dx;
    d.partials = ctx->d_partials;
    d.out = ctx->d_totals;
    d.blocks = TOTALS_BLOCKS;
    cudaError_t e = ctx->p.precision == 32 ? rsol::totals_f32(d, s) : rsol::totals_f64(d, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_moments launch");
    ctx->launches += 2;
    e = cudaMemcpyAsync(h_totals, ctx->d_totals, 16 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_moments copy");
    return RSOL_OK;
}

rsol_status rsol_alfven_fields(rsol_ctx *ctx, const double *h_modes, const double *h_sigma,
                               int32_t n_modes, double t, double B0, double vA,
                               const double *h_u_gas, void *d_fields, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    if (n_modes < 0 || n_modes > 256 || (n_modes > 0 && (!h_modes || !h_sigma)) || !h_u_gas)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_alfven_fields: bad mode arrays");
    if (!d_fields || !aligned16(d_fields))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_alfven_fields: fields NULL or not aligned");
    if (!(std::isfinite(B0) && B0 != 0 && std::isfinite(vA) && std::isfinite(t)))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_alfven_fields: B0, vA, t must be finite, B0 != 0");
    const size_t need = rsol::alfven_scratch_bytes(ctx->p.nx, ctx->p.ny, ctx->p.nz, n_modes > 0 ? n_modes : 1);
    if (ctx->field_bytes < need) {
        if (ctx->field_mem)
            cudaFree(ctx->field_mem);
        ctx->field_mem = nullptr;
        ctx->field_bytes = 0;
        if (cudaMalloc(&ctx->field_mem, need) != cudaSuccess)
            return fail(ctx, RSOL_ERR_OOM, "field scratch: cudaMalloc(%zu) failed", need);
        ctx->field_bytes = need;
    }
    cudaError_t e = rsol::alfven_fields(h_modes, h_sigma, n_modes, t, B0, vA, h_u_gas, ctx->p.c,
                                        ctx->p.dx, ctx->p.nx, ctx->p.ny, ctx->p.nz, ctx->p.precision,
                                        d_fields, ctx->field_mem, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_alfven_fields launch");
    ctx->launches += 2;
    return RSOL_OK;
}

rsol_status rsol_losses(rsol_ctx *ctx, const rsol_particles *P, const void *d_nn,
                        double nn_uniform, double sigma, double dt, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_particles(ctx, P, "rsol_losses");
    if (st != RSOL_OK)
        return st;
    if (!(std::isfinite(dt) && dt > 0) || !(std::isfinite(sigma) && sigma >= 0) ||
        !(std::isfinite(nn_uniform) && nn_uniform >= 0))
        return fail(ctx, RSOL_ERR_INVALID_ARG, "rsol_losses: dt > 0, sigma >= 0, n_n >= 0 required");
    if (P->n == 0)
        return RSOL_OK;
    rsol::LossDesc d{};
    d.n = P->n;
    d.cell = P->cell;
    for (int a = 0; a < 3; ++a) {
        d.off[a] = P->off[a];
        d.u[a] = P->u[a];
    }
    d.w = P->w;
    d.nn = d_nn;
    d.nn_uniform = nn_uniform;
    d.coef = (ctx->p.c_tilde / ctx->p.c) * sigma * ctx->p.c * dt;
    d.nx = ctx->p.nx;
    d.ny = ctx->p.ny;
    d.nz = ctx->p.nz;
    d.shape = ctx->p.shape;
    d.status = ctx->d_status;
    d.sm_count = ctx->sm_count;
    if (ctx->sorted_cell == P->cell && ctx->sorted_n == P->n) {
        d.bin_start = ctx->sort.bin_start;  // n_n tiles per sort bin
        d.bin = ctx->bin;
        d.nbx = ctx->nbx;
        d.nby = ctx->nby;
        d.nbz = ctx->nbz;
    }
    cudaError_t e = ctx->p.precision == 32 ? rsol::losses_f32(d, static_cast<cudaStream_t>(stream))
                                           : rsol::losses_f64(d, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_losses launch");
    ctx->launches += 1;
    return RSOL_OK;
}

rsol_status rsol_check(rsol_ctx *ctx, void *stream)
{
    if (!ctx)
        return RSOL_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "rsol_check");
    if (h & rsol::ST_NONFINITE)
        return fail(ctx, RSOL_ERR_NONFINITE, "a packet momentum or position became non-finite");
    if (h & rsol::ST_COURANT)
        return fail(ctx, RSOL_ERR_COURANT, "a packet moved more than one cell in one step");
    if (h & rsol::ST_TIMEOUT)
        return fail(ctx, RSOL_ERR_TIMEOUT, "a bounded device wait ran out");
    if (h & rsol::ST_BADCELL)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "a packet's cell index lies off the grid (skipped)");
    return RSOL_OK;
}

int64_t rsol_kernel_launches(const rsol_ctx *ctx) { return ctx ? ctx->launches : -1; }

} // extern "C"
