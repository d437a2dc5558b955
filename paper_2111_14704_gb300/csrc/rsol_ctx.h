// Context object behind the opaque rsol_ctx handle of rsol.h, and the
// argument-checking helpers shared by the C-ABI translation units.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/rsol.h"
#include "rsol_internal.h"

struct rsol_ctx {
    rsol_params p;
    int device;
    int sm_count;
    int bin;
    int nbx, nby, nbz;
    int64_t nbins;
    int key_bits;
    char err[512];
    int *d_status;            // device status word
    double *d_totals;         // 16 doubles + partials
    double *d_partials;
    // sort scratch (grown on demand)
    void *sort_mem;
    size_t sort_bytes;
    rsol::SortScratch sort;
    const uint32_t *sorted_cell; // identity of the set the last sort wrote
    int64_t sorted_n;
    // counting-sort scratch (allocated on first use)
    void *count_mem;
    size_t count_bytes;
    rsol::CountScratch count;
    // deterministic-mode fixed-point grid
    long long *fx;
    size_t fx_bytes;
    double fx_scale;
    // field-source scratch
    void *field_mem;
    size_t field_bytes;
    int64_t launches;         // kernels launched through this context
    // differentiable run (rsol_gradient): checkpoints, segment states, adjoints
    void *grad_mem;
    size_t grad_bytes;
    // sub-cycled push: per-packet levels, level-major order, level counts
    void *sub_mem;
    size_t sub_bytes;
};


namespace rsol_api {


constexpr int TOTALS_BLOCKS = 1024;

inline rsol_status fail(rsol_ctx *ctx, rsol_status st, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

inline rsol_status cuda_fail(rsol_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, RSOL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline int elem_bytes(const rsol_ctx *ctx) { return ctx->p.precision == 32 ? 4 : 8; }

inline rsol_status check_particles(rsol_ctx *ctx, const rsol_particles *P, const char *name)
{
    if (!P)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "%s: particle set is NULL", name);
    if (P->n < 0 || P->n > int64_t(0xFFFFFFFFll) - 1)
        return fail(ctx, RSOL_ERR_INVALID_ARG, "%s: n = %lld out of range", name, (long long)P->n);
    if (P->n == 0)
        return RSOL_OK;
    const void *ptrs[8] = {P->cell, P->off[0], P->off[1], P->off[2], P->u[0], P->u[1], P->u[2], P->w};
    for (int i = 0; i < 8; ++i) {
        if (!ptrs[i])
            return fail(ctx, RSOL_ERR_INVALID_ARG, "%s: particle array %d is NULL", name, i);
        if (!aligned16(ptrs[i]))
            return fail(ctx, RSOL_ERR_INVALID_ARG, "%s: particle array %d not 16-byte aligned", name, i);
    }
    return RSOL_OK;
}

inline int64_t n_nodes(const rsol_ctx *ctx) { return int64_t(ctx->p.nx) * ctx->p.ny * ctx->p.nz; }

} // namespace rsol_api

namespace rsol_api {

// Grow-only device buffer owned by the context.
inline rsol_status ensure_buffer(rsol_ctx *ctx, void **mem, size_t *bytes, size_t need, const char *what)
{
    if (*bytes >= need && *mem)
        return RSOL_OK;
    if (*mem)
        cudaFree(*mem);
    *mem = nullptr;
    *bytes = 0;
    if (cudaMalloc(mem, need) != cudaSuccess)
        return fail(ctx, RSOL_ERR_OOM, "%s: cudaMalloc(%zu) failed", what, need);
    *bytes = need;
    return RSOL_OK;
}

} // namespace rsol_api
