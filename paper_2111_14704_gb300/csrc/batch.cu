// Batched boxes: many independent periodic boxes (own grid size, c~ and dt)
// advanced by two launches per step.  The packets of all boxes share one
// structure-of-arrays (box b owns packets offsets[b] .. offsets[b+1]); the
// grids of all boxes are concatenated node-major (box b's nodes start at
// node_off[b] = sum of the earlier boxes' nx*ny*nz).  A box-major cell key
// makes one stable sort order every box at once; the push then runs one warp
// per sparse bin (global gathers and atomics) and, persistently, the binned CTA
// body on every dense bin of every box.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rsol.h"
#include "rsol_device.cuh"
#include "rsol_internal.h"

struct rsol_batch_ctx {
    rsol_params p;
    int bin, n_boxes, device, sm_count, warps;
    std::vector<int> dims;
    std::vector<double> c_tilde, dt;
    std::vector<int64_t> offsets, node_off;
    std::vector<uint32_t> bin_base;
    int64_t total_nodes, total_packets;
    uint32_t total_bins;
    int key_bits;
    void *d_boxes;                    // BatchBox<T>[n_boxes]
    rsol::BatchKeyBox *d_keyboxes;    // [n_boxes]
    int64_t *d_offsets;               // [n_boxes + 1]
    void *sort_mem;
    rsol::SortScratch sort;
    void *count_mem;                  // counting-sort scratch when the key space allows one
    rsol::CountScratch count;
    uint32_t *d_work;                 // push: bin claim counters and the dense-bin list
    const uint32_t *sorted_cell;
    int64_t sorted_n;
    long long *fx;
    int *d_status;
    void *field_mem;
    size_t field_bytes;
    double fx_scale;
    char err[512];
};

namespace {

rsol_status bfail(rsol_batch_ctx *b, rsol_status st, const char *fmt, ...)
{
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

rsol_status check_set(rsol_batch_ctx *b, const rsol_particles *P, const char *name)
{
    if (!P)
        return bfail(b, RSOL_ERR_INVALID_ARG, "%s: particle set is NULL", name);
    if (P->n != b->total_packets)
        return bfail(b, RSOL_ERR_INVALID_ARG, "%s: n = %lld, the batch has %lld packets", name,
                     (long long)P->n, (long long)b->total_packets);
    if (P->n == 0)
        return RSOL_OK;
    const void *ptrs[8] = {P->cell, P->off[0], P->off[1], P->off[2], P->u[0], P->u[1], P->u[2], P->w};
    for (int i = 0; i < 8; ++i)
        if (!ptrs[i] || !aligned16(ptrs[i]))
            return bfail(b, RSOL_ERR_INVALID_ARG, "%s: array %d NULL or not 16-byte aligned", name, i);
    return RSOL_OK;
}

void release(rsol_batch_ctx *b)
{
    void *ptrs[] = {b->d_boxes, b->d_keyboxes, b->d_offsets, b->sort_mem, b->count_mem, b->d_work, b->fx,
                    b->d_status, b->field_mem};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
}

} // namespace

extern "C" {

rsol_status rsol_batch_init(const rsol_params *p, const rsol_batch_desc *desc, rsol_batch_ctx **out)
{
    if (!out)
        return RSOL_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p || !desc || desc->n_boxes < 1 || !desc->h_dims || !desc->h_c_tilde || !desc->h_dt ||
        !desc->h_offsets)
        return RSOL_ERR_INVALID_ARG;
    const int bin = p->bin == 0 ? (p->precision == 32 ? 8 : 4) : p->bin;
    if (!(p->shape == 1 || p->shape == 2) || !(p->precision == 32 || p->precision == 64) ||
        !(p->deterministic == 0 || p->deterministic == 1) || !(bin == 4 || bin == 8) ||
        !(std::isfinite(p->dx) && p->dx > 0 && std::isfinite(p->c) && p->c > 0 &&
          std::isfinite(p->q_over_m) && p->q_over_m != 0 && std::isfinite(p->q) && p->q != 0) ||
        !(desc->warps == 0 || desc->warps == 8 || desc->warps == 16))
        return RSOL_ERR_INVALID_ARG;
    rsol_batch_ctx *b = new (std::nothrow) rsol_batch_ctx();
    if (!b)
        return RSOL_ERR_OOM;
    b->p = *p;
    b->bin = bin;
    b->n_boxes = desc->n_boxes;
    b->warps = desc->warps == 0 ? 16 : desc->warps;
    b->fx_scale = std::ldexp(1.0, p->precision == 32 ? 32 : 40);
    b->offsets.assign(desc->h_offsets, desc->h_offsets + desc->n_boxes + 1);
    if (b->offsets[0] != 0) {
        delete b;
        return RSOL_ERR_INVALID_ARG;
    }
    int64_t nodes = 0;
    uint64_t bins = 0;
    std::vector<rsol::BatchKeyBox> kb(desc->n_boxes);
    std::vector<unsigned char> boxes(rsol::batch_box_size(p->precision) * desc->n_boxes);
    for (int i = 0; i < desc->n_boxes; ++i) {
        const int nx = desc->h_dims[3 * i], ny = desc->h_dims[3 * i + 1], nz = desc->h_dims[3 * i + 2];
        const double ct = desc->h_c_tilde[i], dt = desc->h_dt[i];
        const bool ok = nx >= 2 && ny >= 2 && nz >= 2 && nx <= 1024 && ny <= 1024 && nz <= 1024 &&
                        std::isfinite(ct) && ct > 0 && ct <= p->c && std::isfinite(dt) && dt > 0 &&
                        dt * ct / p->dx <= 1.0 && b->offsets[i + 1] >= b->offsets[i];
        if (!ok) {
            delete b;
            return RSOL_ERR_INVALID_ARG;
        }
        const int nbx = (nx + bin - 1) / bin, nby = (ny + bin - 1) / bin, nbz = (nz + bin - 1) / bin;
        b->dims.insert(b->dims.end(), {nx, ny, nz});
        b->c_tilde.push_back(ct);
        b->dt.push_back(dt);
        b->node_off.push_back(nodes);
        b->bin_base.push_back(uint32_t(bins));
        kb[i] = rsol::BatchKeyBox{nx, ny, nz, nbx, nby, uint32_t(bins)};
        const double h = (ct / p->c) * (p->q_over_m / p->c) * dt / 2.0;
        const double adv = dt * ct / p->dx;
        const double qv = p->q / (p->dx * p->dx * p->dx);
        void *dst = boxes.data() + rsol::batch_box_size(p->precision) * i;
        if (p->precision == 32)
            rsol::fill_batch_box_f32(dst, nx, ny, nz, nbx, nby, nbz, nodes, uint32_t(bins), h, adv, qv, p->c);
        else
            rsol::fill_batch_box_f64(dst, nx, ny, nz, nbx, nby, nbz, nodes, uint32_t(bins), h, adv, qv, p->c);
        nodes += int64_t(nx) * ny * nz;
        bins += uint64_t(nbx) * nby * nbz;
    }
    b->total_nodes = nodes;
    b->total_packets = b->offsets.back();
    int bits = 0;
    while ((uint64_t(1) << bits) < bins * uint64_t(bin) * bin * bin)
        ++bits;
    if (bits > 32 || b->total_packets > int64_t(0xFFFFFFFFll) - 1) {
        delete b;
        return RSOL_ERR_INVALID_ARG;
    }
    b->total_bins = uint32_t(bins);
    b->key_bits = bits;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_boxes, boxes.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_boxes, boxes.data(), boxes.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_keyboxes, sizeof(rsol::BatchKeyBox) * kb.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_keyboxes, kb.data(), sizeof(rsol::BatchKeyBox) * kb.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_offsets, sizeof(int64_t) * b->offsets.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_offsets, b->offsets.data(), sizeof(int64_t) * b->offsets.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_status, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemset(b->d_status, 0, sizeof(int));
    const int64_t nsort = b->total_packets > 0 ? b->total_packets : 1;
    if (e == cudaSuccess)
        e = cudaMalloc(&b->sort_mem, rsol::sort_scratch_bytes(nsort, b->total_bins));
    if (e == cudaSuccess)
        rsol::sort_scratch_carve(b->sort_mem, nsort, b->total_bins, &b->sort);
    // the counting sort by key where the box-major key space allows it (allocated
    // here, so that sorts captured in a CUDA graph allocate nothing)
    const int64_t nkeys = int64_t(bins) * bin * bin * bin;
    if (e == cudaSuccess && rsol::count_sort_applies(b->total_packets, nkeys)) {
        e = cudaMalloc(&b->count_mem, rsol::count_scratch_bytes(b->total_packets, nkeys));
        if (e == cudaSuccess)
            rsol::count_scratch_carve(b->count_mem, b->total_packets, nkeys, &b->count);
    }
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_work, rsol::batch_work_words(b->total_bins) * sizeof(uint32_t));
    if (e == cudaSuccess && p->deterministic) {
        e = cudaMalloc(&b->fx, size_t(b->total_nodes) * 8 * sizeof(long long));
        if (e == cudaSuccess)
            e = cudaMemset(b->fx, 0, size_t(b->total_nodes) * 8 * sizeof(long long));
    }
    if (e != cudaSuccess) {
        release(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? RSOL_ERR_OOM : RSOL_ERR_CUDA;
    }
    *out = b;
    return RSOL_OK;
}

rsol_status rsol_batch_destroy(rsol_batch_ctx *b)
{
    if (!b)
        return RSOL_OK;
    release(b);
    delete b;
    return RSOL_OK;
}

const char *rsol_batch_last_error(const rsol_batch_ctx *b) { return b ? b->err : "no context"; }

int64_t rsol_batch_total_nodes(const rsol_batch_ctx *b) { return b ? b->total_nodes : -1; }

rsol_status rsol_batch_sort(rsol_batch_ctx *b, const rsol_particles *in, rsol_particles *out,
                            void *stream)
{
    if (!b)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_set(b, in, "rsol_batch_sort(in)");
    if (st == RSOL_OK)
        st = check_set(b, out, "rsol_batch_sort(out)");
    if (st != RSOL_OK)
        return st;
    if (in->n > 0 && (in->cell == out->cell || in->w == out->w || in->u[0] == out->u[0]))
        return bfail(b, RSOL_ERR_INVALID_ARG, "rsol_batch_sort: in and out share arrays");
    const int eb = b->p.precision == 32 ? 4 : 8;
    const cudaError_t e =
        b->count_mem && in->n > 0
            ? rsol::count_sort_particles(b->sort, b->count, in->n, eb, in->cell, in->off, in->u, in->w,
                                         out->cell, out->off, out->u, out->w, 0, 0, 0, b->bin,
                                         b->p.shape, b->key_bits, b->total_bins,
                                         static_cast<cudaStream_t>(stream), b->d_offsets,
                                         b->d_keyboxes, b->n_boxes)
            : rsol::sort_particles_batch(b->sort, in->n, eb, in->cell, in->off, in->u, in->w,
                                         out->cell, out->off, out->u, out->w, b->d_offsets,
                                         b->d_keyboxes, b->n_boxes, b->bin, b->p.shape, b->key_bits,
                                         b->total_bins, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return bfail(b, RSOL_ERR_CUDA, "rsol_batch_sort: %s", cudaGetErrorString(e));
    b->sorted_cell = out->cell;
    b->sorted_n = out->n;
    return RSOL_OK;
}

rsol_status rsol_batch_push_gather(rsol_batch_ctx *b, const rsol_particles *P, const void *d_fields,
                                   void *d_feedback, void *stream)
{
    if (!b)
        return RSOL_ERR_INVALID_ARG;
    rsol_status st = check_set(b, P, "rsol_batch_push_gather");
    if (st != RSOL_OK)
        return st;
    if (!d_fields || !aligned16(d_fields) || !d_feedback || !aligned16(d_feedback))
        return bfail(b, RSOL_ERR_INVALID_ARG, "rsol_batch_push_gather: grids NULL or not aligned");
    if (P->n > 0 && !(b->sorted_cell == P->cell && b->sorted_n == P->n))
        return bfail(b, RSOL_ERR_UNSORTED,
                     "rsol_batch_push_gather: the packet set is not the one rsol_batch_sort wrote");
    if (P->n == 0)
        return RSOL_OK;
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
    d.fx = b->p.deterministic ? b->fx : nullptr;
    d.shape = b->p.shape;
    d.det = b->p.deterministic;
    d.fx_scale = b->fx_scale;
    d.status = b->d_status;
    d.sm_count = b->sm_count;
    d.bin_start = b->sort.bin_start;
    d.bin = b->bin;
    d.perm = b->sort.keys[0];  // the sort's key buffer is free until the next sort
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = b->p.precision == 32
                        ? rsol::push_batch_f32(d, b->d_boxes, b->n_boxes, b->total_bins, b->warps, b->d_work, s)
                        : rsol::push_batch_f64(d, b->d_boxes, b->n_boxes, b->total_bins, b->warps, b->d_work, s);
    if (e == cudaSuccess && b->p.deterministic)
        e = b->p.precision == 32
                ? rsol::fixed_to_grid_f32(b->fx, d_feedback, b->total_nodes * 8, 1.0 / b->fx_scale, b->sm_count, s)
                : rsol::fixed_to_grid_f64(b->fx, d_feedback, b->total_nodes * 8, 1.0 / b->fx_scale, b->sm_count, s);
    if (e != cudaSuccess)
        return bfail(b, RSOL_ERR_CUDA, "rsol_batch_push_gather: %s", cudaGetErrorString(e));
    return RSOL_OK;
}

rsol_status rsol_batch_alfven_fields(rsol_batch_ctx *b, int32_t box, const double *h_modes,
                                     const double *h_sigma, int32_t n_modes, double t, double B0,
                                     double vA, const double *h_u_gas, void *d_fields, void *stream)
{
    if (!b || box < 0 || box >= b->n_boxes || !d_fields || !aligned16(d_fields) || !h_u_gas ||
        n_modes < 0 || n_modes > 256 || (n_modes > 0 && (!h_modes || !h_sigma)) ||
        !(std::isfinite(B0) && B0 != 0 && std::isfinite(vA) && std::isfinite(t)))
        return bfail(b, RSOL_ERR_INVALID_ARG, "rsol_batch_alfven_fields: bad arguments");
    const int nx = b->dims[3 * box], ny = b->dims[3 * box + 1], nz = b->dims[3 * box + 2];
    const size_t need = rsol::alfven_scratch_bytes(nx, ny, nz, n_modes > 0 ? n_modes : 1);
    if (b->field_bytes < need) {
        if (b->field_mem)
            cudaFree(b->field_mem);
        b->field_mem = nullptr;
        b->field_bytes = 0;
        if (cudaMalloc(&b->field_mem, need) != cudaSuccess)
            return bfail(b, RSOL_ERR_OOM, "field scratch");
        b->field_bytes = need;
    }
    const size_t esz = b->p.precision == 32 ? 4 : 8;
    void *slice = static_cast<char *>(d_fields) + size_t(b->node_off[box]) * 8 * esz;
    const cudaError_t e = rsol::alfven_fields(h_modes, h_sigma, n_modes, t, B0, vA, h_u_gas, b->p.c,
                                              b->p.dx, nx, ny, nz, b->p.precision, slice,
                                              b->field_mem, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return bfail(b, RSOL_ERR_CUDA, "rsol_batch_alfven_fields: %s", cudaGetErrorString(e));
    return RSOL_OK;
}

rsol_status rsol_batch_check(rsol_batch_ctx *b, void *stream)
{
    if (!b)
        return RSOL_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return bfail(b, RSOL_ERR_CUDA, "rsol_batch_check: %s", cudaGetErrorString(e));
    if (h & rsol::ST_NONFINITE)
        return bfail(b, RSOL_ERR_NONFINITE, "a packet momentum or position became non-finite");
    if (h & rsol::ST_COURANT)
        return bfail(b, RSOL_ERR_COURANT, "a packet moved more than one cell in one step");
    if (h & rsol::ST_BADCELL)
        return bfail(b, RSOL_ERR_INVALID_ARG, "a packet's cell index lies off its box's grid");
    return RSOL_OK;
}

} // extern "C"
