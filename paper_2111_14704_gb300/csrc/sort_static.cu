// rsol_sort_static: the stable cell sort of rsol_sort without any device
// allocation.  Its scratch (keys, indices, digit counts, bin ranges) lives in
// one file-scope static device array, so a program that cannot or must not call
// cudaMalloc -- for example code running on a device whose memory is owned by
// another component's allocator, or a host thread that must not stall on the
// device-wide synchronisation that cudaMalloc / cudaFree may cause -- can still
// sort packets.  The caller passes the input and output packet arrays.
//
// The array is kStaticScratchBytes (5 MiB) on every device that loads this
// library and stays there until the process exits.  All calls share it: calls
// whose work overlaps on the device (different streams, or different host
// threads on one device) race and must be serialised by the caller.  Every
// byte the sort reads is written earlier in the same call, so nothing needs
// clearing between calls.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/rsol.h"
#include "rsol_internal.h"

namespace {
constexpr size_t kStaticScratchBytes = size_t(5) << 20;
} // namespace

static __device__ __align__(256) unsigned char g_rsol_sort_scratch[kStaticScratchBytes];

namespace {

// Device address of the static scratch on the current device.  In host code
// the name g_rsol_sort_scratch is only a handle, not a device address, so the
// address is looked up with the device current.  The lookup allocates nothing
// and is repeated on every call: a cached address would go stale if the
// caller reset the device (cudaDeviceReset) and the module were loaded again.
cudaError_t scratch_on_current_device(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rsol_sort_scratch);
    if (e != cudaSuccess)
        return e;
    *out = p;
    return cudaSuccess;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool particles_ok(const rsol_particles *P)
{
    if (!P || P->n < 0 || P->n > int64_t(0xFFFFFFFFll) - 1)
        return false;
    if (P->n == 0)
        return true;
    const void *ptrs[8] = {P->cell, P->off[0], P->off[1], P->off[2], P->u[0], P->u[1], P->u[2], P->w};
    for (int i = 0; i < 8; ++i)
        if (!ptrs[i] || !aligned16(ptrs[i]))
            return false;
    return true;
}

} // namespace

extern "C" rsol_status rsol_sort_static(const rsol_params *p, const rsol_particles *in,
                                        rsol_particles *out, void *stream)
{
    if (!p || !particles_ok(in) || !particles_ok(out) || in->n != out->n)
        return RSOL_ERR_INVALID_ARG;
    const int bin = p->bin == 0 ? (p->precision == 32 ? 8 : 4) : p->bin;
    const bool grid_ok = p->nx >= 2 && p->ny >= 2 && p->nz >= 2 && p->nx <= 1024 &&
                         p->ny <= 1024 && p->nz <= 1024;
    if (!grid_ok || !(p->shape == 1 || p->shape == 2) || !(p->precision == 32 || p->precision == 64) ||
        !(bin == 1 || bin == 2 || bin == 4 || bin == 8 || bin == 16))
        return RSOL_ERR_INVALID_ARG;
    if (in->n > 0) {
        const void *a[8] = {in->cell, in->off[0], in->off[1], in->off[2], in->u[0], in->u[1], in->u[2], in->w};
        const void *b[8] = {out->cell, out->off[0], out->off[1], out->off[2], out->u[0], out->u[1], out->u[2], out->w};
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j)
                if (a[i] == b[j])
                    return RSOL_ERR_INVALID_ARG;
    }
    const int nbx = (p->nx + bin - 1) / bin, nby = (p->ny + bin - 1) / bin, nbz = (p->nz + bin - 1) / bin;
    const int64_t nbins = int64_t(nbx) * nby * nbz;
    int key_bits = 0;
    while ((int64_t(1) << key_bits) < nbins * bin * bin * bin)
        ++key_bits;
    const int64_t n = in->n;
    // the scratch must hold this sort's buffers: reject larger problems
    if (rsol::sort_scratch_bytes(n > 0 ? n : 1, nbins) > kStaticScratchBytes)
        return RSOL_ERR_INVALID_ARG;
    void *base = nullptr;
    if (scratch_on_current_device(&base) != cudaSuccess)
        return RSOL_ERR_CUDA;
    rsol::SortScratch s;
    rsol::sort_scratch_carve(base, n > 0 ? n : 1, nbins, &s);
    const cudaError_t e = rsol::sort_particles(
        s, n, p->precision == 32 ? 4 : 8, in->cell, in->off, in->u, in->w, out->cell, out->off,
        out->u, out->w, p->nx, p->ny, p->nz, bin, p->shape, key_bits, nbins,
        static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RSOL_OK : RSOL_ERR_CUDA;
}
