// Stable cell sort of the packets (not in the paper: it orders packets so the
// binned push kernel can keep gathers and deposits on chip).
//
// Keys are bin-major keys of each packet's anchor node (the cell for CIC, the
// nearest node for TSC): the bin's linear index, x fastest, times bin^3 plus the
// node's linear index inside the bin.  A least-significant-digit radix sort
// with 8-bit digits orders (key, index) pairs, starting from the identity
// order; every pass is stable (ranks inside a tile follow item order, tiles
// follow tile order), so the final permutation is the unique stable one.  The
// packet arrays are then gathered through the permutation, and the same kernel
// records the per-bin packet ranges.
#include <cstdint>
#include <cuda_runtime.h>

#include "rsol_device.cuh"
#include "rsol_internal.h"

namespace rsol {

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;  // items per block
constexpr int RADIX = 256;

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

int64_t blocks_for(int64_t n) { return (n + SORT_TILE - 1) / SORT_TILE; }

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Anchor node of one axis: the cell (CIC) or the nearest node (TSC, periodic).
template <typename T>
__device__ __forceinline__ uint32_t anchor(uint32_t i, T f, int shape, uint32_t n)
{
    if (shape == 2 && f >= T(0.5))
        return i + 1 == n ? 0u : i + 1;
    return i;
}

// Bin-major key of a packet's anchor node (bin = 1 << lb): the bin's linear
// index, x fastest, times bin^3 plus the node's linear index inside the bin.
template <typename T>
__device__ __forceinline__ uint32_t anchor_key(uint32_t c, T f0, T f1, T f2, int shape, int nx,
                                               int ny, int nz, int lb, int nbx, int nby)
{
    const uint32_t m = (1u << lb) - 1u;
    const uint32_t ix = anchor(uint32_t(cell_x(c)), f0, shape, uint32_t(nx));
    const uint32_t iy = anchor(uint32_t(cell_y(c)), f1, shape, uint32_t(ny));
    const uint32_t iz = anchor(uint32_t(cell_z(c)), f2, shape, uint32_t(nz));
    const uint32_t bin_id = ((iz >> lb) * uint32_t(nby) + (iy >> lb)) * uint32_t(nbx) + (ix >> lb);
    const uint32_t local = (((iz & m) << lb | (iy & m)) << lb) | (ix & m);
    return (bin_id << (3 * lb)) | local;
}

// The radix path's kernels run only when `gate` is null or *gate != 0: after
// a re-sort of a previously sorted set they are launched behind it with the
// re-sort's fallback flag, and do nothing unless it fell back.
__device__ __forceinline__ bool gated_off(const int *gate) { return gate && *gate == 0; }

// Bin-major key of each packet's anchor node; bin = 1 << lb.
template <typename T>
__global__ void keys_kernel(const uint32_t *__restrict__ cell, const T *__restrict__ o0,
                            const T *__restrict__ o1, const T *__restrict__ o2, int64_t n,
                            int shape, int nx, int ny, int nz, int lb, int nbx, int nby,
                            uint32_t *__restrict__ keys, const int *gate = nullptr)
{
    if (gated_off(gate))
        return;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const uint32_t m = (1u << lb) - 1u;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t c = cell[i];
        const uint32_t ix = anchor(uint32_t(cell_x(c)), o0[i], shape, uint32_t(nx));
        const uint32_t iy = anchor(uint32_t(cell_y(c)), o1[i], shape, uint32_t(ny));
        const uint32_t iz = anchor(uint32_t(cell_z(c)), o2[i], shape, uint32_t(nz));
        const uint32_t bin_id = ((iz >> lb) * uint32_t(nby) + (iy >> lb)) * uint32_t(nbx) + (ix >> lb);
        const uint32_t local = (((iz & m) << lb | (iy & m)) << lb) | (ix & m);
        keys[i] = (bin_id << (3 * lb)) | local;
    }
}

// Box-major keys of a batch of boxes sharing one packet array.
template <typename T>
__global__ void batch_keys_kernel(const uint32_t *__restrict__ cell, const T *__restrict__ o0,
                                  const T *__restrict__ o1, const T *__restrict__ o2, int64_t n,
                                  const int64_t *__restrict__ offsets,
                                  const BatchKeyBox *__restrict__ boxes, int n_boxes, int shape,
                                  int lb, uint32_t *__restrict__ keys)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const uint32_t m = (1u << lb) - 1u;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        int lo = 0, hi = n_boxes - 1;  // box b with offsets[b] <= i < offsets[b + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= i)
                lo = mid;
            else
                hi = mid - 1;
        }
        const BatchKeyBox bx = boxes[lo];
        const uint32_t c = cell[i];
        const uint32_t ix = anchor(uint32_t(cell_x(c)), o0[i], shape, uint32_t(bx.nx));
        const uint32_t iy = anchor(uint32_t(cell_y(c)), o1[i], shape, uint32_t(bx.ny));
        const uint32_t iz = anchor(uint32_t(cell_z(c)), o2[i], shape, uint32_t(bx.nz));
        const uint32_t bin_id = bx.bin_base +
                                ((iz >> lb) * uint32_t(bx.nby) + (iy >> lb)) * uint32_t(bx.nbx) +
                                (ix >> lb);
        const uint32_t local = (((iz & m) << lb | (iy & m)) << lb) | (ix & m);
        keys[i] = (bin_id << (3 * lb)) | local;
    }
}

// Per-block digit histograms: counts[d * nblocks + b].  A block's tile is
// SORT_TILE consecutive items; warp w takes the w-th run of SUB items, 32 per
// row (all its keys are loaded before any is counted).
constexpr int SUB = SORT_TILE / SORT_WARPS;

__global__ void __launch_bounds__(SORT_THREADS) upsweep_kernel(const uint32_t *__restrict__ keys,
                                                               int64_t n, int shift,
                                                               uint32_t *__restrict__ counts,
                                                               int64_t nblocks, const int *gate)
{
    if (gated_off(gate))
        return;
    __shared__ uint32_t hist[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x)
        hist[d] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * SORT_TILE + int64_t(warp) * SUB + lane;
    uint32_t d[SORT_ITEMS];
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const int64_t i = base + it * 32;
        d[it] = i < n ? (keys[i] >> shift) & (RADIX - 1) : uint32_t(RADIX);
    }
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const uint32_t peers = __match_any_sync(0xffffffffu, d[it]);
        if (d[it] < RADIX && lane == __ffs(peers) - 1)
            atomicAdd(&hist[d[it]], uint32_t(__popc(peers)));
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < RADIX; dd += blockDim.x)
        counts[int64_t(dd) * nblocks + blockIdx.x] = hist[dd];
}

// Row d of counts: exclusive prefix over blocks, in place; total -> totals[d].
__global__ void __launch_bounds__(1024) row_scan_kernel(uint32_t *__restrict__ counts,
                                                        int64_t nblocks,
                                                        uint32_t *__restrict__ totals,
                                                        const int *gate)
{
    if (gated_off(gate))
        return;
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    uint32_t *row = counts + int64_t(blockIdx.x) * nblocks;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nblocks; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < nblocks ? row[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += y;
        }
        if (lane == 31)
            warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = lane < int(blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o)
                    s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const uint32_t before = (warp > 0 ? warp_sums[warp - 1] : 0u) + carry;
        if (i < nblocks)
            row[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1)
            carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0)
        totals[blockIdx.x] = carry;
}

// Exclusive scan of the 256 digit totals (one block of 256 threads).
__global__ void digit_base_kernel(uint32_t *__restrict__ totals, const int *gate)
{
    if (gated_off(gate))
        return;
    __shared__ uint32_t s[RADIX];
    s[threadIdx.x] = totals[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int d = 0; d < RADIX; ++d) {
            const uint32_t v = s[d];
            s[d] = acc;
            acc += v;
        }
    }
    __syncthreads();
    totals[threadIdx.x] = s[threadIdx.x];
}

// Stable scatter of one radix pass.  The tile (same items and order as the
// upsweep's) is ranked in registers, staged in shared memory in its sorted
// order, and written out digit run by digit run (consecutive addresses).
// An item's rank among the tile's items of its digit is: the items of that
// digit in earlier warps, then in earlier rows of its warp, then in earlier
// lanes of its row, which is the tile's index order, so the pass is stable.
__global__ void __launch_bounds__(SORT_THREADS, 3) downsweep_kernel(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ idx_in, int64_t n, int shift,
    const uint32_t *__restrict__ counts, int64_t nblocks, const uint32_t *__restrict__ digit_base,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ idx_out, const int *gate)
{
    if (gated_off(gate))
        return;
    static_assert(SORT_THREADS == RADIX, "one thread per digit in the digit scans");
    __shared__ uint32_t s_cnt[SORT_WARPS][RADIX];  // per warp: running count, then offset in the digit
    __shared__ uint32_t s_start[RADIX];            // first staged slot of each digit
    __shared__ uint32_t s_gbase[RADIX];            // first output position of the tile's digit
    __shared__ uint32_t s_wsum[SORT_WARPS];
    __shared__ uint32_t s_key[SORT_TILE], s_idx[SORT_TILE];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = 0; w < SORT_WARPS; ++w)
        s_cnt[w][threadIdx.x] = 0;
    const int64_t tile0 = int64_t(blockIdx.x) * SORT_TILE;
    const int64_t base = tile0 + int64_t(warp) * SUB + lane;
    uint32_t k[SORT_ITEMS], v[SORT_ITEMS], r[SORT_ITEMS];
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const int64_t i = base + it * 32;
        const bool valid = i < n;
        k[it] = valid ? keys_in[i] : 0u;
        v[it] = valid ? (idx_in ? idx_in[i] : uint32_t(i)) : 0u;  // first pass: identity
    }
    // an item's digit, RADIX past the end of the input
    auto digit = [&](int it) {
        return base + it * 32 < n ? (k[it] >> shift) & (RADIX - 1) : uint32_t(RADIX);
    };
    __syncthreads();
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const uint32_t d = digit(it);
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const bool ok = d < RADIX;
        const uint32_t before = ok ? s_cnt[warp][d] : 0u;
        r[it] = before + __popc(peers & lt);
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1)
            s_cnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // thread t owns digit t: offsets of each warp's items within the digit,
        // the tile's count of it, then the exclusive scan over digits
        const int t = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = s_cnt[w][t];
            s_cnt[w][t] = run;
            run += c;
        }
        s_gbase[t] = digit_base[t] + counts[int64_t(t) * nblocks + blockIdx.x];
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            s_wsum[warp] = incl;
        __syncthreads();
        uint32_t wb = 0;
        for (int w = 0; w < warp; ++w)
            wb += s_wsum[w];
        s_start[t] = wb + incl - run;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const uint32_t d = digit(it);
        if (d < RADIX) {
            const uint32_t p = s_start[d] + s_cnt[warp][d] + r[it];
            s_key[p] = k[it];
            s_idx[p] = v[it];
        }
    }
    __syncthreads();
    const int tile_n = int(n - tile0 < SORT_TILE ? n - tile0 : SORT_TILE);
    for (int p = threadIdx.x; p < tile_n; p += SORT_THREADS) {
        const uint32_t key = s_key[p];
        const uint32_t dp = (key >> shift) & (RADIX - 1);
        const uint32_t pos = s_gbase[dp] + (uint32_t(p) - s_start[dp]);
        keys_out[pos] = key;
        idx_out[pos] = s_idx[p];
    }
}

// out[i] = in[perm[i]] for the packet arrays, and the bin ranges from the
// sorted keys: bin_start[b] = first sorted position whose key's bin is >= b
// (b = 0..nbins; keys of off-grid cells sort last, past every bin).
template <typename T>
__global__ void gather_kernel(const uint32_t *__restrict__ perm, int64_t n,
                              const uint32_t *__restrict__ cell_in, const T *__restrict__ o0,
                              const T *__restrict__ o1, const T *__restrict__ o2,
                              const T *__restrict__ v0, const T *__restrict__ v1,
                              const T *__restrict__ v2, const T *__restrict__ w,
                              uint32_t *__restrict__ cell_out, T *__restrict__ p0,
                              T *__restrict__ p1, T *__restrict__ p2, T *__restrict__ q0,
                              T *__restrict__ q1, T *__restrict__ q2, T *__restrict__ wo,
                              const uint32_t *__restrict__ keys, int shift3, int64_t nbins,
                              uint32_t *__restrict__ bin_start)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t j = perm ? perm[i] : uint32_t(i);
        cell_out[i] = cell_in[j];
        p0[i] = o0[j];
        p1[i] = o1[j];
        p2[i] = o2[j];
        q0[i] = v0[j];
        q1[i] = v1[j];
        q2[i] = v2[j];
        wo[i] = w[j];
        int64_t prev = i == 0 ? -1 : int64_t(keys[i - 1] >> shift3);
        int64_t cur = int64_t(keys[i] >> shift3);
        prev = prev > nbins ? nbins : prev;
        cur = cur > nbins ? nbins : cur;
        for (int64_t b = prev + 1; b <= cur; ++b)
            bin_start[b] = uint32_t(i);
        if (i == n - 1)
            for (int64_t b = cur + 1; b <= nbins; ++b)
                bin_start[b] = uint32_t(n);
    }
}

// ---------------------------------------------------------------------------
// Re-sort of a set still in the order of this context's previous sort.
// Between sorts a packet moves at most one bin along each axis in every
// workload here, so each new bin's packets come from the 27 old bins around
// it.  The re-sort splits every old bin's packets by the direction of their
// move (ranks follow the old order), places them in the new bins source by
// source in increasing old-bin order, and sorts each new bin by the in-bin
// part of the key, keeping the order of equal keys.  Packets with equal keys
// therefore keep their old order: the permutation is the one the stable sort
// by key gives, bit for bit.  A packet that moved further, a cell off the grid
// or packets past the last old bin set *fell_back; the re-sort's kernels then
// do nothing and the radix path runs behind them instead.

constexpr int NDIR = 27;  // directions of a move: (dz+1)*9 + (dy+1)*3 + (dx+1)

// Step from old bin b to new bin B along a periodic axis of nb >= 3 bins:
// -1, 0, 1, or 2 (further).
__device__ __forceinline__ int bin_step(int b, int B, int nb)
{
    int d = B - b;
    d = d == nb - 1 ? -1 : (d == 1 - nb ? 1 : d);
    return d >= -1 && d <= 1 ? d : 2;
}

__device__ __forceinline__ int wrap_bin(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Direction of the move from old bin (bx, by, bz) to new bin B, or NDIR.
__device__ __forceinline__ int move_dir(int bx, int by, int bz, uint32_t B, int nbx, int nby, int nbz)
{
    if (B >= uint32_t(nbx) * uint32_t(nby) * uint32_t(nbz))
        return NDIR;
    const int Bx = int(B % uint32_t(nbx)), By = int((B / uint32_t(nbx)) % uint32_t(nby));
    const int Bz = int(B / (uint32_t(nbx) * uint32_t(nby)));
    const int dx = bin_step(bx, Bx, nbx), dy = bin_step(by, By, nby), dz = bin_step(bz, Bz, nbz);
    if (dx == 2 || dy == 2 || dz == 2)
        return NDIR;
    return ((dz + 1) * 3 + (dy + 1)) * 3 + (dx + 1);
}

// Per old bin: every packet's new key (in the old order) and the packets per
// direction of move, cnt[b * NDIR + d].
template <typename T>
__global__ void __launch_bounds__(256) resort_count_kernel(
    const uint32_t *__restrict__ cell, const T *__restrict__ o0, const T *__restrict__ o1,
    const T *__restrict__ o2, int64_t n, int shape, int nx, int ny, int nz, int lb, int nbx,
    int nby, int nbz, const uint32_t *__restrict__ old_start, uint32_t *__restrict__ keys,
    uint32_t *__restrict__ cnt, int *__restrict__ fell_back)
{
    __shared__ uint32_t h[NDIR];
    if (threadIdx.x < NDIR)
        h[threadIdx.x] = 0;
    __syncthreads();
    const int b = blockIdx.x;
    const int nbins = nbx * nby * nbz;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const uint32_t lo = old_start[b], hi = old_start[b + 1];
    // packets past the last bin (off the grid at the last sort): the radix path
    int far = (b == 0 && threadIdx.x == 0 && int64_t(old_start[nbins]) != n) ? 1 : 0;
    const int lane = threadIdx.x & 31;
    for (uint32_t i0 = lo; i0 < hi; i0 += blockDim.x) {  // warp-uniform trip count
        const uint32_t i = i0 + threadIdx.x;
        int d = NDIR + 1;  // no packet
        if (i < hi) {
            const uint32_t c = cell[i];
            if (cell_x(c) >= nx || cell_y(c) >= ny || cell_z(c) >= nz) {
                d = NDIR;
            } else {
                const uint32_t key = anchor_key(c, o0[i], o1[i], o2[i], shape, nx, ny, nz, lb, nbx, nby);
                keys[i] = key;
                d = move_dir(bx, by, bz, key >> (3 * lb), nbx, nby, nbz);
            }
        }
        far |= d == NDIR;
        // one shared add per direction and warp (most packets stay in their bin)
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (d < NDIR && lane == __ffs(peers) - 1)
            atomicAdd(&h[d], uint32_t(__popc(peers)));
    }
    if (__syncthreads_or(far)) {
        if (threadIdx.x == 0)
            atomicOr(fell_back, 1);
        return;
    }
    if (threadIdx.x < NDIR)
        cnt[int64_t(b) * NDIR + threadIdx.x] = h[threadIdx.x];
}

// The three old-bin coordinates around new coordinate c on a periodic axis of
// nb >= 3 bins, in increasing order, with the step from each to c.
__device__ __forceinline__ void axis_sources(int c, int nb, int s[3], int st[3])
{
    s[0] = wrap_bin(c - 1, nb);
    s[1] = c;
    s[2] = wrap_bin(c + 1, nb);
    st[0] = 1;
    st[1] = 0;
    st[2] = -1;
    auto order = [&](int i, int j) {
        if (s[i] > s[j]) {
            const int a = s[i], t = st[i];
            s[i] = s[j];
            st[i] = st[j];
            s[j] = a;
            st[j] = t;
        }
    };
    order(0, 1);
    order(1, 2);
    order(0, 1);
}

// Per new bin B: its packets come from the 27 old bins around it, taken in
// increasing old-bin order (the lexicographic order of the sorted per-axis
// sources): off[b * NDIR + d] = where the packets of old bin b that moved in
// direction d start inside B; tot[B] = the packets of B.
__global__ void resort_offsets_kernel(const uint32_t *__restrict__ cnt, int nbx, int nby, int nbz,
                                      uint32_t *__restrict__ off, uint32_t *__restrict__ tot,
                                      const int *__restrict__ fell_back)
{
    if (*fell_back)
        return;
    const int nbins = nbx * nby * nbz;
    for (int B = blockIdx.x * blockDim.x + threadIdx.x; B < nbins; B += gridDim.x * blockDim.x) {
        const int Bx = B % nbx, By = (B / nbx) % nby, Bz = B / (nbx * nby);
        int sx[3], tx[3], sy[3], ty[3], sz[3], tz[3];
        axis_sources(Bx, nbx, sx, tx);
        axis_sources(By, nby, sy, ty);
        axis_sources(Bz, nbz, sz, tz);
        uint32_t acc = 0;
        for (int iz = 0; iz < 3; ++iz)
            for (int iy = 0; iy < 3; ++iy)
                for (int ix = 0; ix < 3; ++ix) {
                    const int64_t src = (int64_t(sz[iz]) * nby + sy[iy]) * nbx + sx[ix];
                    const int d = ((tz[iz] + 1) * 3 + (ty[iy] + 1)) * 3 + (tx[ix] + 1);
                    off[src * NDIR + d] = acc;
                    acc += cnt[src * NDIR + d];
                }
        tot[B] = acc;
    }
}

// Exclusive scan of n values held by a block's 256 threads (v: each thread's
// share of consecutive values, first..first + per - 1), in place in a.
template <int PER>
__device__ __forceinline__ void block_exclusive_scan_256(uint32_t *a, uint32_t *s_wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v[PER], sum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = a[threadIdx.x * PER + k];
        sum += v[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        incl += lane >= o ? y : 0u;
    }
    if (lane == 31)
        s_wsum[warp] = incl;
    __syncthreads();
    uint32_t run = incl - sum;
    for (int w = 0; w < warp; ++w)
        run += s_wsum[w];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        a[threadIdx.x * PER + k] = run;
        run += v[k];
    }
    __syncthreads();
}

// Exclusive scan of the new bins' packet counts: start[0 .. nbins].
__global__ void __launch_bounds__(1024) resort_scan_kernel(const uint32_t *__restrict__ tot, int nbins,
                                                           uint32_t *__restrict__ start,
                                                           const int *__restrict__ fell_back)
{
    if (*fell_back)
        return;
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    for (int base = 0; base < nbins; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nbins ? tot[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            x += lane >= o ? y : 0u;
        }
        if (lane == 31)
            wsum[warp] = x;
        __syncthreads();
        uint32_t before = carry;
        for (int w = 0; w < warp; ++w)
            before += wsum[w];
        if (i < nbins)
            start[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1)
            carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0)
        start[nbins] = carry;
}

// Stable ranks of one round of a CTA's items by bucket: warp w takes the w-th
// run of 32 * ITEMS consecutive items, row by row (32 per row), and keeps a
// running count per bucket in s_cnt[w][] (rank = earlier rows of the warp,
// then earlier lanes).  Then, per bucket, the exclusive prefix over warps goes
// to s_cnt[w][] and the round's total to tot[] (bucket t of thread t / ...).
// An item's place in the round's order of its bucket is s_cnt[warp][b] + rank.
template <int NW, int ITEMS, int NB>
__device__ __forceinline__ void round_ranks(const uint32_t (&bk)[ITEMS], uint32_t (&rank)[ITEMS],
                                            uint32_t (*s_cnt)[NB], uint32_t *tot)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    for (int t = threadIdx.x; t < NW * NB; t += blockDim.x)
        s_cnt[t / NB][t % NB] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        const uint32_t k = bk[r];
        const uint32_t peers = __match_any_sync(0xffffffffu, k);
        const bool ok = k < uint32_t(NB);
        const uint32_t before = ok ? s_cnt[warp][k] : 0u;
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1)
            s_cnt[warp][k] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NB; t += blockDim.x) {
        uint32_t run = 0;
        for (int w = 0; w < NW; ++w) {
            const uint32_t c = s_cnt[w][t];
            s_cnt[w][t] = run;
            run += c;
        }
        tot[t] = run;
    }
    __syncthreads();
}

// Per old bin: every packet (old order) to its place in its new bin, ranks
// per direction following the old order: keys_out / idx_out in bin order.
template <int NW, int ITEMS>
__global__ void __launch_bounds__(NW * 32) resort_scatter_kernel(
    const uint32_t *__restrict__ keys, const uint32_t *__restrict__ old_start,
    const uint32_t *__restrict__ start, const uint32_t *__restrict__ off, int lb, int nbx, int nby,
    int nbz, uint32_t *__restrict__ keys_out, uint32_t *__restrict__ idx_out,
    const int *__restrict__ fell_back)
{
    if (*fell_back)
        return;
    constexpr int ROUND = NW * 32 * ITEMS;
    __shared__ uint32_t s_base[NDIR];  // output slot of the next packet of each direction
    __shared__ uint32_t s_cnt[NW][NDIR];
    __shared__ uint32_t s_tot[NDIR];
    const int b = blockIdx.x;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < NDIR) {
        const int d = threadIdx.x;
        const int Bx = wrap_bin(bx + d % 3 - 1, nbx), By = wrap_bin(by + (d / 3) % 3 - 1, nby),
                  Bz = wrap_bin(bz + d / 9 - 1, nbz);
        s_base[d] = start[(Bz * nby + By) * nbx + Bx] + off[int64_t(b) * NDIR + d];
    }
    const uint32_t lo = old_start[b], hi = old_start[b + 1];
    for (uint32_t r0 = lo; r0 < hi; r0 += ROUND) {
        uint32_t key[ITEMS], dir[ITEMS], rank[ITEMS];
        const uint32_t w0 = r0 + uint32_t(warp) * 32 * ITEMS + lane;
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t i = w0 + uint32_t(r) * 32;
            key[r] = i < hi ? keys[i] : 0u;
            dir[r] = i < hi ? uint32_t(move_dir(bx, by, bz, key[r] >> (3 * lb), nbx, nby, nbz))
                            : uint32_t(NDIR);
        }
        round_ranks<NW, ITEMS, NDIR>(dir, rank, s_cnt, s_tot);
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t i = w0 + uint32_t(r) * 32;
            if (i < hi) {
                const uint32_t pos = s_base[dir[r]] + s_cnt[warp][dir[r]] + rank[r];
                keys_out[pos] = key[r];
                idx_out[pos] = i;
            }
        }
        __syncthreads();
        if (threadIdx.x < NDIR)
            s_base[threadIdx.x] += s_tot[threadIdx.x];
        __syncthreads();
    }
}

// Per new bin: its packets (bin order from the scatter) sorted by the in-bin
// part of the key, equal keys in their incoming order.
template <int LB, int NW, int ITEMS>
__global__ void __launch_bounds__(NW * 32) resort_bin_kernel(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ idx_in,
    const uint32_t *__restrict__ start, uint32_t *__restrict__ keys_out,
    uint32_t *__restrict__ idx_out, const int *__restrict__ fell_back)
{
    constexpr int NL = 1 << (3 * LB);  // in-bin keys (512 for 8^3 bins, 64 for 4^3)
    constexpr int NP = NL > 256 ? NL : 256;
    constexpr int ROUND = NW * 32 * ITEMS;
    static_assert(NW * 32 == 256, "the in-bin key scan assumes 256 threads");
    if (*fell_back)
        return;
    __shared__ uint32_t s_pos[NP];  // next slot of each in-bin key, bin-relative
    __shared__ uint32_t s_cnt[NW][NL];
    __shared__ uint32_t s_tot[NL];
    __shared__ uint32_t s_wsum[NW];
    const int B = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lo = start[B], hi = start[B + 1];
    for (int t = threadIdx.x; t < NP; t += blockDim.x)
        s_pos[t] = 0;
    __syncthreads();
    for (uint32_t i0 = lo; i0 < hi; i0 += blockDim.x) {  // histogram, one add per key and warp
        const uint32_t i = i0 + threadIdx.x;
        const uint32_t L = i < hi ? keys_in[i] & uint32_t(NL - 1) : uint32_t(NL);
        const uint32_t peers = __match_any_sync(0xffffffffu, L);
        if (L < uint32_t(NL) && lane == __ffs(peers) - 1)
            atomicAdd(&s_pos[L], uint32_t(__popc(peers)));
    }
    __syncthreads();
    block_exclusive_scan_256<NP / 256>(s_pos, s_wsum);
    for (uint32_t r0 = lo; r0 < hi; r0 += ROUND) {
        uint32_t key[ITEMS], v[ITEMS], L[ITEMS], rank[ITEMS];
        const uint32_t w0 = r0 + uint32_t(warp) * 32 * ITEMS + lane;
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t i = w0 + uint32_t(r) * 32;
            key[r] = i < hi ? keys_in[i] : 0u;
            v[r] = i < hi ? idx_in[i] : 0u;
            L[r] = i < hi ? key[r] & uint32_t(NL - 1) : uint32_t(NL);
        }
        round_ranks<NW, ITEMS, NL>(L, rank, s_cnt, s_tot);
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            if (L[r] < uint32_t(NL)) {
                const uint32_t pos = lo + s_pos[L[r]] + s_cnt[warp][L[r]] + rank[r];
                keys_out[pos] = key[r];
                idx_out[pos] = v[r];
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NL; t += blockDim.x)
            s_pos[t] += s_tot[t];
        __syncthreads();
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 65535 * 8)
        b = 65535 * 8;
    return int(b < 1 ? 1 : b);
}

} // namespace

size_t sort_scratch_bytes(int64_t n, int64_t nbins)
{
    const int64_t nb = blocks_for(n);
    return 4 * align_up(size_t(n) * 4) + align_up(size_t(RADIX) * nb * 4) +
           align_up(size_t(RADIX) * 4) + align_up(size_t(nbins + 1) * 4);
}

void sort_scratch_carve(void *base, int64_t n, int64_t nbins, SortScratch *s)
{
    char *p = static_cast<char *>(base);
    const int64_t nb = blocks_for(n);
    s->keys[0] = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(n) * 4);
    s->keys[1] = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(n) * 4);
    s->idx[0] = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(n) * 4);
    s->idx[1] = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(n) * 4);
    s->counts = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(RADIX) * nb * 4);
    s->block_sums = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(RADIX) * 4);
    s->bin_start = reinterpret_cast<uint32_t *>(p);
    s->capacity = n;
    s->max_blocks = nb;
}

cudaError_t sort_particles(const SortScratch &s, int64_t n, int elem_bytes,
                           const uint32_t *cell_in, void *const off_in[3], void *const u_in[3],
                           const void *w_in, uint32_t *cell_out, void *const off_out[3],
                           void *const u_out[3], void *w_out, int nx, int ny, int nz, int bin,
                           int shape, int key_bits, int64_t nbins, cudaStream_t st)
{
    int lb = 0;
    while ((1 << lb) < bin)
        ++lb;
    const int nbx = (nx + bin - 1) / bin, nby = (ny + bin - 1) / bin;
    cudaError_t e;
    if (n > 0) {
        if (elem_bytes == 4)
            keys_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(
                cell_in, static_cast<const float *>(off_in[0]), static_cast<const float *>(off_in[1]),
                static_cast<const float *>(off_in[2]), n, shape, nx, ny, nz, lb, nbx, nby, s.keys[0]);
        else
            keys_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(
                cell_in, static_cast<const double *>(off_in[0]),
                static_cast<const double *>(off_in[1]), static_cast<const double *>(off_in[2]), n,
                shape, nx, ny, nz, lb, nbx, nby, s.keys[0]);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        return sort_from_keys(s, n, elem_bytes, cell_in, off_in, u_in, w_in, cell_out, off_out,
                              u_out, w_out, lb, key_bits, nbins, st);
    } else {
        e = cudaMemsetAsync(s.bin_start, 0, size_t(nbins + 1) * 4, st);
        if (e != cudaSuccess)
            return e;
    }
    return cudaGetLastError();
}

cudaError_t sort_from_keys(const SortScratch &s, int64_t n, int elem_bytes,
                       const uint32_t *cell_in, void *const off_in[3], void *const u_in[3],
                       const void *w_in, uint32_t *cell_out, void *const off_out[3],
                       void *const u_out[3], void *w_out, int lb, int key_bits,
                       int64_t nbins, cudaStream_t st, const int *gate)
{
    cudaError_t e;
    const int64_t nb = blocks_for(n);
    int cur = 0;
    for (int shift = 0; shift < key_bits; shift += 8) {
        upsweep_kernel<<<unsigned(nb), SORT_THREADS, 0, st>>>(s.keys[cur], n, shift, s.counts, nb, gate);
        row_scan_kernel<<<RADIX, 1024, 0, st>>>(s.counts, nb, s.block_sums, gate);
        digit_base_kernel<<<1, RADIX, 0, st>>>(s.block_sums, gate);
        downsweep_kernel<<<unsigned(nb), SORT_THREADS, 0, st>>>(
            s.keys[cur], shift == 0 ? nullptr : s.idx[cur], n, shift, s.counts, nb, s.block_sums,
            s.keys[cur ^ 1], s.idx[cur ^ 1], gate);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        cur ^= 1;
    }
    if (elem_bytes == 4)
        gather_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(
            key_bits > 0 ? s.idx[cur] : nullptr, n, cell_in, static_cast<const float *>(off_in[0]),
            static_cast<const float *>(off_in[1]), static_cast<const float *>(off_in[2]),
            static_cast<const float *>(u_in[0]), static_cast<const float *>(u_in[1]),
            static_cast<const float *>(u_in[2]), static_cast<const float *>(w_in), cell_out,
            static_cast<float *>(off_out[0]), static_cast<float *>(off_out[1]),
            static_cast<float *>(off_out[2]), static_cast<float *>(u_out[0]),
            static_cast<float *>(u_out[1]), static_cast<float *>(u_out[2]),
            static_cast<float *>(w_out), s.keys[cur], 3 * lb, nbins, s.bin_start);
    else
        gather_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(
            key_bits > 0 ? s.idx[cur] : nullptr, n, cell_in, static_cast<const double *>(off_in[0]),
            static_cast<const double *>(off_in[1]), static_cast<const double *>(off_in[2]),
            static_cast<const double *>(u_in[0]), static_cast<const double *>(u_in[1]),
            static_cast<const double *>(u_in[2]), static_cast<const double *>(w_in), cell_out,
            static_cast<double *>(off_out[0]), static_cast<double *>(off_out[1]),
            static_cast<double *>(off_out[2]), static_cast<double *>(u_out[0]),
            static_cast<double *>(u_out[1]), static_cast<double *>(u_out[2]),
            static_cast<double *>(w_out), s.keys[cur], 3 * lb, nbins, s.bin_start);
    return cudaGetLastError();
}

size_t resort_scratch_bytes(int64_t n, int64_t nbins)
{
    return 2 * align_up(size_t(n) * 4) + 2 * align_up(size_t(nbins) * NDIR * 4) +
           align_up(size_t(nbins) * 4) + align_up(size_t(nbins + 1) * 4) + align_up(4);
}

void resort_scratch_carve(void *base, int64_t n, int64_t nbins, ResortScratch *r)
{
    char *p = static_cast<char *>(base);
    r->keys = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(n) * 4);
    r->idx = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(n) * 4);
    r->cnt = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(nbins) * NDIR * 4);
    r->off = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(nbins) * NDIR * 4);
    r->tot = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(nbins) * 4);
    r->start = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(nbins + 1) * 4);
    r->fell_back = reinterpret_cast<int *>(p);
    r->capacity = n;
}

bool resort_applies(int bin, int nbx, int nby, int nbz)
{
    return (bin == 4 || bin == 8) && nbx >= 3 && nby >= 3 && nbz >= 3;
}

cudaError_t resort_particles(const SortScratch &s, const ResortScratch &r, int64_t n, int elem_bytes,
                             const uint32_t *cell_in, void *const off_in[3], void *const u_in[3],
                             const void *w_in, uint32_t *cell_out, void *const off_out[3],
                             void *const u_out[3], void *w_out, int nx, int ny, int nz, int bin,
                             int shape, int key_bits, int nbx, int nby, int nbz, cudaStream_t st)
{
    const int lb = bin == 8 ? 3 : 2;
    const int nbins = nbx * nby * nbz;
    cudaError_t e = cudaMemsetAsync(r.fell_back, 0, sizeof(int), st);
    if (e != cudaSuccess)
        return e;
    // new keys, moves per direction (s.bin_start still holds the old bins)
    if (elem_bytes == 4)
        resort_count_kernel<float><<<nbins, 256, 0, st>>>(
            cell_in, static_cast<const float *>(off_in[0]), static_cast<const float *>(off_in[1]),
            static_cast<const float *>(off_in[2]), n, shape, nx, ny, nz, lb, nbx, nby, nbz,
            s.bin_start, s.keys[0], r.cnt, r.fell_back);
    else
        resort_count_kernel<double><<<nbins, 256, 0, st>>>(
            cell_in, static_cast<const double *>(off_in[0]), static_cast<const double *>(off_in[1]),
            static_cast<const double *>(off_in[2]), n, shape, nx, ny, nz, lb, nbx, nby, nbz,
            s.bin_start, s.keys[0], r.cnt, r.fell_back);
    resort_offsets_kernel<<<(nbins + 255) / 256, 256, 0, st>>>(r.cnt, nbx, nby, nbz, r.off, r.tot,
                                                               r.fell_back);
    resort_scan_kernel<<<1, 1024, 0, st>>>(r.tot, nbins, r.start, r.fell_back);
    resort_scatter_kernel<8, 8><<<nbins, 256, 0, st>>>(s.keys[0], s.bin_start, r.start, r.off, lb, nbx,
                                                      nby, nbz, r.keys, r.idx, r.fell_back);
    // the final order where the radix path leaves it (its last pass's buffers):
    // callers that read the permutation find it in the same place either way
    const int fin = ((key_bits + 7) / 8) & 1;
    if (lb == 3)
        resort_bin_kernel<3, 8, 8><<<nbins, 256, 0, st>>>(r.keys, r.idx, r.start, s.keys[fin],
                                                         s.idx[fin], r.fell_back);
    else
        resort_bin_kernel<2, 8, 8><<<nbins, 256, 0, st>>>(r.keys, r.idx, r.start, s.keys[fin],
                                                         s.idx[fin], r.fell_back);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    // the radix path, gated on the fallback (its keys kernel rewrites s.keys[0];
    // a grid-stride grid of a few CTAs per SM, cheap to launch when gated off)
    const int nb1 = nbx, nb2 = nby;
    const int kgrid = grid_for(n, 256) < 4096 ? grid_for(n, 256) : 4096;
    if (elem_bytes == 4)
        keys_kernel<float><<<kgrid, 256, 0, st>>>(
            cell_in, static_cast<const float *>(off_in[0]), static_cast<const float *>(off_in[1]),
            static_cast<const float *>(off_in[2]), n, shape, nx, ny, nz, lb, nb1, nb2, s.keys[0],
            r.fell_back);
    else
        keys_kernel<double><<<kgrid, 256, 0, st>>>(
            cell_in, static_cast<const double *>(off_in[0]), static_cast<const double *>(off_in[1]),
            static_cast<const double *>(off_in[2]), n, shape, nx, ny, nz, lb, nb1, nb2, s.keys[0],
            r.fell_back);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    return sort_from_keys(s, n, elem_bytes, cell_in, off_in, u_in, w_in, cell_out, off_out, u_out,
                          w_out, lb, key_bits, nbins, st, r.fell_back);
}

cudaError_t sort_particles_batch(const SortScratch &s, int64_t n, int elem_bytes,
                                 const uint32_t *cell_in, void *const off_in[3],
                                 void *const u_in[3], const void *w_in, uint32_t *cell_out,
                                 void *const off_out[3], void *const u_out[3], void *w_out,
                                 const int64_t *d_offsets, const BatchKeyBox *d_boxes,
                                 int n_boxes, int bin, int shape, int key_bits, int64_t nbins,
                                 cudaStream_t st)
{
    int lb = 0;
    while ((1 << lb) < bin)
        ++lb;
    if (n <= 0)
        return cudaMemsetAsync(s.bin_start, 0, size_t(nbins + 1) * 4, st);
    if (elem_bytes == 4)
        batch_keys_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(
            cell_in, static_cast<const float *>(off_in[0]), static_cast<const float *>(off_in[1]),
            static_cast<const float *>(off_in[2]), n, d_offsets, d_boxes, n_boxes, shape, lb,
            s.keys[0]);
    else
        batch_keys_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(
            cell_in, static_cast<const double *>(off_in[0]), static_cast<const double *>(off_in[1]),
            static_cast<const double *>(off_in[2]), n, d_offsets, d_boxes, n_boxes, shape, lb,
            s.keys[0]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return sort_from_keys(s, n, elem_bytes, cell_in, off_in, u_in, w_in, cell_out, off_out, u_out,
                          w_out, lb, key_bits, nbins, st);
}

} // namespace rsol
