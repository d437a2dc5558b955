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
//
// Where the key space is small next to the packet count (a few keys per
// packet at most), a counting sort by key gives the same permutation with
// fewer passes over memory; it is described above its kernels.
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

// Runs of equal values in consecutive lanes: the lanes where a run starts,
// and for this lane its run's first lane and (at a run's first lane) its
// length.
struct LaneRun {
    uint32_t heads;  // bit l set: lane l starts a run
    int first;       // first lane of this lane's run
    uint32_t len;    // lanes in the run (meaningful at its first lane)
};
__device__ __forceinline__ LaneRun lane_run(uint32_t v, int lane)
{
    const uint32_t prev = __shfl_up_sync(0xffffffffu, v, 1);
    LaneRun r;
    r.heads = __ballot_sync(0xffffffffu, lane == 0 || prev != v);
    const uint32_t upto = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;  // lanes <= lane
    r.first = 31 - __clz(r.heads & upto);
    const uint32_t after = r.heads & ~upto;
    r.len = uint32_t((after ? __ffs(after) - 1 : 32) - lane);
    return r;
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

// Bin-major key of each packet's anchor node; bin = 1 << lb.
template <typename T>
__global__ void keys_kernel(const uint32_t *__restrict__ cell, const T *__restrict__ o0,
                            const T *__restrict__ o1, const T *__restrict__ o2, int64_t n,
                            int shape, int nx, int ny, int nz, int lb, int nbx, int nby,
                            uint32_t *__restrict__ keys)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        keys[i] = anchor_key(cell[i], o0[i], o1[i], o2[i], shape, nx, ny, nz, lb, nbx, nby);
}

// Box-major key of packet i of a batch of boxes sharing one packet array: the
// packet's box b (offsets[b] <= i < offsets[b + 1]), then the bin-major key of
// its anchor in the box, the box's bins numbered from bin_base.
template <typename T>
__device__ __forceinline__ uint32_t batch_anchor_key(int64_t i, uint32_t c, T f0, T f1, T f2,
                                                     const int64_t *__restrict__ offsets,
                                                     const BatchKeyBox *__restrict__ boxes,
                                                     int n_boxes, int shape, int lb)
{
    int lo = 0, hi = n_boxes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    const BatchKeyBox bx = boxes[lo];
    const uint32_t m = (1u << lb) - 1u;
    const uint32_t ix = anchor(uint32_t(cell_x(c)), f0, shape, uint32_t(bx.nx));
    const uint32_t iy = anchor(uint32_t(cell_y(c)), f1, shape, uint32_t(bx.ny));
    const uint32_t iz = anchor(uint32_t(cell_z(c)), f2, shape, uint32_t(bx.nz));
    const uint32_t bin_id =
        bx.bin_base + ((iz >> lb) * uint32_t(bx.nby) + (iy >> lb)) * uint32_t(bx.nbx) + (ix >> lb);
    const uint32_t local = (((iz & m) << lb | (iy & m)) << lb) | (ix & m);
    return (bin_id << (3 * lb)) | local;
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
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        keys[i] = batch_anchor_key(i, cell[i], o0[i], o1[i], o2[i], offsets, boxes, n_boxes, shape, lb);
}

// Per-block digit histograms: counts[d * nblocks + b].  A block's tile is
// SORT_TILE consecutive items; warp w takes the w-th run of SUB items, 32 per
// row (all its keys are loaded before any is counted).
constexpr int SUB = SORT_TILE / SORT_WARPS;

__global__ void __launch_bounds__(SORT_THREADS) upsweep_kernel(const uint32_t *__restrict__ keys,
                                                               int64_t n, int shift,
                                                               uint32_t *__restrict__ counts,
                                                               int64_t nblocks)
{
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
                                                        uint32_t *__restrict__ totals)
{
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
__global__ void digit_base_kernel(uint32_t *__restrict__ totals)
{
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
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ idx_out)
{
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

// out[i] = in[perm[i]] for the packet arrays and, given the sorted keys (the
// radix sort), the bin ranges: bin_start[b] = first sorted position whose key's
// bin is >= b (b = 0..nbins; keys past the last bin count as bin nbins).  Keys
// are read through key_mask, the bits the sort ordered by, so the bins read
// are nondecreasing even for cells outside the grid (whose keys may be wider
// than the radix sort's bits; those packets then fall in some bin's range,
// where the push flags them).  Each thread moves kGatherItems packets (items
// 256 apart), all its loads issued before its stores.
constexpr int kGatherItems = 4;
constexpr int kGatherTile = 256 * kGatherItems;

template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(
    const uint32_t *__restrict__ perm, int64_t n, const uint32_t *__restrict__ cell_in,
    const T *__restrict__ o0, const T *__restrict__ o1, const T *__restrict__ o2,
    const T *__restrict__ v0, const T *__restrict__ v1, const T *__restrict__ v2,
    const T *__restrict__ w, uint32_t *__restrict__ cell_out, T *__restrict__ p0,
    T *__restrict__ p1, T *__restrict__ p2, T *__restrict__ q0, T *__restrict__ q1,
    T *__restrict__ q2, T *__restrict__ wo, const uint32_t *__restrict__ keys, uint32_t key_mask,
    int shift3, int64_t nbins, uint32_t *__restrict__ bin_start)
{
    const int64_t base = int64_t(blockIdx.x) * kGatherTile + threadIdx.x;
    uint32_t j[kGatherItems], c[kGatherItems];
    T a0[kGatherItems], a1[kGatherItems], a2[kGatherItems], b0[kGatherItems], b1[kGatherItems],
        b2[kGatherItems], ww[kGatherItems];
#pragma unroll
    for (int it = 0; it < kGatherItems; ++it) {
        const int64_t i = base + it * 256;
        j[it] = i < n ? (perm ? perm[i] : uint32_t(i)) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kGatherItems; ++it)
        if (base + it * 256 < n) {
            c[it] = cell_in[j[it]];
            a0[it] = o0[j[it]];
            a1[it] = o1[j[it]];
            a2[it] = o2[j[it]];
            b0[it] = v0[j[it]];
            b1[it] = v1[j[it]];
            b2[it] = v2[j[it]];
            ww[it] = w[j[it]];
        }
#pragma unroll
    for (int it = 0; it < kGatherItems; ++it) {
        const int64_t i = base + it * 256;
        if (i >= n)
            break;
        cell_out[i] = c[it];
        p0[i] = a0[it];
        p1[i] = a1[it];
        p2[i] = a2[it];
        q0[i] = b0[it];
        q1[i] = b1[it];
        q2[i] = b2[it];
        wo[i] = ww[it];
        if (!keys)  // the counting sort records the bin ranges itself
            continue;
        int64_t prev = i == 0 ? -1 : int64_t((keys[i - 1] & key_mask) >> shift3);
        int64_t cur = int64_t((keys[i] & key_mask) >> shift3);
        prev = prev > nbins ? nbins : prev;
        cur = cur > nbins ? nbins : cur;
        for (int64_t b = prev + 1; b <= cur; ++b)
            bin_start[b] = uint32_t(i);
        if (i == n - 1)
            for (int64_t b = cur + 1; b <= nbins; ++b)
                bin_start[b] = uint32_t(n);
    }
}

int gather_grid(int64_t n) { return int((n + kGatherTile - 1) / kGatherTile); }

// ---------------------------------------------------------------------------
// Counting sort by key (the key space is at most a few keys per packet).
// Buckets are the keys 0 .. nkeys-1 plus one bucket nkeys for keys past the
// last bin (from cells outside the grid), which sorts last.
//   1. count_keys_kernel: each packet's key, and the packets per bucket
//      (a run of consecutive lanes with the same bucket adds once).
//   2. bucket_sums_kernel, chunk_scan_kernel (more than 1024 chunks),
//      bucket_scan_kernel: exclusive prefix of the counts, in place:
//      cursor[b] = first output position of bucket b.
//   3. place_kernel: each packet takes the next position of its bucket
//      (one atomic per run of lanes; lanes in lane order).  Afterwards
//      cursor[b] = end of bucket b = start of bucket b + 1.
//   4. The atomics leave each bucket's packets in arbitrary order; sorting
//      each bucket's source indices ascending restores input order among equal
//      keys, which makes the result the unique stable sort.  Buckets of up to
//      16 packets are sorted by one thread with a sorting network, up to
//      kWarpCap by one warp and up to kLongCap by one block, both in shared
//      memory; longer ones in runs of kLongCap merged pairwise in global
//      memory by one block (fix_kernel).  The same kernel records the bin
//      ranges: a bin starts where the bucket of its first key starts.
//   5. gather_kernel moves the packets; the sorted keys are never written.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;  // counters per scan block
constexpr int kFixThreads = 512;
constexpr int kWarpCap = 64;                           // bucket sorted by one warp
constexpr int kLongCap = 8192;                         // bucket sorted in shared memory

__device__ __forceinline__ uint32_t bucket_of(uint32_t key, uint32_t nkeys)
{
    return key < nkeys ? key : nkeys;
}

// Items per thread of the count and placement kernels: a warp takes 32 x
// kPlaceItems consecutive packets, row by row, with all of its loads (and
// atomics) in flight at once.
constexpr int kPlaceItems = 4;
constexpr int kPlaceTile = 256 * kPlaceItems;  // packets per block

template <typename T>
__global__ void __launch_bounds__(256) count_keys_kernel(
    const uint32_t *__restrict__ cell, const T *__restrict__ o0, const T *__restrict__ o1,
    const T *__restrict__ o2, int64_t n, int shape, int nx, int ny, int nz, int lb, int nbx, int nby,
    const int64_t *__restrict__ offsets, const BatchKeyBox *__restrict__ boxes, int n_boxes,
    uint32_t nkeys, uint32_t *__restrict__ keys, uint32_t *__restrict__ count)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kPlaceTile + int64_t(warp) * (32 * kPlaceItems) + lane;
    uint32_t c[kPlaceItems], b[kPlaceItems];
    T f0[kPlaceItems], f1[kPlaceItems], f2[kPlaceItems];
#pragma unroll
    for (int it = 0; it < kPlaceItems; ++it) {  // all loads first
        const int64_t i = base + it * 32;
        const bool ok = i < n;
        c[it] = ok ? cell[i] : 0u;
        f0[it] = ok ? o0[i] : T(0);
        f1[it] = ok ? o1[i] : T(0);
        f2[it] = ok ? o2[i] : T(0);
    }
#pragma unroll
    for (int it = 0; it < kPlaceItems; ++it) {
        const int64_t i = base + it * 32;
        b[it] = 0xffffffffu;  // past the end
        if (i < n) {
            const uint32_t k =
                boxes ? batch_anchor_key(i, c[it], f0[it], f1[it], f2[it], offsets, boxes, n_boxes, shape, lb)
                      : anchor_key(c[it], f0[it], f1[it], f2[it], shape, nx, ny, nz, lb, nbx, nby);
            keys[i] = k;
            b[it] = bucket_of(k, nkeys);
        }
    }
#pragma unroll
    for (int it = 0; it < kPlaceItems; ++it) {
        const LaneRun r = lane_run(b[it], lane);
        if (b[it] != 0xffffffffu && r.first == lane)
            atomicAdd(&count[b[it]], r.len);
    }
}

// Sum of each kScanChunk counters.
__global__ void __launch_bounds__(kScanThreads) bucket_sums_kernel(const uint32_t *__restrict__ count,
                                                                   int64_t nbuckets,
                                                                   uint32_t *__restrict__ sums)
{
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int64_t base = int64_t(blockIdx.x) * kScanChunk;
    uint32_t acc = 0;
    for (int j = threadIdx.x; j < kScanChunk; j += kScanThreads)
        acc += base + j < nbuckets ? count[base + j] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0)
        s_warp[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w)
            t += s_warp[w];
        sums[blockIdx.x] = t;
    }
}

// Exclusive prefix of the chunk sums, in place (one block, any number of
// chunks: tiles of 1024 with a running carry).
__global__ void __launch_bounds__(1024) chunk_scan_kernel(uint32_t *__restrict__ sums, int64_t chunks)
{
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        s_carry = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < chunks; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        const uint32_t v = i < chunks ? sums[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += y;
        }
        if (lane == 31)
            s_warp[warp] = x;
        __syncthreads();
        uint32_t before = s_carry;
        for (int w = 0; w < warp; ++w)
            before += s_warp[w];
        if (i < chunks)
            sums[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1)
            s_carry = before + x;
        __syncthreads();
    }
}

// Exclusive prefix of the counters, in place: this chunk's base plus the
// prefix inside the chunk.  The base is sums[chunk] when the chunk sums were
// scanned (prescanned), else the sum of the chunk sums before it (few chunks).
__global__ void __launch_bounds__(kScanThreads) bucket_scan_kernel(uint32_t *__restrict__ count,
                                                                   int64_t nbuckets,
                                                                   const uint32_t *__restrict__ sums,
                                                                   int prescanned)
{
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (prescanned) {
        if (threadIdx.x == 0)
            s_base = sums[blockIdx.x];
    } else {
        uint32_t before = 0;
        for (int j = threadIdx.x; j < int(blockIdx.x); j += kScanThreads)
            before += sums[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            before += __shfl_xor_sync(0xffffffffu, before, o);
        if (lane == 0)
            s_warp[warp] = before;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kScanThreads / 32; ++w)
                t += s_warp[w];
            s_base = t;
        }
    }
    __syncthreads();
    // thread t owns kScanItems consecutive counters (16-byte loads and stores
    // when all of them exist; the counters start 256-byte aligned)
    static_assert(kScanItems % 4 == 0, "whole 16-byte words per thread");
    const int64_t first = int64_t(blockIdx.x) * kScanChunk + int64_t(threadIdx.x) * kScanItems;
    const bool full = first + kScanItems <= nbuckets;
    uint32_t v[kScanItems];
    uint32_t mine = 0;
    if (full) {
#pragma unroll
        for (int j = 0; j < kScanItems; j += 4) {
            const uint4 x = *reinterpret_cast<const uint4 *>(count + first + j);
            v[j] = x.x;
            v[j + 1] = x.y;
            v[j + 2] = x.z;
            v[j + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j)
            v[j] = first + j < nbuckets ? count[first + j] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        mine += v[j];
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    __syncthreads();  // s_warp is reused
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    uint32_t run = s_base;
    for (int w = 0; w < warp; ++w)
        run += s_warp[w];
    run += incl - mine;
    uint32_t out[kScanItems];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        out[j] = run;
        run += v[j];
    }
    if (full) {
#pragma unroll
        for (int j = 0; j < kScanItems; j += 4)
            *reinterpret_cast<uint4 *>(count + first + j) = make_uint4(out[j], out[j + 1], out[j + 2], out[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j)
            if (first + j < nbuckets)
                count[first + j] = out[j];
    }
}

// Each packet's output position: its bucket's cursor, advanced once per run
// of lanes with the same bucket in a row (the input is close to sorted, so
// equal buckets mostly sit in consecutive lanes); a run takes consecutive
// positions in lane order.  The run detection, the atomics and the stores
// each go over all rows in turn, so that a thread has all its atomics in
// flight.  Only the source index is written: the bin ranges come from the
// counters (fix_kernel), so the sorted keys are not needed.
__global__ void __launch_bounds__(256) place_kernel(const uint32_t *__restrict__ keys_in, int64_t n,
                                                    uint32_t nkeys, uint32_t *__restrict__ cursor,
                                                    uint32_t *__restrict__ idx_out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kPlaceTile + int64_t(warp) * (32 * kPlaceItems) + lane;
    uint32_t b[kPlaceItems], pos[kPlaceItems];
    LaneRun r[kPlaceItems];
#pragma unroll
    for (int it = 0; it < kPlaceItems; ++it) {
        const int64_t i = base + it * 32;
        b[it] = i < n ? bucket_of(keys_in[i], nkeys) : 0xffffffffu;
    }
#pragma unroll
    for (int it = 0; it < kPlaceItems; ++it)
        r[it] = lane_run(b[it], lane);
#pragma unroll
    for (int it = 0; it < kPlaceItems; ++it) {
        pos[it] = 0;
        if (b[it] != 0xffffffffu && r[it].first == lane)
            pos[it] = atomicAdd(&cursor[b[it]], r[it].len);
    }
#pragma unroll
    for (int it = 0; it < kPlaceItems; ++it) {
        pos[it] = __shfl_sync(0xffffffffu, pos[it], r[it].first) + uint32_t(lane - r[it].first);
        const int64_t i = base + it * 32;
        if (i < n)
            idx_out[pos[it]] = uint32_t(i);
    }
}

// Batcher's odd-even merge sort of N (a power of two) values in registers,
// ascending.  The comparators are generated by compile-time recursion (merge
// size P = 1, 2, 4, ..; distance K = P, P/2, .., 1; blocks J from K mod P in
// steps of 2K; I = 0 .. K-1 within a block, where elements I+J and I+J+K lie
// in the same 2P-block), so every array index is a constant and the values
// stay in registers.
template <int N, int P, int K, int J, int I>
__device__ __forceinline__ void net_cmp(uint32_t (&v)[N])
{
    if constexpr (I < K && J + K < N) {
        if constexpr (I + J + K < N && (I + J) / (2 * P) == (I + J + K) / (2 * P)) {
            const uint32_t a = v[I + J], b = v[I + J + K];
            v[I + J] = min(a, b);
            v[I + J + K] = max(a, b);
        }
        net_cmp<N, P, K, J, I + 1>(v);
    }
}
template <int N, int P, int K, int J>
__device__ __forceinline__ void net_j(uint32_t (&v)[N])
{
    if constexpr (J + K < N) {
        net_cmp<N, P, K, J, 0>(v);
        net_j<N, P, K, J + 2 * K>(v);
    }
}
template <int N, int P, int K>
__device__ __forceinline__ void net_k(uint32_t (&v)[N])
{
    if constexpr (K >= 1) {
        net_j<N, P, K, K % P>(v);
        net_k<N, P, K / 2>(v);
    }
}
template <int N, int P>
__device__ __forceinline__ void net_p(uint32_t (&v)[N])
{
    if constexpr (P < N) {
        net_k<N, P, P>(v);
        net_p<N, 2 * P>(v);
    }
}
template <int N>
__device__ __forceinline__ void sort_network(uint32_t (&v)[N])
{
    net_p<N, 1>(v);
}

template <int N>
__device__ __forceinline__ void sort_segment(uint32_t *__restrict__ seg, uint32_t m)
{
    uint32_t v[N];
#pragma unroll
    for (int j = 0; j < N; ++j)
        v[j] = uint32_t(j) < m ? seg[j] : 0xffffffffu;  // padding sorts last
    sort_network<N>(v);
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (uint32_t(j) < m)
            seg[j] = v[j];
}

// Ascending bitonic sort of s[0 .. P) in shared memory (P a power of two),
// by the whole block.
__device__ void block_bitonic(uint32_t *s, int P)
{
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (j - 1));  // lower element of the t-th pair
                const int l = i + j;
                const bool up = (i & k) == 0;
                const uint32_t a = s[i], b = s[l];
                if ((a > b) == up) {
                    s[i] = b;
                    s[l] = a;
                }
            }
            __syncthreads();
        }
}

// Sort src[0 .. m) (m <= kLongCap) into dst[0 .. m) through shared memory.
__device__ void sort_run_shared(const uint32_t *src, uint32_t *dst, int m, uint32_t *s)
{
    int P = 64;
    while (P < m)
        P <<= 1;
    for (int j = threadIdx.x; j < P; j += blockDim.x)
        s[j] = j < m ? src[j] : 0xffffffffu;
    __syncthreads();
    block_bitonic(s, P);
    for (int j = threadIdx.x; j < m; j += blockDim.x)
        dst[j] = s[j];
    __syncthreads();
}

// Merge the sorted runs a[0 .. na) and b[0 .. nb) into out (distinct values):
// each thread finds where its slice of the output splits between a and b
// (a binary search along the diagonal) and merges its slice.
__device__ void block_merge(const uint32_t *a, int64_t na, const uint32_t *b, int64_t nb,
                            uint32_t *out)
{
    constexpr int E = 8;
    const int64_t total = na + nb;
    for (int64_t d = int64_t(threadIdx.x) * E; d < total; d += int64_t(blockDim.x) * E) {
        int64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
        while (lo < hi) {  // first i whose a[i] is not among the first d outputs
            const int64_t mid = (lo + hi) >> 1;
            if (a[mid] < b[d - 1 - mid])
                lo = mid + 1;
            else
                hi = mid;
        }
        int64_t i = lo, j = d - lo;
        const int64_t end = d + E < total ? d + E : total;
        for (int64_t o = d; o < end; ++o) {
            const bool take_a = j >= nb || (i < na && a[i] < b[j]);
            out[o] = take_a ? a[i++] : b[j++];
        }
    }
}

// Bitonic sort of one bucket of up to kWarpCap indices by one warp, in its
// slot ws[0 .. kWarpCap) of shared memory.
__device__ __forceinline__ void warp_sort_bucket(uint32_t *seg, uint32_t m, uint32_t *ws, int lane)
{
    ws[lane] = uint32_t(lane) < m ? seg[lane] : 0xffffffffu;
    ws[lane + 32] = uint32_t(lane + 32) < m ? seg[lane + 32] : 0xffffffffu;
    __syncwarp();
    for (int k = 2; k <= kWarpCap; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int i = 2 * lane - (lane & (j - 1));  // one pair per lane
            const bool up = (i & k) == 0;
            const uint32_t x = ws[i], y = ws[i + j];
            if ((x > y) == up) {
                ws[i] = y;
                ws[i + j] = x;
            }
            __syncwarp();
        }
    if (uint32_t(lane) < m)
        seg[lane] = ws[lane];
    if (uint32_t(lane + 32) < m)
        seg[lane + 32] = ws[lane + 32];
    __syncwarp();
}

// Sort one bucket of m > kWarpCap indices with the whole block: in shared
// memory up to kLongCap, else runs of kLongCap merged pairwise through tmp.
__device__ void block_sort_bucket(uint32_t *seg, uint32_t *alt, int64_t m, uint32_t *s)
{
    for (int64_t r = 0; r < m; r += kLongCap) {
        const int len = int(m - r < kLongCap ? m - r : kLongCap);
        sort_run_shared(seg + r, seg + r, len, s);
    }
    uint32_t *src = seg, *dst = alt;
    for (int64_t w = kLongCap; w < m; w <<= 1) {
        for (int64_t r = 0; r < m; r += 2 * w) {
            const int64_t na = m - r < w ? m - r : w;
            const int64_t nb = m - r - na < w ? m - r - na : w;
            block_merge(src + r, na, src + r + na, nb, dst + r);
        }
        __syncthreads();
        uint32_t *t = src;
        src = dst;
        dst = t;
    }
    if (src != seg) {
        for (int64_t j = threadIdx.x; j < m; j += blockDim.x)
            seg[j] = src[j];
        __syncthreads();
    }
}

// Sort every bucket's source indices ascending, and record the bin ranges.
// Block c takes the chunk of
// kFixThreads buckets from c * kFixThreads (contiguous indices; staged in
// shared memory with coalesced copies when they fit); each thread sorts its
// bucket if it holds up to 16 packets (sorting network in registers), each
// warp sorts its lanes' buckets of up to kWarpCap, and the block then sorts
// the chunk's longer buckets one by one.  tmp has the layout of idx (same
// offsets) and is free while this kernel runs.
__global__ void __launch_bounds__(kFixThreads, 3) fix_kernel(const uint32_t *__restrict__ cursor,
                                                          int64_t nbuckets, uint32_t *__restrict__ idx,
                                                          uint32_t *__restrict__ tmp,
                                                          uint32_t keys_per_bin,
                                                          uint32_t *__restrict__ bin_start)
{
    static_assert((kFixThreads / 32) * kWarpCap <= kLongCap, "warp slots inside the block buffer");
    __shared__ uint32_t s[kLongCap];
    __shared__ uint32_t s_queue[kFixThreads];
    __shared__ uint32_t s_nq;
    __shared__ uint32_t s_span_lo, s_span_hi;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *ws = s + warp * kWarpCap;
    const int64_t chunk = int64_t(blockIdx.x) * kFixThreads;
    const int64_t b = chunk + threadIdx.x;
    uint32_t lo = 0, m = 0;
    if (b < nbuckets) {
        lo = b == 0 ? 0u : cursor[b - 1];
        m = cursor[b] - lo;
    }
    // bin ranges: bin b starts where its first key's bucket starts (the last
    // bucket, past every bin, gives bin_start[nbins])
    if (b < nbuckets && uint32_t(b) % keys_per_bin == 0)
        bin_start[uint32_t(b) / keys_per_bin] = lo;
    // a chunk of empty and one-packet buckets (about one packet per key) has
    // nothing more to do: one barrier decides it for the whole block
    if (__syncthreads_or(m >= 2 && m <= 16)) {
        if (threadIdx.x == 0) {
            // the chunk's buckets are contiguous: [span_lo, span_hi)
            const int64_t last = (chunk + kFixThreads < nbuckets ? chunk + kFixThreads : nbuckets) - 1;
            s_span_lo = chunk == 0 ? 0u : cursor[chunk - 1];
            s_span_hi = cursor[last];
        }
        __syncthreads();
        const uint32_t span_lo = s_span_lo, span = s_span_hi - s_span_lo;
        if (span <= uint32_t(kLongCap)) {
            // short buckets through shared memory: the span in and out coalesced
            for (uint32_t j = threadIdx.x; j < span; j += blockDim.x)
                s[j] = idx[span_lo + j];
            __syncthreads();
            if (m >= 2 && m <= 8)
                sort_segment<8>(s + (lo - span_lo), m);
            else if (m > 8 && m <= 16)
                sort_segment<16>(s + (lo - span_lo), m);
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < span; j += blockDim.x)
                idx[span_lo + j] = s[j];
            __syncthreads();  // s is reused below
        } else if (m >= 2 && m <= 8) {
            sort_segment<8>(idx + lo, m);
        } else if (m > 8 && m <= 16) {
            sort_segment<16>(idx + lo, m);
        }
    }
    uint32_t mid = __ballot_sync(0xffffffffu, m > 16 && m <= kWarpCap);
    while (mid) {
        const int src = __ffs(mid) - 1;
        mid &= mid - 1;
        const uint32_t lo_s = __shfl_sync(0xffffffffu, lo, src);
        const uint32_t m_s = __shfl_sync(0xffffffffu, m, src);
        warp_sort_bucket(idx + lo_s, m_s, ws, lane);
    }
    // (also the barrier after the warp sorts, whose slots the block sorts reuse)
    if (__syncthreads_or(m > kWarpCap)) {
        if (threadIdx.x == 0)
            s_nq = 0;
        __syncthreads();
        if (m > kWarpCap)
            s_queue[atomicAdd(&s_nq, 1u)] = uint32_t(b);
        __syncthreads();
        const uint32_t nq = s_nq;
        for (uint32_t e = 0; e < nq; ++e) {
            const uint32_t bb = s_queue[e];
            const uint32_t lo_b = bb == 0 ? 0u : cursor[bb - 1];
            block_sort_bucket(idx + lo_b, tmp + lo_b, int64_t(cursor[bb]) - lo_b, s);
        }
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
                       int64_t nbins, cudaStream_t st)
{
    cudaError_t e;
    const int64_t nb = blocks_for(n);
    // the passes order by the low ceil(key_bits / 8) * 8 bits
    const int sorted_bits = (key_bits + 7) / 8 * 8;
    const uint32_t radix_mask = sorted_bits >= 32 ? 0xffffffffu : (1u << sorted_bits) - 1u;
    int cur = 0;
    for (int shift = 0; shift < key_bits; shift += 8) {
        upsweep_kernel<<<unsigned(nb), SORT_THREADS, 0, st>>>(s.keys[cur], n, shift, s.counts, nb);
        row_scan_kernel<<<RADIX, 1024, 0, st>>>(s.counts, nb, s.block_sums);
        digit_base_kernel<<<1, RADIX, 0, st>>>(s.block_sums);
        downsweep_kernel<<<unsigned(nb), SORT_THREADS, 0, st>>>(
            s.keys[cur], shift == 0 ? nullptr : s.idx[cur], n, shift, s.counts, nb, s.block_sums,
            s.keys[cur ^ 1], s.idx[cur ^ 1]);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        cur ^= 1;
    }
    if (elem_bytes == 4)
        gather_kernel<float><<<gather_grid(n), 256, 0, st>>>(
            key_bits > 0 ? s.idx[cur] : nullptr, n, cell_in, static_cast<const float *>(off_in[0]),
            static_cast<const float *>(off_in[1]), static_cast<const float *>(off_in[2]),
            static_cast<const float *>(u_in[0]), static_cast<const float *>(u_in[1]),
            static_cast<const float *>(u_in[2]), static_cast<const float *>(w_in), cell_out,
            static_cast<float *>(off_out[0]), static_cast<float *>(off_out[1]),
            static_cast<float *>(off_out[2]), static_cast<float *>(u_out[0]),
            static_cast<float *>(u_out[1]), static_cast<float *>(u_out[2]),
            static_cast<float *>(w_out), s.keys[cur], radix_mask, 3 * lb, nbins, s.bin_start);
    else
        gather_kernel<double><<<gather_grid(n), 256, 0, st>>>(
            key_bits > 0 ? s.idx[cur] : nullptr, n, cell_in, static_cast<const double *>(off_in[0]),
            static_cast<const double *>(off_in[1]), static_cast<const double *>(off_in[2]),
            static_cast<const double *>(u_in[0]), static_cast<const double *>(u_in[1]),
            static_cast<const double *>(u_in[2]), static_cast<const double *>(w_in), cell_out,
            static_cast<double *>(off_out[0]), static_cast<double *>(off_out[1]),
            static_cast<double *>(off_out[2]), static_cast<double *>(u_out[0]),
            static_cast<double *>(u_out[1]), static_cast<double *>(u_out[2]),
            static_cast<double *>(w_out), s.keys[cur], radix_mask, 3 * lb, nbins, s.bin_start);
    return cudaGetLastError();
}

bool count_sort_applies(int64_t n, int64_t nkeys)
{
    return nkeys >= 2 && nkeys <= (int64_t(1) << 26) && nkeys <= 2 * n;
}

int count_sort_launches(int64_t nkeys)
{
    const int64_t chunks = (nkeys + 1 + kScanChunk - 1) / kScanChunk;
    return chunks > 1024 ? 7 : 6;
}

size_t count_scratch_bytes(int64_t n, int64_t nkeys)
{
    const int64_t nbuckets = nkeys + 1;
    const int64_t chunks = (nbuckets + kScanChunk - 1) / kScanChunk;
    return align_up(size_t(nbuckets) * 4) + align_up(size_t(chunks) * 4);
}

void count_scratch_carve(void *base, int64_t n, int64_t nkeys, CountScratch *c)
{
    char *p = static_cast<char *>(base);
    const int64_t nbuckets = nkeys + 1;
    c->cursor = reinterpret_cast<uint32_t *>(p);
    p += align_up(size_t(nbuckets) * 4);
    c->sums = reinterpret_cast<uint32_t *>(p);
    c->nbuckets = nbuckets;
    c->capacity = n;
}

cudaError_t count_sort_particles(const SortScratch &s, const CountScratch &c, int64_t n,
                                 int elem_bytes, const uint32_t *cell_in, void *const off_in[3],
                                 void *const u_in[3], const void *w_in, uint32_t *cell_out,
                                 void *const off_out[3], void *const u_out[3], void *w_out, int nx,
                                 int ny, int nz, int bin, int shape, int key_bits, int64_t nbins,
                                 cudaStream_t st,
                                 const int64_t *d_offsets, const BatchKeyBox *d_boxes,
                                 int n_boxes)
{
    int lb = 0;
    while ((1 << lb) < bin)
        ++lb;
    const int nbx = (nx + bin - 1) / bin, nby = (ny + bin - 1) / bin;
    const uint32_t nkeys = uint32_t(c.nbuckets - 1);
    const int fin = ((key_bits + 7) / 8) & 1;  // where the radix sort leaves its result
    uint32_t *keys_in = s.keys[fin ^ 1];
    cudaError_t e = cudaMemsetAsync(c.cursor, 0, size_t(c.nbuckets) * 4, st);
    if (e != cudaSuccess)
        return e;
    const unsigned gt = unsigned((n + kPlaceTile - 1) / kPlaceTile);
    if (elem_bytes == 4)
        count_keys_kernel<float><<<gt, 256, 0, st>>>(
            cell_in, static_cast<const float *>(off_in[0]), static_cast<const float *>(off_in[1]),
            static_cast<const float *>(off_in[2]), n, shape, nx, ny, nz, lb, nbx, nby, d_offsets,
            d_boxes, n_boxes, nkeys, keys_in, c.cursor);
    else
        count_keys_kernel<double><<<gt, 256, 0, st>>>(
            cell_in, static_cast<const double *>(off_in[0]), static_cast<const double *>(off_in[1]),
            static_cast<const double *>(off_in[2]), n, shape, nx, ny, nz, lb, nbx, nby, d_offsets,
            d_boxes, n_boxes, nkeys, keys_in, c.cursor);
    const unsigned chunks = unsigned((c.nbuckets + kScanChunk - 1) / kScanChunk);
    bucket_sums_kernel<<<chunks, kScanThreads, 0, st>>>(c.cursor, c.nbuckets, c.sums);
    // many chunks: scan their sums in one block first (summing the predecessors
    // in every block would cost chunks^2 / 2 loads)
    const int prescan = chunks > 1024 ? 1 : 0;
    if (prescan)
        chunk_scan_kernel<<<1, 1024, 0, st>>>(c.sums, chunks);
    bucket_scan_kernel<<<chunks, kScanThreads, 0, st>>>(c.cursor, c.nbuckets, c.sums, prescan);
    place_kernel<<<gt, 256, 0, st>>>(keys_in, n, nkeys, c.cursor, s.idx[fin]);
    const int64_t fix_chunks = (c.nbuckets + kFixThreads - 1) / kFixThreads;
    fix_kernel<<<unsigned(fix_chunks), kFixThreads, 0, st>>>(
        c.cursor, c.nbuckets, s.idx[fin], s.idx[fin ^ 1], 1u << (3 * lb), s.bin_start);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if (elem_bytes == 4)
        gather_kernel<float><<<gather_grid(n), 256, 0, st>>>(
            s.idx[fin], n, cell_in, static_cast<const float *>(off_in[0]),
            static_cast<const float *>(off_in[1]), static_cast<const float *>(off_in[2]),
            static_cast<const float *>(u_in[0]), static_cast<const float *>(u_in[1]),
            static_cast<const float *>(u_in[2]), static_cast<const float *>(w_in), cell_out,
            static_cast<float *>(off_out[0]), static_cast<float *>(off_out[1]),
            static_cast<float *>(off_out[2]), static_cast<float *>(u_out[0]),
            static_cast<float *>(u_out[1]), static_cast<float *>(u_out[2]),
            static_cast<float *>(w_out), nullptr, 0xffffffffu, 3 * lb, nbins, s.bin_start);
    else
        gather_kernel<double><<<gather_grid(n), 256, 0, st>>>(
            s.idx[fin], n, cell_in, static_cast<const double *>(off_in[0]),
            static_cast<const double *>(off_in[1]), static_cast<const double *>(off_in[2]),
            static_cast<const double *>(u_in[0]), static_cast<const double *>(u_in[1]),
            static_cast<const double *>(u_in[2]), static_cast<const double *>(w_in), cell_out,
            static_cast<double *>(off_out[0]), static_cast<double *>(off_out[1]),
            static_cast<double *>(off_out[2]), static_cast<double *>(u_out[0]),
            static_cast<double *>(u_out[1]), static_cast<double *>(u_out[2]),
            static_cast<double *>(w_out), nullptr, 0xffffffffu, 3 * lb, nbins, s.bin_start);
    return cudaGetLastError();
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
