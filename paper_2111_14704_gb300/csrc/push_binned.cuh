// Binned push kernel: one CTA per sort bin of B^3 anchor nodes.
//
// The packets of a bin are contiguous after rsol_sort (keyed on the anchor
// node of their stencil: the cell for CIC, the nearest node for TSC), so the
// CTA stages the E, B tile of its bin plus a two-node halo in shared memory,
// and deposits into a shared-memory tile that is added to the global grid
// once at the end.  Per warp and batch of 32 packets:
//   phase 1, one packet per lane: weights, gather from the tile, Boris,
//            feedback densities, drift; the packet's stencil weights and its
//            eight densities are staged per warp.
//   phase 2, one stencil offset per lane (TSC: 27 lanes x 8 quantities;
//            CIC: 8 offsets x 4 pairs of quantities): walk the runs of equal
//            stencil origin along the lanes (equal anchors are adjacent after
//            the sort), accumulate W * Q in registers and add the run's sum
//            to the tile once per run.
// Before the batches, a histogram pass over the bin's packets sets the tile's
// fixed-point scale and, once drift since the sort has broken the origin order,
// a counting sort local to the CTA gives the order the batches visit.
// Packets whose stencil leaves the tile (they drifted more than a node since
// the sort) take the order-free path: gather from global memory and deposit
// with global atomics.  Results equal the order-free kernel's up to the order
// of floating-point additions (bitwise run to run in deterministic mode).
#pragma once

#include <type_traits>

#include "push.cuh"
#include "tma.cuh"

namespace rsol {

// Bins with at most this many packets skip the shared-memory tiles: staging
// and flushing a (B + 4)^3 tile then costs more than the packets' own global
// gathers and atomics (measured on the batch of 512 boxes, sparse bins one
// warp each: the crossover lies near 0.45 packets per tile node).
template <int B>
__host__ __device__ constexpr uint32_t sparse_bin_limit()
{
    return B == 8 ? 768u : 256u;
}

struct BinGeom {
    const uint32_t *bin_start;
    int nbx, nby, nbz;
};

template <typename T, int SHAPE, int B, int NW, bool DET>
struct BinnedCfg {
    static constexpr int NP = SHAPE == 1 ? 2 : 3;   // stencil nodes per axis
    static constexpr int NS = NP * NP * NP;         // stencil nodes
    static constexpr int TE = B + 4;                // tile edge in nodes, origin at bin origin - 2
    static constexpr int RS = TE;                   // row stride (dense: one bulk tensor copy)
    static constexpr int PS = TE * RS;              // plane stride
    static constexpr int TN = TE * PS;              // tile slots
    // deposit-tile element: 64-bit fixed point (deterministic mode), 32-bit
    // fixed point with a per-CTA scale (FP32: native integer shared atomics are
    // ~3.5x faster than emulated float ones), or double (FP64)
    static constexpr bool I32 = !DET && sizeof(T) == 4;
    using Acc = typename std::conditional<DET, long long,
                                          typename std::conditional<I32, int, T>::type>::type;
    // the deposit tile, and everything keyed by a packet's stencil origin (the
    // origin histogram, the kept keys, the local sort, the run walk), has its own
    // strides: padded so that the 27 stencil lanes of a TSC flush hit 27
    // distinct banks with 4-byte elements (the dense field-tile strides put the
    // z = 0 and z = 2 planes on the same banks)
    static constexpr int DRS = sizeof(Acc) == 4 ? (TE == 12 ? 14 : (TE == 8 ? 11 : RS)) : RS;
    static constexpr int DPS = sizeof(Acc) == 4 ? (TE == 12 ? 171 : (TE == 8 ? 89 : PS)) : PS;
    static constexpr int DTN = TE * DPS;
    static constexpr size_t fields_bytes = size_t(TN) * 8 * sizeof(T);   // [slot][8]: E, B, 2 unused
    static constexpr size_t dep_bytes = size_t(DTN) * 8 * sizeof(Acc);   // [q][slot]
    // per warp: stencil weights W[32][WS] and densities + origin QO[32][12]
    static constexpr int WS = NS == 27 ? 28 : NS;   // weight rows padded to 16-byte stores
    static constexpr int QO = 12;                   // 48-byte rows: conflict-free 16-byte stores
    static constexpr size_t stage_words = 32 * (WS + QO);
    static constexpr size_t stage_bytes = size_t(NW) * stage_words * sizeof(T);
    // 32-bit fixed point: the stencil-origin key of each of the bin's first KEYCAP
    // packets, kept from the histogram pass for the local sort
    static constexpr int KEYCAP = I32 ? 8192 : 0;
    static constexpr size_t key_bytes = size_t(KEYCAP) * sizeof(uint16_t);
    // the field tile is the destination of a bulk tensor copy: 128-byte
    // aligned, so the dynamic allocation carries up to 128 bytes of padding
    static constexpr size_t align_pad = 128;
    static constexpr size_t smem_bytes = align_pad + fields_bytes + dep_bytes + stage_bytes + key_bytes;
};

__device__ __forceinline__ int wrap_mod(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// v periodic in [0, n) for v in [-n, 2n)
__device__ __forceinline__ int wrap_once(int v, int n)
{
    v += v < 0 ? n : 0;
    return v - (v >= n ? n : 0);
}

// Anchor node and stencil data of one axis: returns the anchor (periodic) and
// the first stencil node offset relative to the anchor; w[] are the weights of
// the stencil nodes first, first+1, first+2 (relative to the anchor).
template <int SHAPE, typename T>
__device__ __forceinline__ int anchor_axis(int i, T f, int n, T w[3], int &first_rel)
{
    const int first = axis_weights<SHAPE>(f, w);  // relative to the cell
    if (SHAPE == 1) {
        first_rel = 0;
        return i;
    }
    // TSC: anchor = cell + (first + 1); stencil starts one node below it
    first_rel = -1;
    int j = i + first + 1;
    j -= (j >= n) ? n : 0;
    return j;
}

// Tile-local stencil-origin slot of a packet (cell c, offsets f0..f2) for the
// tile whose first node is (ox, oy, oz): lz * PS + ly * RS + lx, or TN when the
// packet is off the grid or its stencil leaves the tile.
template <int SHAPE, int TE, int RS, int PS, int TN, typename T>
__device__ __forceinline__ int origin_slot(uint32_t c, T f0, T f1, T f2, int ox, int oy, int oz,
                                           int nx, int ny, int nz)
{
    constexpr int NP = SHAPE == 1 ? 2 : 3;
    const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
    if (ix >= nx || iy >= ny || iz >= nz)
        return TN;
    T w3[3];
    int rx, ry, rz;
    const int jx = anchor_axis<SHAPE>(ix, f0, nx, w3, rx);
    const int jy = anchor_axis<SHAPE>(iy, f1, ny, w3, ry);
    const int jz = anchor_axis<SHAPE>(iz, f2, nz, w3, rz);
    const int lx = wrap_once(jx + rx - ox, nx), ly = wrap_once(jy + ry - oy, ny),
              lz = wrap_once(jz + rz - oz, nz);
    return lx + NP <= TE && ly + NP <= TE && lz + NP <= TE ? lz * PS + ly * RS + lx : TN;
}

__device__ __forceinline__ void lds_node(const float *p, float F[6])
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float2 b = *reinterpret_cast<const float2 *>(p + 4);
    F[0] = a.x; F[1] = a.y; F[2] = a.z; F[3] = a.w; F[4] = b.x; F[5] = b.y;
}
__device__ __forceinline__ void lds_node(const double *p, double F[6])
{
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    const double2 c = *reinterpret_cast<const double2 *>(p + 4);
    F[0] = a.x; F[1] = a.y; F[2] = b.x; F[3] = b.y; F[4] = c.x; F[5] = c.y;
}

// E, B of one node into a tile slot of 8 elements (16-byte stores)
__device__ __forceinline__ void sts_node(float *p, const float F[6])
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(F[0], F[1], F[2], F[3]);
    reinterpret_cast<float2 *>(p)[2] = make_float2(F[4], F[5]);
}
__device__ __forceinline__ void sts_node(double *p, const double F[6])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(F[0], F[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(F[2], F[3]);
    reinterpret_cast<double2 *>(p)[2] = make_double2(F[4], F[5]);
}

__device__ __forceinline__ void store_q8(float *p, const float Q[8])
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(Q[0], Q[1], Q[2], Q[3]);
    reinterpret_cast<float4 *>(p)[1] = make_float4(Q[4], Q[5], Q[6], Q[7]);
}
__device__ __forceinline__ void store_q8(double *p, const double Q[8])
{
#pragma unroll
    for (int q = 0; q < 8; q += 2)
        reinterpret_cast<double2 *>(p)[q / 2] = make_double2(Q[q], Q[q + 1]);
}
// one packet's stencil weights into its padded staging row (16-byte stores)
template <int WS, int NS>
__device__ __forceinline__ void store_wrow(float *p, const float (&W)[NS])
{
#pragma unroll
    for (int k = 0; k < WS; k += 4)
        reinterpret_cast<float4 *>(p)[k / 4] =
            make_float4(W[k], k + 1 < NS ? W[k + 1] : 0.f, k + 2 < NS ? W[k + 2] : 0.f,
                        k + 3 < NS ? W[k + 3] : 0.f);
}
template <int WS, int NS>
__device__ __forceinline__ void store_wrow(double *p, const double (&W)[NS])
{
#pragma unroll
    for (int k = 0; k < WS; k += 2)
        reinterpret_cast<double2 *>(p)[k / 2] = make_double2(W[k], k + 1 < NS ? W[k + 1] : 0.0);
}

// the N densities of a phase-2 lane role, starting at p (N = 8: all; N = 2: a pair)
template <int N>
__device__ __forceinline__ void load_qpart(const float *p, float Q[N])
{
    if constexpr (N == 8) {
        const float4 a = reinterpret_cast<const float4 *>(p)[0];
        const float4 b = reinterpret_cast<const float4 *>(p)[1];
        Q[0] = a.x; Q[1] = a.y; Q[2] = a.z; Q[3] = a.w; Q[4] = b.x; Q[5] = b.y; Q[6] = b.z; Q[7] = b.w;
    } else {
        const float2 a = *reinterpret_cast<const float2 *>(p);
        Q[0] = a.x; Q[1] = a.y;
    }
}
template <int N>
__device__ __forceinline__ void load_qpart(const double *p, double Q[N])
{
#pragma unroll
    for (int q = 0; q < N; q += 2) {
        const double2 v = reinterpret_cast<const double2 *>(p)[q / 2];
        Q[q] = v.x;
        Q[q + 1] = v.y;
    }
}

__device__ __forceinline__ void load_q8(const float *p, float Q[8])
{
    const float4 a = reinterpret_cast<const float4 *>(p)[0];
    const float4 b = reinterpret_cast<const float4 *>(p)[1];
    Q[0] = a.x; Q[1] = a.y; Q[2] = a.z; Q[3] = a.w; Q[4] = b.x; Q[5] = b.y; Q[6] = b.z; Q[7] = b.w;
}
__device__ __forceinline__ void load_q8(const double *p, double Q[8])
{
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        const double2 v = reinterpret_cast<const double2 *>(p)[q / 2];
        Q[q] = v.x;
        Q[q + 1] = v.y;
    }
}

// L2 prefetch of elements [lo, hi) of p: one 128-byte line per thread and pass;
// every address issued is that of an element of the range.
template <typename E>
__device__ __forceinline__ void prefetch_l2(const E *p, uint32_t lo, uint32_t hi)
{
    if (lo >= hi)
        return;
    const uintptr_t s = reinterpret_cast<uintptr_t>(p + lo), e = reinterpret_cast<uintptr_t>(p + hi);
    for (uintptr_t l = (s & ~uintptr_t(127)) + uintptr_t(threadIdx.x) * 128; l < e;
         l += uintptr_t(blockDim.x) * 128) {
        const uintptr_t addr = l < s ? s : l;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(addr));
    }
}

// Exclusive prefix sum of the origin histogram hist[0..TN) of a CTA of NW warps
// into cursor[] (each origin's first position in origin order); *s_out = the
// packets counted, i.e. the first position after them.  Ends synchronised.
template <int NW, int TN>
__device__ __forceinline__ void origin_cursors(const int *hist, int *cursor, int *s_out)
{
    __shared__ int s_wsum[NW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int CH = (TN + NW * 32 - 1) / (NW * 32);
    const int t0 = int(threadIdx.x) * CH;
    int vals[CH];
    int tsum = 0;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
        vals[u] = t0 + u < TN ? hist[t0 + u] : 0;
        tsum += vals[u];
    }
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        incl += lane >= o ? v : 0;
    }
    if (lane == 31)
        s_wsum[warp] = incl;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w)
        wbase += s_wsum[w];
    if (threadIdx.x == blockDim.x - 1)
        *s_out = wbase + incl;
    int run = wbase + incl - tsum;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
        if (t0 + u < TN)
            cursor[t0 + u] = run;
        run += vals[u];
    }
    __syncthreads();
}

// Largest total weight any node of a tile can receive from the packets counted
// in hist (packets per tile-local stencil origin, slot z PS + y RS + x): the
// sum over the stencil origins around the node of (packets at the origin) x
// (largest axis weights for that offset: CIC 1, 1; TSC 1/2, 3/4, 1/2 per
// axis).  The weights are per-axis products, so the sum is three 3-tap passes
// along x, y and z, one tile row per thread and pass; exact in float (the terms
// are small integers times products of 1/2 and 3/4).  scratch holds 2 TE^3
// floats.  Returns this thread's largest node value (reduce over the CTA);
// ends with scratch still in use by no thread, but without a final barrier.
template <int SHAPE, int TE, int RS, int PS, int NW>
__device__ __forceinline__ float tile_weight_bound(const int *hist, float *scratch)
{
    constexpr int NP = SHAPE == 1 ? 2 : 3;
    constexpr int TT = TE * TE * TE;
    float *g1 = scratch, *g2 = scratch + TT;  // [z][y][x], TE each
    auto tap = [](int c) { return SHAPE == 1 ? 1.f : (c == 1 ? 0.75f : 0.5f); };
    for (int r = threadIdx.x; r < TE * TE; r += blockDim.x) {  // along x: rows (z, y)
        const int y = r % TE, z = r / TE;
        float h[TE];
#pragma unroll
        for (int x = 0; x < TE; ++x)
            h[x] = float(hist[z * PS + y * RS + x]);
#pragma unroll
        for (int x = 0; x < TE; ++x) {
            float v = 0.f;
#pragma unroll
            for (int c = 0; c < NP; ++c)
                v += x >= c ? tap(c) * h[x - c] : 0.f;
            g1[(z * TE + y) * TE + x] = v;
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < TE * TE; r += blockDim.x) {  // along y: rows (z, x)
        const int x = r % TE, z = r / TE;
        float h[TE];
#pragma unroll
        for (int y = 0; y < TE; ++y)
            h[y] = g1[(z * TE + y) * TE + x];
#pragma unroll
        for (int y = 0; y < TE; ++y) {
            float v = 0.f;
#pragma unroll
            for (int c = 0; c < NP; ++c)
                v += y >= c ? tap(c) * h[y - c] : 0.f;
            g2[(z * TE + y) * TE + x] = v;
        }
    }
    __syncthreads();
    float gmax = 0.f;
    for (int r = threadIdx.x; r < TE * TE; r += blockDim.x) {  // along z: rows (y, x)
        const int x = r % TE, y = r / TE;
        float h[TE];
#pragma unroll
        for (int z = 0; z < TE; ++z)
            h[z] = g2[(z * TE + y) * TE + x];
#pragma unroll
        for (int z = 0; z < TE; ++z) {
            float v = 0.f;
#pragma unroll
            for (int c = 0; c < NP; ++c)
                v += z >= c ? tap(c) * h[z - c] : 0.f;
            gmax = fmaxf(gmax, v);
        }
    }
    return gmax;
}

// The work of one CTA on one bin: packets [lo, hi) of the bin whose anchors
// were in bin (bx, by, bz) of the box described by a at the last sort.
template <typename T, int SHAPE, int B, int NW, bool DET>
__device__ __forceinline__ void binned_cta(const PushArgs<T> &a, uint32_t lo, uint32_t hi,
                                           int bx, int by, int bz,
                                           const CUtensorMap *tmap = nullptr)
{
    using Cfg = BinnedCfg<T, SHAPE, B, NW, DET>;
    using Acc = typename Cfg::Acc;
    constexpr bool F2 = std::is_same<T, float>::value;  // f32x2 gather and deposit
    constexpr int TE = Cfg::TE, RS = Cfg::RS, PS = Cfg::PS;          // field tile
    constexpr int DRS = Cfg::DRS, DPS = Cfg::DPS, DTN = Cfg::DTN;  // deposit tile, origin keys
    constexpr int NP = Cfg::NP, NS = Cfg::NS, WS = Cfg::WS, QO = Cfg::QO;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((Cfg::align_pad - (smem_addr(smem_raw) & (Cfg::align_pad - 1))) &
                                      (Cfg::align_pad - 1));
    T *sf = reinterpret_cast<T *>(smem);
    Acc *sd = reinterpret_cast<Acc *>(smem + Cfg::fields_bytes);
    T *stage = reinterpret_cast<T *>(smem + Cfg::fields_bytes + Cfg::dep_bytes);
    uint16_t *s_key = reinterpret_cast<uint16_t *>(smem + Cfg::fields_bytes + Cfg::dep_bytes +
                                                   Cfg::stage_bytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *sW = stage + warp * Cfg::stage_words;  // [32][WS]
    T *sQ = sW + 32 * WS;                     // [32][QO]: Q[0..7]

    if (lo >= hi)
        return;
    if (hi - lo <= sparse_bin_limit<B>()) {
        // few packets: staging and flushing the tiles would cost more than the
        // packets' own global-memory gathers and atomics
        int sflag = 0;
        auto gather_global = [&](int64_t node, T F[6]) { load_node(a.fields + node * 8, F); };
        auto deposit_global = [&](int64_t node, T W, const T Q[8]) {
            if (DET)
                red_node_fixed(a.fx + node * 8, W, Q, a.fx_scale);
            else
                red_node(a.fb + node * 8, W, Q);
        };
        for (uint32_t j = lo + threadIdx.x; j < hi; j += blockDim.x)
            push_one<T, SHAPE, true>(a, int64_t(j), gather_global, deposit_global, &sflag);
        if (sflag)
            atomicOr(a.status, sflag);
        return;
    }
    const int ox = bx * B - 2, oy = by * B - 2, oz = bz * B - 2;
    // A tile that does not wrap around the periodic grid on any axis is one box
    // of the field grid: one bulk tensor copy (TMA) issued by thread 0 lands it
    // while the threads make the origin histogram below.  FP32 only, with the
    // tensor map the host encoded for this field grid.
    constexpr int TT = TE * TE * TE;
    const bool tma = Cfg::I32 && tmap != nullptr && ox >= 0 && oy >= 0 && oz >= 0 &&
                     ox + TE <= a.nx && oy + TE <= a.ny && oz + TE <= a.nz;
    __shared__ uint64_t s_tma_bar;
    if (tma && threadIdx.x == 0)
        mbar_init(&s_tma_bar, 1);
    // grid offsets of the tile's rows along each axis (periodic): node of tile
    // point (lx, ly, lz) = s_axis[lx] + s_axis[TE + ly] + s_axis[2 TE + lz]
    __shared__ int s_axis[3 * TE];
    if (threadIdx.x < 3 * TE) {
        const int ax = threadIdx.x / TE, l = threadIdx.x % TE;
        const int o = ax == 0 ? ox : (ax == 1 ? oy : oz);
        const int n = ax == 0 ? a.nx : (ax == 1 ? a.ny : a.nz);
        const int stride = ax == 0 ? 1 : (ax == 1 ? a.nx : a.nx * a.ny);
        s_axis[threadIdx.x] = wrap_mod(o + l, n) * stride;
    }
    __syncthreads();

    // stage the field tile (periodic) and clear the deposit tile; track the
    // largest |E| and, per axis a, the largest |B| across a (B with its a
    // component removed) of the tile for the fixed-point scale
    T e2max = T(0), bp2max[3] = {T(0), T(0), T(0)};
    auto field_bounds = [&](const T F[6]) {
        e2max = fmax(e2max, F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
        const T bx2 = F[3] * F[3], by2 = F[4] * F[4], bz2 = F[5] * F[5];
        bp2max[0] = fmax(bp2max[0], by2 + bz2);
        bp2max[1] = fmax(bp2max[1], bx2 + bz2);
        bp2max[2] = fmax(bp2max[2], bx2 + by2);
    };
    if (tma && threadIdx.x == 0) {
        mbar_arrive_expect_tx(&s_tma_bar, uint32_t(TT * 8 * sizeof(T)));
        tma_load_4d(sf, tmap, 0, ox, oy, oz, &s_tma_bar);
    }
    constexpr int UF = 4;  // nodes per thread per pass: all loads issued first
    for (int t0 = threadIdx.x; !tma && t0 < TT; t0 += UF * blockDim.x) {
        T F[UF][6];
#pragma unroll
        for (int u = 0; u < UF; ++u) {
            const int t = t0 + u * int(blockDim.x);
            if (t < TT) {
                const int lx = t % TE, ly = (t / TE) % TE, lz = t / (TE * TE);
                const int node = s_axis[lx] + s_axis[TE + ly] + s_axis[2 * TE + lz];
                load_node(a.fields + int64_t(node) * 8, F[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < UF; ++u) {
            const int t = t0 + u * int(blockDim.x);
            if (t < TT) {
                const int lx = t % TE, ly = (t / TE) % TE, lz = t / (TE * TE);
                const int slot = lz * PS + ly * RS + lx;
                sts_node(sf + slot * 8, F[u]);
                field_bounds(F[u]);
            }
        }
    }
    // clear the whole deposit tile, padding slots included (the origin histogram
    // below reads every slot)
    for (int t = threadIdx.x; t < 8 * DTN; t += blockDim.x)
        sd[t] = Acc(0);
    // 32-bit fixed point: scale_q = 2^e with (packets in bin) * Wmax * bound_q
    // below 2^30, bound_q a bound on one packet's |Q_q| (|beta_bar| < 1):
    //   rho: w q / dx^3;  J: rho c;  S_a: rho (|E| + |B across a|), since
    //   |(beta_bar x B)_a| <= |beta_bar| |B with its a component removed|;
    //   H: rho c |E| (1 + h |E|)
    __shared__ float s_scale[8], s_iscale[8];  // 32-bit fixed point: 2^e and 2^-e per density
    __shared__ int s_local_sorted;  // 1: phase 1 visits the packets in a.perm order
    if (threadIdx.x == 0)
        s_local_sorted = 0;
    if (Cfg::I32) {
        // packets per stencil origin (histogram in the zeroed deposit tile): a node
        // receives from at most NS origins, so NS * (largest origin count) bounds
        // the packets that reach any one node
        // It also counts descents of the origin along the packet order (lanes
        // against their left neighbour): a bin still in the order of the last
        // global sort needs no local sort below.
        __shared__ int s_desc;
        if (threadIdx.x == 0)
            s_desc = 0;
        __syncthreads();
        int *hist = reinterpret_cast<int *>(sd);
        T wmax = T(0);
        int desc = 0;
        constexpr int U = 4;  // packets per thread per pass: all loads issued first
        for (uint32_t jb = lo; jb < hi; jb += U * blockDim.x) {  // warp-uniform trip count
            const uint32_t j0 = jb + threadIdx.x;
            uint32_t cc[U];
            T f0[U], f1[U], f2[U], ww[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = j0 + uint32_t(u) * blockDim.x;
                const bool ok = j < hi;
                cc[u] = ok ? a.cell[j] : 0xFFFFFFFFu;
                f0[u] = ok ? a.off0[j] : T(0);
                f1[u] = ok ? a.off1[j] : T(0);
                f2[u] = ok ? a.off2[j] : T(0);
                ww[u] = ok ? a.w[j] : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                wmax = fmax(wmax, fabs(ww[u]));
                // out of the tile or off the grid: DTN, which sorts last
                const int key = origin_slot<SHAPE, TE, DRS, DPS, DTN>(cc[u], f0[u], f1[u], f2[u], ox,
                                                                      oy, oz, a.nx, a.ny, a.nz);
                if (key < DTN)
                    atomicAdd(&hist[key], 1);
                {
                    const uint32_t jr = j0 + uint32_t(u) * blockDim.x - lo;  // rank in the bin
                    if (jr < hi - lo && jr < uint32_t(Cfg::KEYCAP))
                        s_key[jr] = uint16_t(key);
                }
                const int prev = __shfl_up_sync(0xffffffffu, key, 1);
                desc += (lane > 0 && j0 + uint32_t(u) * blockDim.x < hi && key < prev) ? 1 : 0;
            }
        }
        desc = __reduce_add_sync(0xffffffffu, desc);
        if (lane == 0 && desc)
            atomicAdd(&s_desc, desc);
        __syncthreads();
        // largest weight a node can receive in total (this thread's share)
        static_assert(Cfg::stage_bytes >= 2 * size_t(TT) * sizeof(float), "stage too small");
        float gmax = tile_weight_bound<SHAPE, TE, DRS, DPS, NW>(hist, reinterpret_cast<float *>(stage));
        __syncthreads();
        // sort locally once more than one packet in 32 breaks the origin order
        if (a.perm && s_desc * 32 > int(hi - lo)) {
            // counting sort of the bin's packets by stencil origin (local to the
            // CTA): the histogram gives each origin's first position, and phase 1
            // then visits the packets origin by origin, so a phase-2 run spans
            // a whole origin however far the packets drifted since the last
            // global sort.  Out-of-tile and off-grid packets go last.
            int *cursor = reinterpret_cast<int *>(stage);  // free until the batches
            if (threadIdx.x == 0)
                s_local_sorted = 1;
            __shared__ int s_out;
            origin_cursors<NW, DTN>(hist, cursor, &s_out);
            if (hi - lo <= uint32_t(Cfg::KEYCAP)) {  // keys kept from the histogram pass
                for (uint32_t jr = threadIdx.x; jr < hi - lo; jr += blockDim.x) {
                    const int key = s_key[jr];
                    const int pos = key < DTN ? atomicAdd(&cursor[key], 1) : atomicAdd(&s_out, 1);
                    a.perm[lo + uint32_t(pos)] = lo + jr;
                }
            } else {
                for (uint32_t j0 = lo + threadIdx.x; j0 < hi; j0 += U * blockDim.x) {
                    uint32_t cc[U];
                    T f0[U], f1[U], f2[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const uint32_t j = j0 + uint32_t(u) * blockDim.x;
                        const bool ok = j < hi;
                        cc[u] = ok ? a.cell[j] : 0xFFFFFFFFu;
                        f0[u] = ok ? a.off0[j] : T(0);
                        f1[u] = ok ? a.off1[j] : T(0);
                        f2[u] = ok ? a.off2[j] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const uint32_t j = j0 + uint32_t(u) * blockDim.x;
                        if (j >= hi)
                            continue;
                        const int slot = origin_slot<SHAPE, TE, DRS, DPS, DTN>(
                            cc[u], f0[u], f1[u], f2[u], ox, oy, oz, a.nx, a.ny, a.nz);
                        const int pos = slot < DTN ? atomicAdd(&cursor[slot], 1) : atomicAdd(&s_out, 1);
                        a.perm[lo + uint32_t(pos)] = j;
                    }
                }
            }
            __syncthreads();
        }
        for (int t = threadIdx.x; t < DTN; t += blockDim.x)
            hist[t] = 0;
        if (tma) {
            // the bulk copy: wait for it (bounded), then the field bounds from the tile
            const bool arrived = mbar_wait_bounded(&s_tma_bar, 0, kTmaWaitCycles);
            if (!__syncthreads_and(arrived)) {
                // report it, give the copy one more bounded wait, skip the bin
                if (threadIdx.x == 0) {
                    atomicOr(a.status, ST_TIMEOUT);
                    mbar_wait_bounded(&s_tma_bar, 0, kTmaWaitCycles);
                }
                __syncthreads();
                return;
            }
            for (int t = threadIdx.x; t < TT; t += blockDim.x) {
                T F[6];
                lds_node(sf + t * 8, F);
                field_bounds(F);
            }
        }
        __shared__ T s_red[5][NW];
        __shared__ float s_gmax[NW];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e2max = fmax(e2max, __shfl_xor_sync(0xffffffffu, e2max, o));
#pragma unroll
            for (int a = 0; a < 3; ++a)
                bp2max[a] = fmax(bp2max[a], __shfl_xor_sync(0xffffffffu, bp2max[a], o));
            wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
            gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        }
        if (lane == 0) {
            s_red[0][warp] = e2max;
            s_red[1][warp] = wmax;
            s_red[2][warp] = bp2max[0];
            s_red[3][warp] = bp2max[1];
            s_red[4][warp] = bp2max[2];
            s_gmax[warp] = gmax;
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            const int q = threadIdx.x;
            const int bp = q >= 4 && q < 7 ? 2 + (q - 4) : 2;  // S_q: |B| across axis q - 4
            T em = T(0), bm = T(0), wm = T(0);
            float gm = 0.f;
            for (int w = 0; w < NW; ++w) {
                em = fmax(em, s_red[0][w]);
                wm = fmax(wm, s_red[1][w]);
                bm = fmax(bm, s_red[bp][w]);
                gm = fmaxf(gm, s_gmax[w]);
            }
            em = Math<T>::sqrt(em);
            bm = Math<T>::sqrt(bm);
            const T rho = wm * fabs(a.k.qv);
            T bound = q == 0 ? rho
                    : q < 4  ? rho * a.k.c
                    : q < 7  ? rho * (em + bm)
                             : rho * a.k.c * em * (T(1) + fabs(a.k.h) * em);
            bound *= T(gm > 1.f ? gm : 1.f);
            int e = 30;
            if (bound > T(0) && isfinite(bound))
                e = 30 - int(ceilf(log2f(float(bound))));
            e = e > 60 ? 60 : (e < -60 ? -60 : e);
            s_scale[q] = ldexpf(1.0f, e);
            s_iscale[q] = ldexpf(1.0f, -e);
        }
    }
    __syncthreads();

    // phase-2 lane role: stencil offset and quantity range [q0, q0 + 2 or 8)
    const int off_id = SHAPE == 1 ? (lane & 7) : (lane < 27 ? lane : 0);
    const bool p2_active = SHAPE == 1 ? true : lane < 27;
    const int pax = off_id % NP, pay = (off_id / NP) % NP, paz = off_id / (NP * NP);
    const int q0 = SHAPE == 1 ? 2 * (lane >> 3) : 0;
    const int lane_off = paz * DPS + pay * DRS + pax;

    int flag = 0;
    // each warp walks a contiguous slice of the bin, so a run of equal stencil
    // origin that straddles two batches is carried over instead of flushed twice
    const uint32_t n_bin = hi - lo;
    const uint32_t per_warp = ((n_bin + NW - 1) / NW + 31) & ~31u;
    const uint32_t w_lo = lo + per_warp * uint32_t(warp);
    const uint32_t w_hi = w_lo + per_warp < hi ? w_lo + per_warp : hi;
    int carry_origin = -1;
    constexpr int NQ_ = SHAPE == 1 ? 2 : 8;
    T acc[NQ_];
#pragma unroll
    for (int q = 0; q < NQ_; ++q)
        acc[q] = T(0);
    f32x2 acc2[NQ_ / 2];  // FP32: the densities in pairs (f32x2 arithmetic)
#pragma unroll
    for (int q = 0; q < NQ_ / 2; ++q)
        acc2[q] = 0;
    auto flush_acc = [&](int origin) {
        if (p2_active && origin >= 0) {
            const int t = origin + lane_off;
            if constexpr (F2) {
#pragma unroll
                for (int q = 0; q < NQ_ / 2; ++q)
                    f2_unpack(acc2[q], acc[2 * q], acc[2 * q + 1]);
            }
#pragma unroll
            for (int q = 0; q < NQ_; ++q) {
                if (DET)
                    atomicAdd(reinterpret_cast<unsigned long long *>(&sd[(q0 + q) * DTN + t]),
                              static_cast<unsigned long long>(to_fixed(acc[q] * a.fx_scale)));
                else if (Cfg::I32)
                    atomicAdd(reinterpret_cast<int *>(&sd[(q0 + q) * DTN + t]),
                              __float2int_rn(float(acc[q])));  // densities staged pre-scaled
                else
                    atomicAdd(reinterpret_cast<T *>(&sd[(q0 + q) * DTN + t]), acc[q]);
            }
        }
    };
    // software pipeline: the packet fields of batch k+1 are loaded into
    // registers while batch k is pushed and deposited
    // (with the local sort, position jj of the bin holds packet perm[jj])
    const bool use_perm = Cfg::I32 && s_local_sorted != 0;
    uint32_t n_c = 0, n_j = 0;
    T n_o[3] = {T(0), T(0), T(0)}, n_u[3] = {T(0), T(0), T(0)}, n_w = T(0);
    auto prefetch = [&](uint32_t jj) {
        if (jj < w_hi) {
            const uint32_t jp = use_perm ? a.perm[jj] : jj;
            n_j = jp;
            n_c = a.cell[jp];
            n_o[0] = a.off0[jp];
            n_o[1] = a.off1[jp];
            n_o[2] = a.off2[jp];
            n_u[0] = a.u0[jp];
            n_u[1] = a.u1[jp];
            n_u[2] = a.u2[jp];
            n_w = a.w[jp];
        }
    };
    prefetch(w_lo + uint32_t(lane));
    for (uint32_t base = w_lo; base < w_hi; base += 32) {
        const uint32_t j = base + uint32_t(lane);
        const uint32_t c = n_c;
        T fx = n_o[0], fy = n_o[1], fz = n_o[2];
        const T u0[3] = {n_u[0], n_u[1], n_u[2]};
        const T wj = n_w;
        const uint32_t jp = n_j;  // the packet at sorted position j
        prefetch(j + 32);
        int staged = -1;
        if (j < w_hi) {
            const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
            if (ix >= a.nx || iy >= a.ny || iz >= a.nz) {
                flag |= ST_BADCELL;
            } else {
                T wx[3], wy[3], wz[3];
                int rx, ry, rz;
                const int jx = anchor_axis<SHAPE>(ix, fx, a.nx, wx, rx);
                const int jy = anchor_axis<SHAPE>(iy, fy, a.ny, wy, ry);
                const int jz = anchor_axis<SHAPE>(iz, fz, a.nz, wz, rz);
                // tile-local stencil origin
                int lx = jx + rx - ox, ly = jy + ry - oy, lz = jz + rz - oz;
                lx += lx < 0 ? a.nx : 0;
                ly += ly < 0 ? a.ny : 0;
                lz += lz < 0 ? a.nz : 0;
                lx -= lx >= a.nx ? a.nx : 0;
                ly -= ly >= a.ny ? a.ny : 0;
                lz -= lz >= a.nz ? a.nz : 0;
                const bool in_tile = lx >= 0 && ly >= 0 && lz >= 0 && lx + NP <= TE &&
                                     ly + NP <= TE && lz + NP <= TE;
                T E[3] = {T(0), T(0), T(0)}, Bf[3] = {T(0), T(0), T(0)};
                T Wk[NS];
#pragma unroll
                for (int cz = 0; cz < NP; ++cz)
#pragma unroll
                    for (int cy = 0; cy < NP; ++cy) {
                        const T wyz = wy[cy] * wz[cz];
#pragma unroll
                        for (int cx = 0; cx < NP; ++cx)
                            Wk[(cz * NP + cy) * NP + cx] = wx[cx] * wyz;
                    }
                int kx[3], ky[3], kz[3];
                if (in_tile) {
                    const int s0 = lz * PS + ly * RS + lx;
                    if constexpr (F2) {
                        // pairs {Ex, Ey}, {Ez, Bx}, {By, Bz}: a node is one 16-byte
                        // and one 8-byte load and three paired multiply-adds
                        f32x2 g01 = 0, g23 = 0, g45 = 0;  // +0.0f in both halves
#pragma unroll
                        for (int cz = 0; cz < NP; ++cz)
#pragma unroll
                            for (int cy = 0; cy < NP; ++cy)
#pragma unroll
                                for (int cx = 0; cx < NP; ++cx) {
                                    const float W = Wk[(cz * NP + cy) * NP + cx];
                                    const f32x2 W2 = f2_pack(W, W);
                                    const float *p = sf + (s0 + cz * PS + cy * RS + cx) * 8;
                                    const ulonglong2 a2 = *reinterpret_cast<const ulonglong2 *>(p);
                                    const f32x2 b2 = *reinterpret_cast<const f32x2 *>(p + 4);
                                    g01 = f2_fma(W2, a2.x, g01);
                                    g23 = f2_fma(W2, a2.y, g23);
                                    g45 = f2_fma(W2, b2, g45);
                                }
                        f2_unpack(g01, E[0], E[1]);
                        f2_unpack(g23, E[2], Bf[0]);
                        f2_unpack(g45, Bf[1], Bf[2]);
                    } else {
#pragma unroll
                        for (int cz = 0; cz < NP; ++cz)
#pragma unroll
                            for (int cy = 0; cy < NP; ++cy)
#pragma unroll
                                for (int cx = 0; cx < NP; ++cx) {
                                    const T W = Wk[(cz * NP + cy) * NP + cx];
                                    T F[6];
                                    lds_node(sf + (s0 + cz * PS + cy * RS + cx) * 8, F);
#pragma unroll
                                    for (int q = 0; q < 3; ++q) {
                                        E[q] += W * F[q];
                                        Bf[q] += W * F[3 + q];
                                    }
                                }
                    }
                    staged = lz * DPS + ly * DRS + lx;
                } else {
                    axis_nodes(jx, rx, a.nx, kx);
                    axis_nodes(jy, ry, a.ny, ky);
                    axis_nodes(jz, rz, a.nz, kz);
#pragma unroll
                    for (int cz = 0; cz < NP; ++cz)
#pragma unroll
                        for (int cy = 0; cy < NP; ++cy) {
                            const int64_t row = (int64_t(kz[cz]) * a.ny + ky[cy]) * a.nx;
#pragma unroll
                            for (int cx = 0; cx < NP; ++cx) {
                                const T W = Wk[(cz * NP + cy) * NP + cx];
                                T F[6];
                                load_node(a.fields + (row + kx[cx]) * 8, F);
#pragma unroll
                                for (int q = 0; q < 3; ++q) {
                                    E[q] += W * F[q];
                                    Bf[q] += W * F[3 + q];
                                }
                            }
                        }
                }
                const BorisOut<T> b = boris(a.k.h, E, Bf, u0);
                const T g0 = Math<T>::sqrt(T(1) + dot3(u0, u0));
                T Q[8];
                feedback(a.k, wj, E, Bf, b, g0, Q);
                if (in_tile) {
                    store_wrow<WS>(sW + lane * WS, Wk);
                    if (Cfg::I32) {  // the tile's fixed-point scale (a power of two: exact)
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            Q[q] *= T(s_scale[q]);
                    }
                    store_q8(sQ + lane * QO, Q);
                } else {
#pragma unroll
                    for (int cz = 0; cz < NP; ++cz)
#pragma unroll
                        for (int cy = 0; cy < NP; ++cy) {
                            const int64_t row = (int64_t(kz[cz]) * a.ny + ky[cy]) * a.nx;
#pragma unroll
                            for (int cx = 0; cx < NP; ++cx) {
                                const T W = Wk[(cz * NP + cy) * NP + cx];
                                if (DET)
                                    red_node_fixed(a.fx + (row + kx[cx]) * 8, W, Q, a.fx_scale);
                                else
                                    red_node(a.fb + (row + kx[cx]) * 8, W, Q);
                            }
                        }
                }
                if (Math<T>::finite(b.u1[0]) && Math<T>::finite(b.u1[1]) &&
                    Math<T>::finite(b.u1[2])) {
                    const T s = a.k.adv * b.inv_g1;
                    const int nx_ = drift_axis(ix, fx, s * b.u1[0], a.nx, &flag);
                    const int ny_ = drift_axis(iy, fy, s * b.u1[1], a.ny, &flag);
                    const int nz_ = drift_axis(iz, fz, s * b.u1[2], a.nz, &flag);
                    a.cell[jp] = pack_cell(nx_, ny_, nz_);
                    a.off0[jp] = fx;
                    a.off1[jp] = fy;
                    a.off2[jp] = fz;
                    a.u0[jp] = b.u1[0];
                    a.u1[jp] = b.u1[1];
                    a.u2[jp] = b.u1[2];
                } else {
                    flag |= ST_NONFINITE;
                }
            }
        }
        // runs of equal stencil origin along the lanes (the sorted order; equal
        // origin = same stencil nodes); a lane with no staged packet (-1: out of
        // the tile, or past the slice) starts a run that phase 2 skips
        const int left = __shfl_up_sync(0xffffffffu, staged, 1);
        const uint32_t starts = __ballot_sync(0xffffffffu, lane == 0 || staged != left);
        __syncwarp();

        // phase 2: stencil-offset lanes sum each run in registers (two packets per
        // pass) and add the sum to the tile when the origin changes (runs continue
        // across batches); all control below is warp-uniform
        uint32_t st = starts;
        while (st) {
            const int L = __ffs(st) - 1;
            st &= st - 1;
            const int R = st ? __ffs(st) - 1 : 32;
            const int origin = __shfl_sync(0xffffffffu, staged, L);
            if (origin < 0) {
                flush_acc(carry_origin);
                carry_origin = origin;
                continue;
            }
            const T *wrow = sW + L * WS + off_id;
            const T *qrow = sQ + L * QO + q0;
            int p = L;
            if constexpr (F2) {
                // densities in pairs: a packet is one weight load, two (TSC) or
                // one (CIC) 16/8-byte density loads and NQ/2 paired multiply-adds
                auto qpairs = [&](const float *qp, f32x2 (&Q2)[NQ_ / 2]) {
                    if constexpr (NQ_ == 8) {
                        const ulonglong2 x = reinterpret_cast<const ulonglong2 *>(qp)[0];
                        const ulonglong2 y = reinterpret_cast<const ulonglong2 *>(qp)[1];
                        Q2[0] = x.x; Q2[1] = x.y; Q2[2] = y.x; Q2[3] = y.y;
                    } else {
                        Q2[0] = *reinterpret_cast<const f32x2 *>(qp);
                    }
                };
                if (origin != carry_origin) {  // a new run: its first packet starts the sums
                    flush_acc(carry_origin);
                    carry_origin = origin;
                    const f32x2 W2 = f2_pack(wrow[0], wrow[0]);
                    f32x2 Q2[NQ_ / 2];
                    qpairs(qrow, Q2);
#pragma unroll
                    for (int q = 0; q < NQ_ / 2; ++q)
                        acc2[q] = f2_mul(W2, Q2[q]);
                    ++p;
                    wrow += WS;
                    qrow += QO;
                }
                for (; p + 1 < R; p += 2, wrow += 2 * WS, qrow += 2 * QO) {
                    const f32x2 Wa = f2_pack(wrow[0], wrow[0]), Wb = f2_pack(wrow[WS], wrow[WS]);
                    f32x2 Qa[NQ_ / 2], Qb[NQ_ / 2];
                    qpairs(qrow, Qa);
                    qpairs(qrow + QO, Qb);
#pragma unroll
                    for (int q = 0; q < NQ_ / 2; ++q) {
                        acc2[q] = f2_fma(Wa, Qa[q], acc2[q]);
                        acc2[q] = f2_fma(Wb, Qb[q], acc2[q]);
                    }
                }
                if (p < R) {
                    const f32x2 W2 = f2_pack(wrow[0], wrow[0]);
                    f32x2 Q2[NQ_ / 2];
                    qpairs(qrow, Q2);
#pragma unroll
                    for (int q = 0; q < NQ_ / 2; ++q)
                        acc2[q] = f2_fma(W2, Q2[q], acc2[q]);
                }
            } else {
                if (origin != carry_origin) {  // a new run: its first packet starts the sums
                    flush_acc(carry_origin);
                    carry_origin = origin;
                    const T W = wrow[0];
                    T Qp[NQ_];
                    load_qpart<NQ_>(qrow, Qp);
#pragma unroll
                    for (int q = 0; q < NQ_; ++q)
                        acc[q] = W * Qp[q];
                    ++p;
                    wrow += WS;
                    qrow += QO;
                }
                for (; p + 1 < R; p += 2, wrow += 2 * WS, qrow += 2 * QO) {
                    const T W = wrow[0], W2 = wrow[WS];
                    T Qp[NQ_], Qp2[NQ_];
                    load_qpart<NQ_>(qrow, Qp);
                    load_qpart<NQ_>(qrow + QO, Qp2);
#pragma unroll
                    for (int q = 0; q < NQ_; ++q) {
                        acc[q] += W * Qp[q];
                        acc[q] += W2 * Qp2[q];
                    }
                }
                if (p < R) {
                    const T W = wrow[0];
                    T Qp[NQ_];
                    load_qpart<NQ_>(qrow, Qp);
#pragma unroll
                    for (int q = 0; q < NQ_; ++q)
                        acc[q] += W * Qp[q];
                }
            }
        }
        __syncwarp();
    }
    flush_acc(carry_origin);
    __syncthreads();

    // add the deposit tile to the global grid (skip untouched nodes)
    for (int t = threadIdx.x; t < TE * TE * TE; t += blockDim.x) {
        const int lx = t % TE, ly = (t / TE) % TE, lz = t / (TE * TE);
        const int slot = lz * DPS + ly * DRS + lx;
        const int64_t node = s_axis[lx] + s_axis[TE + ly] + s_axis[2 * TE + lz];
        if (DET) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const long long v = sd[q * DTN + slot];
                if (v != 0)
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.fx + node * 8 + q),
                              static_cast<unsigned long long>(v));
            }
        } else {
            T v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                v[q] = Cfg::I32 ? T(float(sd[q * DTN + slot]) * s_iscale[q]) : T(sd[q * DTN + slot]);
            if (sizeof(T) == 4) {
                float *p = reinterpret_cast<float *>(a.fb) + node * 8;
                if (v[0] != T(0) || v[1] != T(0) || v[2] != T(0) || v[3] != T(0))
                    atomicAdd(reinterpret_cast<float4 *>(p),
                              make_float4(float(v[0]), float(v[1]), float(v[2]), float(v[3])));
                if (v[4] != T(0) || v[5] != T(0) || v[6] != T(0) || v[7] != T(0))
                    atomicAdd(reinterpret_cast<float4 *>(p + 4),
                              make_float4(float(v[4]), float(v[5]), float(v[6]), float(v[7])));
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (v[q] != T(0))
                        atomicAdd(reinterpret_cast<double *>(a.fb) + node * 8 + q, double(v[q]));
            }
        }
    }
    if (flag)
        atomicOr(a.status, flag);
    if (tma && threadIdx.x == 0)  // every thread waited on it before the batches
        mbar_inval(&s_tma_bar);
}

template <typename T, int SHAPE, int B, int NW, bool DET>
__global__ void __launch_bounds__(NW * 32)
    push_binned_kernel(PushArgs<T> a, BinGeom g, int ahead, const __grid_constant__ CUtensorMap tmap,
                       int use_tma)
{
    const int bin = blockIdx.x;
    const int bx = bin % g.nbx, by = (bin / g.nbx) % g.nby, bz = bin / (g.nbx * g.nby);
    // the bin that starts about one wave of CTAs later: its packets into L2 now
    if (bin + ahead < int(gridDim.x)) {
        const uint32_t plo = g.bin_start[bin + ahead], phi = g.bin_start[bin + ahead + 1];
        prefetch_l2(a.cell, plo, phi);
        prefetch_l2(a.off0, plo, phi);
        prefetch_l2(a.off1, plo, phi);
        prefetch_l2(a.off2, plo, phi);
        prefetch_l2(a.u0, plo, phi);
        prefetch_l2(a.u1, plo, phi);
        prefetch_l2(a.u2, plo, phi);
        prefetch_l2(a.w, plo, phi);
    }
    binned_cta<T, SHAPE, B, NW, DET>(a, g.bin_start[bin], g.bin_start[bin + 1], bx, by, bz,
                                     use_tma ? &tmap : nullptr);
}

// One box of a batch: grid, node offset into the concatenated grids, first
// global bin, and its step constants (c~ and dt differ between boxes).
template <typename T>
struct BatchBox {
    int nx, ny, nz, nbx, nby, nbz;
    int64_t node_off;
    uint32_t bin_base;
    StepConst<T> k;
};

// Box of global bin gb: the last box whose first bin is <= gb.
template <typename T>
__device__ __forceinline__ int batch_box_of(const BatchBox<T> *__restrict__ boxes, int n_boxes,
                                            uint32_t gb)
{
    int lo_b = 0, hi_b = n_boxes - 1;
    while (lo_b < hi_b) {
        const int mid = (lo_b + hi_b + 1) >> 1;
        if (boxes[mid].bin_base <= gb)
            lo_b = mid;
        else
            hi_b = mid - 1;
    }
    return lo_b;
}

// The batch's push arguments narrowed to one box: its geometry, constants and
// slices of the concatenated grids.
template <typename T>
__device__ __forceinline__ PushArgs<T> batch_box_args(const PushArgs<T> &base, const BatchBox<T> &bx_)
{
    PushArgs<T> a = base;
    a.nx = bx_.nx;
    a.ny = bx_.ny;
    a.nz = bx_.nz;
    a.k = bx_.k;
    a.fields = base.fields + bx_.node_off * 8;
    a.fb = base.fb ? base.fb + bx_.node_off * 8 : nullptr;
    a.fx = base.fx ? base.fx + bx_.node_off * 8 : nullptr;
    return a;
}

// Work area of a batch push (device, 3 + total_bins words): claim counters,
// zeroed before each push, and the list of the dense bins of this push.
constexpr int kClaimSparse = 0;  // next bin a warp of the sparse kernel claims
constexpr int kDenseCount = 1;   // dense bins listed by the sparse kernel
constexpr int kClaimDense = 2;   // next list entry a CTA of the tiled kernel claims
constexpr int kDenseList = 3;    // the list itself (at most total_bins entries)

// The sparse bins of a batch (at most sparse_bin_limit packets): one warp per
// bin, each lane one packet at a time, gathering from global memory and
// depositing with global vector atomics.  Independent warps in small CTAs
// keep more gathers and atomics in flight than the tiled kernel's CTAs, which
// would stall a whole CTA on each sparse bin.  Warps claim the bins in order
// from a counter (a bin's cost follows its packet count, so a fixed share per
// warp would leave some warps with several large bins); a dense bin is only
// listed for the tiled kernel.  Each bin is claimed once, so the list holds at
// most total_bins entries.
constexpr int kSparseWarps = 4;
template <typename T, int SHAPE, int B, bool DET>
__global__ void __launch_bounds__(kSparseWarps * 32) push_batch_sparse_kernel(
    PushArgs<T> base, const BatchBox<T> *__restrict__ boxes, int n_boxes,
    const uint32_t *__restrict__ bin_start, uint32_t total_bins, uint32_t *work)
{
    const int lane = threadIdx.x & 31;
    int sflag = 0;
    uint32_t next = 0;
    if (lane == 0)
        next = atomicAdd(&work[kClaimSparse], 1u);
    uint32_t gb = __shfl_sync(0xffffffffu, next, 0);
    while (gb < total_bins) {
        if (lane == 0)  // the next claim is in flight while this bin is pushed
            next = atomicAdd(&work[kClaimSparse], 1u);
        const uint32_t lo = bin_start[gb], hi = bin_start[gb + 1];
        if (hi - lo > sparse_bin_limit<B>()) {
            if (lane == 0)
                work[kDenseList + atomicAdd(&work[kDenseCount], 1u)] = gb;
        } else if (lo < hi) {
            const PushArgs<T> a = batch_box_args(base, boxes[batch_box_of(boxes, n_boxes, gb)]);
            auto gather_global = [&](int64_t node, T F[6]) { load_node(a.fields + node * 8, F); };
            auto deposit_global = [&](int64_t node, T W, const T Q[8]) {
                if (DET)
                    red_node_fixed(a.fx + node * 8, W, Q, a.fx_scale);
                else
                    red_node(a.fb + node * 8, W, Q);
            };
            for (uint32_t j = lo + uint32_t(lane); j < hi; j += 32)
                push_one<T, SHAPE, true>(a, int64_t(j), gather_global, deposit_global, &sflag);
        }
        gb = __shfl_sync(0xffffffffu, next, 0);
    }
    if (sflag)
        atomicOr(base.status, sflag);
}

// Persistent kernel over the dense bins the sparse kernel listed: CTAs claim
// list entries from a counter (dynamic balance: a dense bin holds from just
// over sparse_bin_limit to tens of thousands of packets); each bin is processed by the same
// CTA body as the single-box kernel, with its box's geometry, grids and
// constants.
template <typename T, int SHAPE, int B, int NW, bool DET>
__global__ void __launch_bounds__(NW * 32) push_batch_kernel(PushArgs<T> base,
                                                             const BatchBox<T> *__restrict__ boxes,
                                                             int n_boxes,
                                                             const uint32_t *__restrict__ bin_start,
                                                             uint32_t *work)
{
    __shared__ uint32_t s_gb;
    const uint32_t n_dense = work[kDenseCount];  // complete: the sparse kernel ran before
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t i = atomicAdd(&work[kClaimDense], 1u);
            s_gb = i < n_dense ? work[kDenseList + i] : 0xFFFFFFFFu;
        }
        __syncthreads();
        const uint32_t gb = s_gb;
        if (gb == 0xFFFFFFFFu)
            break;  // block-uniform
        const int ib = batch_box_of(boxes, n_boxes, gb);
        const BatchBox<T> bx_ = boxes[ib];
        PushArgs<T> a = batch_box_args(base, bx_);
        const int lb = int(gb - bx_.bin_base);
        const int bx = lb % bx_.nbx, by = (lb / bx_.nbx) % bx_.nby, bz = lb / (bx_.nbx * bx_.nby);
        binned_cta<T, SHAPE, B, NW, DET>(a, bin_start[gb], bin_start[gb + 1], bx, by, bz);
        __syncthreads();  // the next bin reuses the shared tiles and s_gb
    }
}

// Warps per CTA: as many as the shared-memory budget allows (at most 16, a
// multiple of 4); 0 when even four warps do not fit (the order-free kernel runs).
template <typename T, int SHAPE, int B, bool DET>
constexpr int binned_warps()
{
    using C0 = BinnedCfg<T, SHAPE, B, 0, DET>;
    constexpr size_t budget = 232448 - 1024;  // leave room for static shared memory
    constexpr size_t fixed = C0::align_pad + C0::fields_bytes + C0::dep_bytes + C0::key_bytes;
    constexpr size_t per_warp = C0::stage_words * sizeof(T);
    constexpr size_t fit = fixed >= budget ? 0 : (budget - fixed) / per_warp;
    constexpr int cap = DET ? 8 : 16;  // deterministic kernels need more registers
    constexpr int nw = int(fit > size_t(cap) ? size_t(cap) : fit) & ~3;
    return nw;
}

// Tensor map of a node-major FP32 field grid (eight components per node)
// whose box is one bin's tile of te^3 nodes; false (no bulk copies: the tiles
// are staged with ordinary loads) when the driver does not provide the encoder,
// the grid is smaller than a tile or the grid is not 16-byte aligned.
inline bool encode_field_tile_map(CUtensorMap *map, const void *fields, int nx, int ny, int nz, int te)
{
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static const Encode encode = []() -> Encode {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<Encode>(f);
    }();
    if (!encode || (reinterpret_cast<uintptr_t>(fields) & 15u) || nx < te || ny < te || nz < te)
        return false;
    const cuuint64_t dims[4] = {8, cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(nz)};
    const cuuint64_t strides[3] = {32, 32ull * uint64_t(nx), 32ull * uint64_t(nx) * uint64_t(ny)};
    const cuuint32_t box[4] = {8, cuuint32_t(te), cuuint32_t(te), cuuint32_t(te)};
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(fields), dims, strides,
                  box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, int SHAPE, int B, bool DET, int NW>
cudaError_t launch_binned_nw(const PushArgs<T> &a, const BinGeom &g, int nbins, int sm_count,
                             cudaStream_t s)
{
    using Cfg = BinnedCfg<T, SHAPE, B, NW, DET>;
    static_assert(Cfg::smem_bytes <= 232448, "binned tile exceeds shared memory");
    auto kern = push_binned_kernel<T, SHAPE, B, NW, DET>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(Cfg::smem_bytes));
    if (e != cudaSuccess)
        return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, Cfg::smem_bytes);
    if (e != cudaSuccess)
        return e;
    const int wave = sm_count * (per_sm > 0 ? per_sm : 1);  // CTAs resident at a time
    // FP32 tiles: interior bins take their fields with one bulk tensor copy
    CUtensorMap map{};
    const int use_tma = Cfg::I32 && encode_field_tile_map(&map, a.fields, a.nx, a.ny, a.nz, Cfg::TE);
    kern<<<nbins, NW * 32, Cfg::smem_bytes, s>>>(a, g, wave, map, use_tma);
    return cudaGetLastError();
}

// The binned kernel with the requested CTA width: 8 warps, or (0, 16) the
// widest that fits shared memory; the order-free kernel if not even 4 fit.
template <typename T, int SHAPE, int B, bool DET>
cudaError_t launch_binned(const PushArgs<T> &a, const BinGeom &g, int nbins, int sm_count, int warps,
                          cudaStream_t s)
{
    constexpr int NW = binned_warps<T, SHAPE, B, DET>();
    if constexpr (NW < 4) {
        return launch_unbinned<T, SHAPE, true, DET>(a, sm_count, s);
    } else if constexpr (NW > 8) {
        if (warps == 8)
            return launch_binned_nw<T, SHAPE, B, DET, 8>(a, g, nbins, sm_count, s);
        return launch_binned_nw<T, SHAPE, B, DET, NW>(a, g, nbins, sm_count, s);
    } else {
        return launch_binned_nw<T, SHAPE, B, DET, NW>(a, g, nbins, sm_count, s);
    }
}

template <typename T>
cudaError_t push_binned_dispatch(const PushDesc &d, cudaStream_t s)
{
    const PushArgs<T> a = make_push_args<T>(d);
    BinGeom g{d.bin_start, d.nbx, d.nby, d.nbz};
    const int nbins = d.nbx * d.nby * d.nbz;
    const bool det = d.det != 0;
#define RSOL_BINNED(SH, BB)                                                                  \
    return det ? launch_binned<T, SH, BB, true>(a, g, nbins, d.sm_count, d.warps, s)        \
               : launch_binned<T, SH, BB, false>(a, g, nbins, d.sm_count, d.warps, s)
    if (d.shape == 1) {
        if (d.bin == 4) { RSOL_BINNED(1, 4); }
        RSOL_BINNED(1, 8);
    }
    if (d.bin == 4) { RSOL_BINNED(2, 4); }
    RSOL_BINNED(2, 8);
#undef RSOL_BINNED
}

template <typename T, int SHAPE, int B, bool DET, int NWREQ>
cudaError_t launch_batch(const PushArgs<T> &a, const BatchBox<T> *boxes, int n_boxes,
                         const uint32_t *bin_start, uint32_t total_bins, uint32_t *work,
                         int sm_count, cudaStream_t s)
{
    constexpr int NWMAX = binned_warps<T, SHAPE, B, DET>();
    constexpr int NW = NWREQ < NWMAX ? NWREQ : NWMAX;
    if constexpr (NW < 4) {
        return cudaErrorInvalidConfiguration;
    } else {
        using Cfg = BinnedCfg<T, SHAPE, B, NW, DET>;
        auto kern = push_batch_kernel<T, SHAPE, B, NW, DET>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(Cfg::smem_bytes));
        if (e != cudaSuccess)
            return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, Cfg::smem_bytes);
        if (e != cudaSuccess)
            return e;
        uint32_t grid = uint32_t(sm_count) * uint32_t(per_sm > 0 ? per_sm : 1);
        if (grid > total_bins)
            grid = total_bins > 0 ? total_bins : 1;
        // the sparse bins first (one warp per bin; the dense ones listed), then the
        // dense ones
        e = cudaMemsetAsync(work, 0, kDenseList * sizeof(uint32_t), s);
        if (e != cudaSuccess)
            return e;
        auto sk = push_batch_sparse_kernel<T, SHAPE, B, DET>;
        int sp_per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sp_per_sm, sk, kSparseWarps * 32, 0);
        if (e != cudaSuccess)
            return e;
        uint64_t sgrid = uint64_t(sm_count) * uint64_t(sp_per_sm > 0 ? sp_per_sm : 1);
        const uint64_t sgrid_max = (uint64_t(total_bins) + kSparseWarps - 1) / kSparseWarps;
        if (sgrid > sgrid_max)
            sgrid = sgrid_max > 0 ? sgrid_max : 1;
        sk<<<unsigned(sgrid), kSparseWarps * 32, 0, s>>>(a, boxes, n_boxes, bin_start, total_bins, work);
        kern<<<grid, NW * 32, Cfg::smem_bytes, s>>>(a, boxes, n_boxes, bin_start, work);
        return cudaGetLastError();
    }
}

template <typename T>
cudaError_t push_batch_dispatch(const PushDesc &d, const void *boxes, int n_boxes,
                                uint32_t total_bins, int warps, uint32_t *work, cudaStream_t s)
{
    const PushArgs<T> a = make_push_args<T>(d);
    const BatchBox<T> *bx = static_cast<const BatchBox<T> *>(boxes);
    const bool det = d.det != 0;
    const bool w8 = warps == 8;
#define RSOL_BATCH(SH, BB)                                                                 \
    if (det)                                                                              \
        return w8 ? launch_batch<T, SH, BB, true, 8>(a, bx, n_boxes, d.bin_start, total_bins, work, d.sm_count, s) \
                  : launch_batch<T, SH, BB, true, 16>(a, bx, n_boxes, d.bin_start, total_bins, work, d.sm_count, s); \
    return w8 ? launch_batch<T, SH, BB, false, 8>(a, bx, n_boxes, d.bin_start, total_bins, work, d.sm_count, s) \
              : launch_batch<T, SH, BB, false, 16>(a, bx, n_boxes, d.bin_start, total_bins, work, d.sm_count, s)
    if (d.shape == 1) {
        if (d.bin == 4) { RSOL_BATCH(1, 4); }
        RSOL_BATCH(1, 8);
    }
    if (d.bin == 4) { RSOL_BATCH(2, 4); }
    RSOL_BATCH(2, 8);
#undef RSOL_BATCH
}

inline size_t batch_box_bytes(int precision)
{
    return precision == 32 ? sizeof(BatchBox<float>) : sizeof(BatchBox<double>);
}

template <typename T>
void fill_batch_box(void *dst, int nx, int ny, int nz, int nbx, int nby, int nbz, int64_t node_off,
                    uint32_t bin_base, double h, double adv, double qv, double c)
{
    BatchBox<T> b;
    b.nx = nx; b.ny = ny; b.nz = nz; b.nbx = nbx; b.nby = nby; b.nbz = nbz;
    b.node_off = node_off;
    b.bin_base = bin_base;
    b.k.h = T(h); b.k.adv = T(adv); b.k.qv = T(qv); b.k.c = T(c);
    *static_cast<BatchBox<T> *>(dst) = b;
}

} // namespace rsol
