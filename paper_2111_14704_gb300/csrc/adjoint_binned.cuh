// Tiled reverse step: the adjoint of one push step for a packet set in the
// order of the last sort, one CTA per sort bin.  The bin's field tile and
// accumulated momentum-source tile (bin + 2-node halo) are staged in shared
// memory; each packet's gathers read the tiles and its share of dL/dF goes
// to a shared-memory tile of six components, summed within a warp per run of
// equal stencil origin along the lanes (stencil-offset lanes; the CTA sorts its
// bin by origin first once drift has broken the order) before each shared add,
// and added to the global field adjoint once per CTA.  The arithmetic
// per packet is adjoint_packet, as in the order-free kernel; packets whose
// stencil left the tile, and bins with few packets, take the order-free path.
#pragma once

#include "adjoint.cuh"
#include "push_binned.cuh"

namespace rsol {

template <typename T, int SHAPE, int B, int NW>
struct AdjTileCfg {
    static constexpr int NP = SHAPE == 1 ? 2 : 3;
    static constexpr int NS = NP * NP * NP;
    static constexpr int TE = B + 4;
    static constexpr int RS = TE + 1;
    static constexpr int PS = TE * RS + 1;
    static constexpr int TN = TE * PS;
    // the adjoint tile has its own strides: FP32 puts the 27 stencil lanes of a
    // TSC flush on 27 distinct banks (the field and source tiles keep TN)
    static constexpr bool F4 = sizeof(T) == 4;
    static constexpr int DRS = F4 && TE == 12 ? 14 : (F4 && TE == 8 ? 11 : RS);
    static constexpr int DPS = F4 && TE == 12 ? 171 : (F4 && TE == 8 ? 89 : PS);
    static constexpr int DTN = TE * DPS;
    static constexpr int QO = 8;  // staged Ebar, Bbar (6 used; 16-byte rows)
    static constexpr size_t fields_bytes = size_t(TN) * 8 * sizeof(T);  // [slot][8]: E, B, 2 unused
    static constexpr size_t src_bytes = size_t(TN) * 4 * sizeof(T);     // [slot][4]: S, 1 unused
    static constexpr size_t bar_bytes = size_t(DTN) * 6 * sizeof(T);    // [q][slot]
    static constexpr size_t stage_words = 32 * (NS + QO);
    static constexpr size_t stage_bytes = size_t(NW) * stage_words * sizeof(T);
    // local visiting order of the bin's first KEYCAP packets (the origin keys and
    // the per-origin cursors of the local sort live in the stage area meanwhile)
    static constexpr int KEYCAP = 8192;
    static constexpr size_t perm_bytes = size_t(KEYCAP) * sizeof(uint16_t);
    static_assert(stage_bytes >= perm_bytes + size_t(TN) * sizeof(int),
                  "the stage area holds the keys and cursors of the local sort");
    static constexpr size_t smem_bytes = fields_bytes + src_bytes + bar_bytes + stage_bytes + perm_bytes;
};

template <typename T, int SHAPE, int B, int NW>
__global__ void __launch_bounds__(NW * 32) adjoint_binned_kernel(AdjArgs<T> a, BinGeom g)
{
    using Cfg = AdjTileCfg<T, SHAPE, B, NW>;
    constexpr int TE = Cfg::TE, RS = Cfg::RS, PS = Cfg::PS, TN = Cfg::TN;
    constexpr int NP = Cfg::NP, NS = Cfg::NS, QO = Cfg::QO;
    extern __shared__ __align__(16) unsigned char smem[];
    T *sf = reinterpret_cast<T *>(smem);
    T *ssrc = reinterpret_cast<T *>(smem + Cfg::fields_bytes);
    T *sbar = reinterpret_cast<T *>(smem + Cfg::fields_bytes + Cfg::src_bytes);
    T *stage = reinterpret_cast<T *>(smem + Cfg::fields_bytes + Cfg::src_bytes + Cfg::bar_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *sW = stage + warp * Cfg::stage_words;  // [32][NS]
    T *sQ = sW + 32 * NS;                     // [32][QO]
    uint16_t *s_perm = reinterpret_cast<uint16_t *>(smem + Cfg::fields_bytes + Cfg::src_bytes +
                                                    Cfg::bar_bytes + Cfg::stage_bytes);

    const int bin = blockIdx.x;
    const int bx = bin % g.nbx, by = (bin / g.nbx) % g.nby, bz = bin / (g.nbx * g.nby);
    const uint32_t lo = g.bin_start[bin], hi = g.bin_start[bin + 1];
    if (lo >= hi)
        return;
    const T inv_L = T(a.loss[1]);
    int flag = 0;
    if (hi - lo <= sparse_bin_limit<B>()) {
        for (uint32_t j = lo + threadIdx.x; j < hi; j += blockDim.x)
            adjoint_one<T, SHAPE>(a, int64_t(j), inv_L, &flag);
        if (flag)
            atomicOr(a.status, flag);
        return;
    }
    const int ox = bx * B - 2, oy = by * B - 2, oz = bz * B - 2;

    // stage the field and source tiles (periodic); clear the adjoint tile
    constexpr int TT = TE * TE * TE;
    for (int t = threadIdx.x; t < TT; t += blockDim.x) {
        const int lx = t % TE, ly = (t / TE) % TE, lz = t / (TE * TE);
        const int64_t node = (int64_t(wrap_mod(oz + lz, a.nz)) * a.ny + wrap_mod(oy + ly, a.ny)) * a.nx +
                             wrap_mod(ox + lx, a.nx);
        const int slot = lz * PS + ly * RS + lx;
        T F[6], S[3];
        load_node(a.fields + node * 8, F);
        load_s(a.fb + node * 8, S);
        sts_node(sf + slot * 8, F);
        ssrc[slot * 4] = S[0];
        ssrc[slot * 4 + 1] = S[1];
        ssrc[slot * 4 + 2] = S[2];
    }
    for (int t = threadIdx.x; t < 6 * Cfg::DTN; t += blockDim.x)
        sbar[t] = T(0);
    __shared__ int s_desc, s_sorted, s_out;
    if (threadIdx.x == 0) {
        s_desc = 0;
        s_sorted = 0;
    }
    __syncthreads();

    // The reverse sweep meets packets up to a checkpoint segment past their sort,
    // so their stencil origins are no longer in order.  Once more than one packet
    // in 32 breaks the order, a counting sort by origin local to the CTA (as in
    // the push) gives the order the batches visit, so the runs below span whole
    // origins.  Bins of more than KEYCAP packets keep the sort's order.
    const uint32_t n_bin = hi - lo;
    if (n_bin <= uint32_t(Cfg::KEYCAP)) {
        int *hist = reinterpret_cast<int *>(sbar);  // the cleared adjoint tile
        uint16_t *s_key = reinterpret_cast<uint16_t *>(stage);
        int *cursor = reinterpret_cast<int *>(stage) + Cfg::KEYCAP / 2;
        int desc = 0;
        for (uint32_t rb = 0; rb < n_bin; rb += blockDim.x) {  // warp-uniform trip count
            const uint32_t r = rb + threadIdx.x;
            int key = TN;
            if (r < n_bin) {
                const uint32_t j = lo + r;
                key = origin_slot<SHAPE, TE, RS, PS, TN>(a.cell[j], a.off0[j], a.off1[j], a.off2[j], ox,
                                                         oy, oz, a.nx, a.ny, a.nz);
                if (key < TN)
                    atomicAdd(&hist[key], 1);
                s_key[r] = uint16_t(key);
            }
            const int prev = __shfl_up_sync(0xffffffffu, key, 1);
            desc += (lane > 0 && r < n_bin && key < prev) ? 1 : 0;
        }
        desc = __reduce_add_sync(0xffffffffu, desc);
        if (lane == 0 && desc)
            atomicAdd(&s_desc, desc);
        __syncthreads();
        if (s_desc * 32 > int(n_bin)) {
            origin_cursors<NW, TN>(hist, cursor, &s_out);
            for (uint32_t r = threadIdx.x; r < n_bin; r += blockDim.x) {
                const int key = s_key[r];
                const int pos = key < TN ? atomicAdd(&cursor[key], 1) : atomicAdd(&s_out, 1);
                s_perm[pos] = uint16_t(r);
            }
            if (threadIdx.x == 0)
                s_sorted = 1;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < TN; t += blockDim.x)
            hist[t] = 0;
        __syncthreads();
    }
    const bool use_perm = s_sorted != 0;

    // phase-2 lane role: stencil offset and component range [q0, q0 + NQ_)
    constexpr int NQ_ = SHAPE == 1 ? 2 : 6;
    const int off_id = SHAPE == 1 ? (lane & 7) : (lane < 27 ? lane : 0);
    const bool p2_active = SHAPE == 1 ? lane < 24 : lane < 27;
    const int q0 = SHAPE == 1 ? 2 * (lane >> 3) : 0;
    const int pax = off_id % NP, pay = (off_id / NP) % NP, paz = off_id / (NP * NP);
    const int lane_off = paz * Cfg::DPS + pay * Cfg::DRS + pax;
    T acc[NQ_];
#pragma unroll
    for (int q = 0; q < NQ_; ++q)
        acc[q] = T(0);
    int carry_origin = -1;
    auto flush_acc = [&](int origin) {
        if (p2_active && origin >= 0) {
#pragma unroll
            for (int q = 0; q < NQ_; ++q)
                atomicAdd(&sbar[(q0 + q) * Cfg::DTN + origin + lane_off], acc[q]);
        }
    };

    const uint32_t per_warp = ((n_bin + NW - 1) / NW + 31) & ~31u;
    const uint32_t w_lo = lo + per_warp * uint32_t(warp);
    const uint32_t w_hi = w_lo + per_warp < hi ? w_lo + per_warp : hi;
    for (uint32_t base = w_lo; base < w_hi; base += 32) {
        int staged = -1;
        if (base + uint32_t(lane) < w_hi) {
            // the packet at visiting position base + lane
            const uint32_t j = use_perm ? lo + s_perm[base + uint32_t(lane) - lo] : base + uint32_t(lane);
            const uint32_t c = a.cell[j];
            const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
            if (ix >= a.nx || iy >= a.ny || iz >= a.nz) {
                flag |= ST_BADCELL;
            } else {
                const T fx = a.off0[j], fy = a.off1[j], fz = a.off2[j];
                T w3[3];
                int rx, ry, rz;
                const int jx = anchor_axis<SHAPE>(ix, fx, a.nx, w3, rx);
                const int jy = anchor_axis<SHAPE>(iy, fy, a.ny, w3, ry);
                const int jz = anchor_axis<SHAPE>(iz, fz, a.nz, w3, rz);
                int lx = jx + rx - ox, ly = jy + ry - oy, lz = jz + rz - oz;
                lx += lx < 0 ? a.nx : 0;
                ly += ly < 0 ? a.ny : 0;
                lz += lz < 0 ? a.nz : 0;
                lx -= lx >= a.nx ? a.nx : 0;
                ly -= ly >= a.ny ? a.ny : 0;
                lz -= lz >= a.nz ? a.nz : 0;
                const bool in_tile = lx >= 0 && ly >= 0 && lz >= 0 && lx + NP <= TE &&
                                     ly + NP <= TE && lz + NP <= TE;
                if (in_tile) {
                    const int s0 = lz * PS + ly * RS + lx;
                    const T u0[3] = {a.u0[j], a.u1[j], a.u2[j]};
                    T xb[3] = {a.xb0[j], a.xb1[j], a.xb2[j]};
                    T ub[3] = {a.ub0[j], a.ub1[j], a.ub2[j]};
                    auto load = [&](int cz, int cy, int cx, T F[6], T S[3]) {
                        const int sl = s0 + cz * PS + cy * RS + cx;
                        lds_node(sf + sl * 8, F);
                        S[0] = ssrc[sl * 4];
                        S[1] = ssrc[sl * 4 + 1];
                        S[2] = ssrc[sl * 4 + 2];
                    };
                    auto scatter = [&](int cz, int cy, int cx, T W, const T Eb[3], const T Bb[3]) {
                        sW[lane * NS + (cz * NP + cy) * NP + cx] = W;
                        if (cz == 0 && cy == 0 && cx == 0) {
                            T *q = sQ + lane * QO;
                            q[0] = Eb[0];
                            q[1] = Eb[1];
                            q[2] = Eb[2];
                            q[3] = Bb[0];
                            q[4] = Bb[1];
                            q[5] = Bb[2];
                        }
                    };
                    adjoint_packet<T, SHAPE>(a.k, a.w[j], inv_L, fx, fy, fz, u0, xb, ub, load, scatter,
                                             &flag);
                    a.xb0[j] = xb[0];
                    a.xb1[j] = xb[1];
                    a.xb2[j] = xb[2];
                    a.ub0[j] = ub[0];
                    a.ub1[j] = ub[1];
                    a.ub2[j] = ub[2];
                    staged = lz * Cfg::DPS + ly * Cfg::DRS + lx;  // the adjoint tile's slot
                } else {
                    adjoint_one<T, SHAPE>(a, int64_t(j), inv_L, &flag);
                }
            }
        }
        // runs of equal stencil origin along the lanes (a lane with no staged
        // packet starts a run that is skipped); stencil-offset lanes sum each
        // run in registers, two packets per pass, and add the sum to the adjoint
        // tile when the origin changes
        const int left = __shfl_up_sync(0xffffffffu, staged, 1);
        uint32_t st = __ballot_sync(0xffffffffu, lane == 0 || staged != left);
        __syncwarp();
        while (st) {  // warp-uniform
            const int L = __ffs(st) - 1;
            st &= st - 1;
            const int R = st ? __ffs(st) - 1 : 32;
            const int origin = __shfl_sync(0xffffffffu, staged, L);
            if (origin < 0) {
                flush_acc(carry_origin);
                carry_origin = origin;
                continue;
            }
            int p = L;
            if (origin != carry_origin) {  // a new run: its first packet starts the sums
                flush_acc(carry_origin);
                carry_origin = origin;
                const T W = sW[p * NS + off_id];
                const T *q = sQ + p * QO + q0;
#pragma unroll
                for (int k = 0; k < NQ_; ++k)
                    acc[k] = W * q[k];
                ++p;
            }
            for (; p + 1 < R; p += 2) {
                const T W = sW[p * NS + off_id], W2 = sW[(p + 1) * NS + off_id];
                const T *q = sQ + p * QO + q0;
#pragma unroll
                for (int k = 0; k < NQ_; ++k) {
                    acc[k] += W * q[k];
                    acc[k] += W2 * q[QO + k];
                }
            }
            if (p < R) {
                const T W = sW[p * NS + off_id];
                const T *q = sQ + p * QO + q0;
#pragma unroll
                for (int k = 0; k < NQ_; ++k)
                    acc[k] += W * q[k];
            }
        }
        __syncwarp();
    }
    flush_acc(carry_origin);
    __syncthreads();

    // add the adjoint tile to the global grid (untouched nodes skipped)
    for (int t = threadIdx.x; t < TT; t += blockDim.x) {
        const int lx = t % TE, ly = (t / TE) % TE, lz = t / (TE * TE);
        const int slot = lz * Cfg::DPS + ly * Cfg::DRS + lx;
        T v[6];
        bool any = false;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            v[q] = sbar[q * Cfg::DTN + slot];
            any = any || v[q] != T(0);
        }
        if (!any)
            continue;
        const int64_t node = (int64_t(wrap_mod(oz + lz, a.nz)) * a.ny + wrap_mod(oy + ly, a.ny)) * a.nx +
                             wrap_mod(ox + lx, a.nx);
        red_field_bar(a.fbar + node * 8, T(1), v, v + 3);
    }
    if (flag)
        atomicOr(a.status, flag);
}

template <typename T, int SHAPE, int B>
cudaError_t launch_adjoint_binned(const AdjArgs<T> &a, const BinGeom &g, int64_t nbins, cudaStream_t s)
{
    // FP32: 16 warps at 128 registers fill the register file; FP64 needs 8
    constexpr int NW = sizeof(T) == 4 ? 16 : 8;
    using Cfg = AdjTileCfg<T, SHAPE, B, NW>;
    static_assert(Cfg::smem_bytes <= 232448 - 1024, "adjoint tiles exceed shared memory");
    auto kern = adjoint_binned_kernel<T, SHAPE, B, NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem_bytes));
    if (e != cudaSuccess)
        return e;
    kern<<<unsigned(nbins), NW * 32, Cfg::smem_bytes, s>>>(a, g);
    return cudaGetLastError();
}

} // namespace rsol

namespace rsol {

// The tiled kernel for a set in the order of the last sort (bin_start given),
// else the order-free one.
template <typename T>
cudaError_t adjoint_dispatch(const AdjDesc &d, cudaStream_t s)
{
    const bool tiled = d.bin_start != nullptr && (d.bin == 4 || (d.bin == 8 && sizeof(T) == 4));
    if (!tiled)
        return launch_adjoint<T>(d, s);
    AdjArgs<T> a = make_adj_args<T>(d);
    BinGeom g;
    g.bin_start = d.bin_start;
    g.nbx = d.nbx;
    g.nby = d.nby;
    g.nbz = d.nbz;
    const int64_t nbins = int64_t(d.nbx) * d.nby * d.nbz;
    if (d.shape == 1)
        return d.bin == 4 ? launch_adjoint_binned<T, 1, 4>(a, g, nbins, s)
                          : launch_adjoint_binned<T, 1, (sizeof(T) == 4 ? 8 : 4)>(a, g, nbins, s);
    return d.bin == 4 ? launch_adjoint_binned<T, 2, 4>(a, g, nbins, s)
                      : launch_adjoint_binned<T, 2, (sizeof(T) == 4 ? 8 : 4)>(a, g, nbins, s);
}

} // namespace rsol
