// State moments (Sec. 2 packet totals per unit volume: n, N m c u,
// N gamma m c^2, N q c beta) deposited with W at the current positions, for a
// packet set in the order rsol_sort wrote: one CTA per sort bin sums its
// packets into a shared-memory tile (bin + 2-node halo) and adds the tile to
// the grid once.  Within a warp, runs of packets of equal stencil origin
// along the lanes are summed in registers by stencil-offset lanes before each
// shared-memory add, as in the binned push's deposit.  No field gather: the
// tile holds only the eight moments.  FP64 accumulates them in doubles.  FP32
// holds all eight as 32-bit fixed point with per-CTA scales from a bound on
// the bin's packets (largest weight, largest |u|^2; |beta| < 1 bounds the
// current), added with native integer atomics; the three momentum-density
// components, whose sums over isotropic packets cancel, also keep each
// addition's rounding remainder in three more planes.
#pragma once

#include <type_traits>

#include "push_binned.cuh"

namespace rsol {

template <typename T, int SHAPE, int B, int NW>
struct MomCfg {
    static constexpr int NP = SHAPE == 1 ? 2 : 3;
    static constexpr int NS = NP * NP * NP;
    static constexpr int TE = B + 4;
    // padded strides: FP32 puts the 27 stencil lanes of a TSC flush on 27
    // distinct banks; FP64 (8-byte elements) spreads rows and planes
    static constexpr bool F4 = sizeof(T) == 4;
    static constexpr int RS = F4 && TE == 12 ? 14 : (F4 && TE == 8 ? 11 : TE + 1);
    static constexpr int PS = F4 && TE == 12 ? 171 : (F4 && TE == 8 ? 89 : TE * RS + 1);
    static constexpr int TN = TE * PS;
    static constexpr int WS = NS == 27 ? 28 : NS;  // weight rows padded to 16-byte stores
    static constexpr int QO = 12;
    // FP32: eight 32-bit fixed-point planes plus the low parts of the momentum
    // density (planes 8..10); FP64: eight double planes
    static constexpr int NPL = sizeof(T) == 4 ? 11 : 8;
    static constexpr size_t tile_bytes = size_t(TN) * NPL * sizeof(T);
    static constexpr size_t stage_words = 32 * (WS + QO);
    // origin keys and local visiting order of the bin's first KEYCAP packets
    static constexpr int KEYCAP = sizeof(T) == 4 ? 8192 : 4096;
    static constexpr size_t stage_bytes = size_t(NW) * stage_words * sizeof(T);
    static constexpr size_t smem_bytes = tile_bytes + stage_bytes + 2 * size_t(KEYCAP) * sizeof(uint16_t);
};

// The eight state moments of one packet (weight w, momentum u).
template <typename T>
__device__ __forceinline__ void state_moments(const MomArgs<T> &a, T w, const T u[3], T Q[8])
{
    const T g = Math<T>::sqrt(T(1) + dot3(u, u));
    const T N = w * a.inv_vol;
    Q[0] = N;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        Q[1 + q] = N * a.mc * u[q];
    Q[4] = N * g * a.mc2;
    const T ig = Math<T>::div(T(1), g);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        Q[5 + q] = N * a.qc * (u[q] * ig);
}

template <typename T, int SHAPE, int B, int NW>
__global__ void __launch_bounds__(NW * 32) moments_binned_kernel(MomArgs<T> a, BinGeom g)
{
    using Cfg = MomCfg<T, SHAPE, B, NW>;
    constexpr int TE = Cfg::TE, RS = Cfg::RS, PS = Cfg::PS, TN = Cfg::TN;
    constexpr int NP = Cfg::NP, NS = Cfg::NS, WS = Cfg::WS, QO = Cfg::QO;
    extern __shared__ __align__(16) unsigned char smem[];
    T *sd = reinterpret_cast<T *>(smem);  // [q][slot]
    T *stage = reinterpret_cast<T *>(smem + Cfg::tile_bytes);
    uint16_t *s_key = reinterpret_cast<uint16_t *>(smem + Cfg::tile_bytes + Cfg::stage_bytes);
    uint16_t *s_perm = s_key + Cfg::KEYCAP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *sW = stage + warp * Cfg::stage_words;  // [32][WS]
    T *sQ = sW + 32 * WS;                     // [32][QO]
    // FP32: every moment in 32-bit fixed point with a per-CTA scale.  The
    // momentum density (q = 1..3), whose node sums cancel, keeps the rounding
    // remainder of each addition as well: plane 7 + q holds the remainders in
    // units of 2^-s_lo_bits of the main plane's unit.
    constexpr bool FX = std::is_same<T, float>::value;
    __shared__ float s_scale[8], s_iscale[8];
    __shared__ float s_lo, s_ilo;  // 2^s_lo_bits and its inverse

    const int bin = blockIdx.x;
    const int bx = bin % g.nbx, by = (bin / g.nbx) % g.nby, bz = bin / (g.nbx * g.nby);
    const uint32_t lo = g.bin_start[bin], hi = g.bin_start[bin + 1];
    if (lo >= hi)
        return;

    // the packet's own nodes in the global grid
    auto deposit_global = [&](int ix, int iy, int iz, const T wx[3], const T wy[3], const T wz[3],
                              int rx, int ry, int rz, const T Q[8]) {
        int kx[3], ky[3], kz[3];
        axis_nodes(ix, rx, a.nx, kx);
        axis_nodes(iy, ry, a.ny, ky);
        axis_nodes(iz, rz, a.nz, kz);
#pragma unroll
        for (int cz = 0; cz < NP; ++cz)
#pragma unroll
            for (int cy = 0; cy < NP; ++cy) {
                const T wyz = wy[cy] * wz[cz];
                const int64_t row = (int64_t(kz[cz]) * a.ny + ky[cy]) * a.nx;
#pragma unroll
                for (int cx = 0; cx < NP; ++cx)
                    red_node(a.grid + (row + kx[cx]) * 8, wx[cx] * wyz, Q);
            }
    };

    if (hi - lo <= sparse_bin_limit<B>()) {  // few packets: the tile would cost more than their atomics
        for (uint32_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
            const uint32_t c = a.cell[j];
            const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
            if (ix >= a.nx || iy >= a.ny || iz >= a.nz)
                continue;
            const T u[3] = {a.u0[j], a.u1[j], a.u2[j]};
            T Q[8], wx[3], wy[3], wz[3];
            state_moments(a, a.w[j], u, Q);
            const int rx = axis_weights<SHAPE>(a.off0[j], wx);
            const int ry = axis_weights<SHAPE>(a.off1[j], wy);
            const int rz = axis_weights<SHAPE>(a.off2[j], wz);
            deposit_global(ix, iy, iz, wx, wy, wz, rx, ry, rz, Q);
        }
        return;
    }
    const int ox = bx * B - 2, oy = by * B - 2, oz = bz * B - 2;
    for (int t = threadIdx.x; t < Cfg::NPL * TN; t += blockDim.x)
        sd[t] = T(0);
    __shared__ int s_desc, s_sorted, s_out;
    if (threadIdx.x == 0) {
        s_desc = 0;
        s_sorted = 0;
    }
    __syncthreads();

    // packets drifted since the last global sort break the origin order; once
    // more than one in 32 does, a counting sort by stencil origin (local to the
    // CTA, as in the binned push) gives the order the runs below are taken in
    const uint32_t n_bin = hi - lo;
    const bool keep = n_bin <= uint32_t(Cfg::KEYCAP);  // origin keys kept for a local sort
    if (FX || keep) {
        // origin histogram (packets per stencil origin), order breaks and, for
        // FP32, the largest weight and |u|^2 of the bin's packets
        int *hist = reinterpret_cast<int *>(sd);  // plane 0 of the zeroed tile
        int desc = 0;
        T wmax = T(0), u2max = T(0);
        for (uint32_t rb = 0; rb < n_bin; rb += blockDim.x) {  // warp-uniform trip count
            const uint32_t r = rb + threadIdx.x;
            int key = TN;  // out of the tile or off the grid: last
            if (r < n_bin) {
                const uint32_t j = lo + r;
                key = origin_slot<SHAPE, TE, RS, PS, TN>(a.cell[j], a.off0[j], a.off1[j], a.off2[j], ox,
                                                         oy, oz, a.nx, a.ny, a.nz);
                if (key < TN)
                    atomicAdd(&hist[key], 1);
                if (keep)
                    s_key[r] = uint16_t(key);
                if (FX) {
                    const T u[3] = {a.u0[j], a.u1[j], a.u2[j]};
                    wmax = fmax(wmax, fabs(a.w[j]));
                    u2max = fmax(u2max, dot3(u, u));
                }
            }
            const int prev = __shfl_up_sync(0xffffffffu, key, 1);
            desc += (lane > 0 && r < n_bin && key < prev) ? 1 : 0;
        }
        desc = __reduce_add_sync(0xffffffffu, desc);
        if (lane == 0 && desc)
            atomicAdd(&s_desc, desc);
        __syncthreads();
        if constexpr (FX) {
            // fixed-point scale 2^e per moment: (largest total weight of a node)
            // x (bound on one packet's moment) below 2^30; bounds per packet:
            // n: w/dx^3;  momentum: n m c |u|_max;  energy: n m c^2 gamma_max;
            // current: n |q| c
            float gmax = tile_weight_bound<SHAPE, TE, RS, PS, NW>(hist, reinterpret_cast<float *>(stage));
            __shared__ float s_red[3][NW];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
                wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
                u2max = fmax(u2max, __shfl_xor_sync(0xffffffffu, u2max, o));
            }
            if (lane == 0) {
                s_red[0][warp] = gmax;
                s_red[1][warp] = float(wmax);
                s_red[2][warp] = float(u2max);
            }
            __syncthreads();
            if (threadIdx.x < 8) {
                float gm = 0.f, wm = 0.f, um = 0.f;
                for (int w = 0; w < NW; ++w) {
                    gm = fmaxf(gm, s_red[0][w]);
                    wm = fmaxf(wm, s_red[1][w]);
                    um = fmaxf(um, s_red[2][w]);
                }
                const int q = threadIdx.x;
                const float n1 = wm * fabsf(float(a.inv_vol));
                float bound = q == 0 ? n1
                            : q < 4  ? n1 * fabsf(float(a.mc)) * sqrtf(um)
                            : q == 4 ? n1 * fabsf(float(a.mc2)) * sqrtf(1.f + um)
                                     : n1 * fabsf(float(a.qc));
                bound *= gm > 1.f ? gm : 1.f;
                int e = 30;
                if (bound > 0.f && isfinite(bound))
                    e = 30 - int(ceilf(log2f(bound)));
                e = e > 60 ? 60 : (e < -60 ? -60 : e);
                s_scale[q] = ldexpf(1.0f, e);
                s_iscale[q] = ldexpf(1.0f, -e);
                if (q == 0) {
                    // a remainder is at most 2^(k-1) units; a node receives at most
                    // one per run, i.e. at most n_bin: n_bin 2^(k-1) < 2^30
                    int k = 31 - int(ceilf(log2f(float(n_bin) + 1.f)));
                    k = k > 16 ? 16 : (k < 0 ? 0 : k);
                    s_lo = ldexpf(1.0f, k);
                    s_ilo = ldexpf(1.0f, -k);
                }
            }
            __syncthreads();
        }
        if (keep && s_desc * 32 > int(n_bin)) {
            int *cursor = reinterpret_cast<int *>(stage);  // free until the batches
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

    // phase-2 lane role: stencil offset and quantity range [q0, q0 + 2 or 8)
    const int off_id = SHAPE == 1 ? (lane & 7) : (lane < 27 ? lane : 0);
    const bool p2_active = SHAPE == 1 ? true : lane < 27;
    const int pax = off_id % NP, pay = (off_id / NP) % NP, paz = off_id / (NP * NP);
    const int q0 = SHAPE == 1 ? 2 * (lane >> 3) : 0;
    const int lane_off = paz * PS + pay * RS + pax;
    constexpr int NQ_ = SHAPE == 1 ? 2 : 8;
    T acc[NQ_];
#pragma unroll
    for (int q = 0; q < NQ_; ++q)
        acc[q] = T(0);
    f32x2 acc2[NQ_ / 2];  // FP32: the moments in pairs (f32x2 arithmetic)
#pragma unroll
    for (int q = 0; q < NQ_ / 2; ++q)
        acc2[q] = 0;
    int carry_origin = -1;
    auto flush_acc = [&](int origin) {
        if (p2_active && origin >= 0) {
            if constexpr (FX) {
#pragma unroll
                for (int q = 0; q < NQ_ / 2; ++q)
                    f2_unpack(acc2[q], acc[2 * q], acc[2 * q + 1]);
            }
#pragma unroll
            for (int q = 0; q < NQ_; ++q) {
                const int qq = q0 + q;
                T *dst = &sd[qq * TN + origin + lane_off];
                if constexpr (FX) {  // pre-scaled to the tile's fixed point
                    const float x = float(acc[q]);
                    const int hi = __float2int_rn(x);
                    atomicAdd(reinterpret_cast<int *>(dst), hi);
                    if (qq >= 1 && qq <= 3) {
                        // x - hi is exact (hi is x rounded to an integer), |x - hi| <= 1/2
                        const int rem = __float2int_rn((x - float(hi)) * s_lo);
                        if (rem != 0)
                            atomicAdd(reinterpret_cast<int *>(&sd[(7 + qq) * TN + origin + lane_off]), rem);
                    }
                } else {
                    atomicAdd(dst, acc[q]);
                }
            }
        }
    };

    // each warp walks a contiguous slice of the bin (runs carry across batches)
    const uint32_t per_warp = ((n_bin + NW - 1) / NW + 31) & ~31u;
    const uint32_t w_lo = lo + per_warp * uint32_t(warp);
    const uint32_t w_hi = w_lo + per_warp < hi ? w_lo + per_warp : hi;
    // software pipeline: the packet of visiting position pos (base + lane) of
    // the next batch is loaded into registers while this batch is deposited
    uint32_t n_c = 0xFFFFFFFFu;
    T n_o[3] = {T(0), T(0), T(0)}, n_u[3] = {T(0), T(0), T(0)}, n_w = T(0);
    auto prefetch = [&](uint32_t pos) {
        n_c = 0xFFFFFFFFu;  // off the grid: nothing to deposit
        if (pos < w_hi) {
            const uint32_t j = use_perm ? lo + s_perm[pos - lo] : pos;
            n_c = a.cell[j];
            n_o[0] = a.off0[j];
            n_o[1] = a.off1[j];
            n_o[2] = a.off2[j];
            n_u[0] = a.u0[j];
            n_u[1] = a.u1[j];
            n_u[2] = a.u2[j];
            n_w = a.w[j];
        }
    };
    prefetch(w_lo + uint32_t(lane));
    for (uint32_t base = w_lo; base < w_hi; base += 32) {
        const uint32_t c = n_c;
        const T f[3] = {n_o[0], n_o[1], n_o[2]};
        const T u[3] = {n_u[0], n_u[1], n_u[2]};
        const T wj = n_w;
        prefetch(base + 32 + uint32_t(lane));
        int staged = -1;
        {
            const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
            if (ix < a.nx && iy < a.ny && iz < a.nz) {
                T Q[8], wx[3], wy[3], wz[3];
                state_moments(a, wj, u, Q);
                int rx, ry, rz;
                const int jx = anchor_axis<SHAPE>(ix, f[0], a.nx, wx, rx);
                const int jy = anchor_axis<SHAPE>(iy, f[1], a.ny, wy, ry);
                const int jz = anchor_axis<SHAPE>(iz, f[2], a.nz, wz, rz);
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
                    store_wrow<WS>(sW + lane * WS, Wk);
                    if constexpr (FX) {  // the tile's fixed-point scales (powers of two: exact)
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            Q[q] *= T(s_scale[q]);
                    }
                    store_q8(sQ + lane * QO, Q);
                    staged = lz * PS + ly * RS + lx;
                } else {
                    deposit_global(jx, jy, jz, wx, wy, wz, rx, ry, rz, Q);
                }
            }
        }
        // runs of equal stencil origin along the lanes; a lane with no staged
        // packet (-1) starts a run that is skipped
        const int left = __shfl_up_sync(0xffffffffu, staged, 1);
        uint32_t st = __ballot_sync(0xffffffffu, lane == 0 || staged != left);
        __syncwarp();
        while (st) {  // warp-uniform: one run per pass, summed in registers
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
            if constexpr (FX) {
                // moments in pairs: a packet is one weight load, two (TSC) or one
                // (CIC) 16/8-byte moment loads and NQ/2 paired multiply-adds
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
                continue;
            }
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
        __syncwarp();
    }
    flush_acc(carry_origin);
    __syncthreads();

    // add the tile to the global grid (untouched nodes skipped)
    for (int t = threadIdx.x; t < TE * TE * TE; t += blockDim.x) {
        const int lx = t % TE, ly = (t / TE) % TE, lz = t / (TE * TE);
        const int slot = lz * PS + ly * RS + lx;
        const int64_t node =
            (int64_t(wrap_mod(oz + lz, a.nz)) * a.ny + wrap_mod(oy + ly, a.ny)) * a.nx +
            wrap_mod(ox + lx, a.nx);
        T v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if constexpr (FX) {
                const int *si = reinterpret_cast<const int *>(sd);
                float x = float(si[q * TN + slot]);
                if (q >= 1 && q <= 3)
                    x += float(si[(7 + q) * TN + slot]) * s_ilo;
                v[q] = T(x * s_iscale[q]);
            } else {
                v[q] = sd[q * TN + slot];
            }
        }
        if (sizeof(T) == 4) {
            float *p = reinterpret_cast<float *>(a.grid) + node * 8;
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
                    atomicAdd(reinterpret_cast<double *>(a.grid) + node * 8 + q, double(v[q]));
        }
    }
}

template <typename T, int SHAPE, int B>
cudaError_t launch_moments_binned(const MomArgs<T> &a, const BinGeom &g, int64_t nbins, cudaStream_t s)
{
    constexpr int NW = (sizeof(T) == 8 && B == 8) ? 8 : 16;  // FP64 8^3 tiles: fewer warps fit
    using Cfg = MomCfg<T, SHAPE, B, NW>;
    static_assert(Cfg::smem_bytes <= 232448 - 1024, "moments tiles exceed shared memory");
    auto kern = moments_binned_kernel<T, SHAPE, B, NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem_bytes));
    if (e != cudaSuccess)
        return e;
    kern<<<unsigned(nbins), NW * 32, Cfg::smem_bytes, s>>>(a, g);
    return cudaGetLastError();
}

} // namespace rsol

namespace rsol {

template <typename T>
cudaError_t moments_binned_dispatch(const MomentsDesc &d, cudaStream_t s)
{
    MomArgs<T> a;
    a.n = d.n;
    a.cell = d.cell;
    a.off0 = static_cast<const T *>(d.off[0]);
    a.off1 = static_cast<const T *>(d.off[1]);
    a.off2 = static_cast<const T *>(d.off[2]);
    a.u0 = static_cast<const T *>(d.u[0]);
    a.u1 = static_cast<const T *>(d.u[1]);
    a.u2 = static_cast<const T *>(d.u[2]);
    a.w = static_cast<const T *>(d.w);
    a.grid = static_cast<T *>(d.grid);
    a.fx = nullptr;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.inv_vol = T(d.inv_vol);
    a.mc = T(d.mc);
    a.mc2 = T(d.mc2);
    a.qc = T(d.qc);
    a.fx_scale = T(0);
    BinGeom g;
    g.bin_start = d.bin_start;
    g.nbx = d.nbx;
    g.nby = d.nby;
    g.nbz = d.nbz;
    const int64_t nbins = int64_t(d.nbx) * d.nby * d.nbz;
    if (d.shape == 1)
        return d.bin == 4 ? launch_moments_binned<T, 1, 4>(a, g, nbins, s)
                          : launch_moments_binned<T, 1, 8>(a, g, nbins, s);
    return d.bin == 4 ? launch_moments_binned<T, 2, 4>(a, g, nbins, s)
                      : launch_moments_binned<T, 2, 8>(a, g, nbins, s);
}

} // namespace rsol

namespace rsol {

template <typename T>
struct LossBinArgs {
    int64_t n;
    const uint32_t *cell;
    const T *o0, *o1, *o2, *u0, *u1, *u2;
    T *w;
    const T *nn;
    T coef;
    int nx, ny, nz;
    int *status;
    BinGeom g;
};

// Catastrophic losses (Sec. 2) for the last sort's output with a gathered
// n_n: one CTA per bin stages the bin's n_n tile (bin + 2-node halo) in shared
// memory and gathers each packet's n_n from it; packets whose stencil left the
// tile read the grid.  Same arithmetic as losses_kernel.
template <typename T, int SHAPE, int B>
__global__ void __launch_bounds__(256) losses_binned_kernel(LossBinArgs<T> a)
{
    constexpr int NP = SHAPE == 1 ? 2 : 3;
    constexpr int TE = B + 4;
    __shared__ T tile[TE * TE * TE];
    const int bin = blockIdx.x;
    const int bx = bin % a.g.nbx, by = (bin / a.g.nbx) % a.g.nby, bz = bin / (a.g.nbx * a.g.nby);
    const uint32_t lo = a.g.bin_start[bin], hi = a.g.bin_start[bin + 1];
    if (lo >= hi)
        return;
    const int ox = bx * B - 2, oy = by * B - 2, oz = bz * B - 2;
    // grid offsets of the tile's rows along each axis (periodic)
    __shared__ int s_axis[3 * TE];
    if (threadIdx.x < 3 * TE) {
        const int ax = threadIdx.x / TE, l = threadIdx.x % TE;
        const int o = ax == 0 ? ox : (ax == 1 ? oy : oz);
        const int n = ax == 0 ? a.nx : (ax == 1 ? a.ny : a.nz);
        const int stride = ax == 0 ? 1 : (ax == 1 ? a.nx : a.nx * a.ny);
        s_axis[threadIdx.x] = wrap_mod(o + l, n) * stride;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < TE * TE * TE; t += blockDim.x) {
        const int lx = t % TE, ly = (t / TE) % TE, lz = t / (TE * TE);
        tile[t] = a.nn[s_axis[lx] + s_axis[TE + ly] + s_axis[2 * TE + lz]];
    }
    __syncthreads();
    int flag = 0;
    constexpr int U = 4;  // packets per thread per pass: their loads are issued first
    for (uint32_t jb = lo + threadIdx.x; jb < hi; jb += U * blockDim.x) {
        uint32_t cc[U];
        T f0[U], f1[U], f2[U], v0[U], v1[U], v2[U], ww[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t j = jb + uint32_t(k) * blockDim.x;
            const bool ok = j < hi;
            cc[k] = ok ? a.cell[j] : 0xFFFFFFFFu;
            f0[k] = ok ? a.o0[j] : T(0);
            f1[k] = ok ? a.o1[j] : T(0);
            f2[k] = ok ? a.o2[j] : T(0);
            v0[k] = ok ? a.u0[j] : T(0);
            v1[k] = ok ? a.u1[j] : T(0);
            v2[k] = ok ? a.u2[j] : T(0);
            ww[k] = ok ? a.w[j] : T(0);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t j = jb + uint32_t(k) * blockDim.x;
            if (j >= hi)
                continue;
            const T u[3] = {v0[k], v1[k], v2[k]};
            const T uu = dot3(u, u);
            const T beta = Math<T>::sqrt(uu) * Math<T>::rsqrt(T(1) + uu);
            const uint32_t c = cc[k];
            const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
            if (ix >= a.nx || iy >= a.ny || iz >= a.nz) {
                flag |= ST_BADCELL;
                continue;
            }
            T wx[3], wy[3], wz[3];
            const int rx = axis_weights<SHAPE>(f0[k], wx);
            const int ry = axis_weights<SHAPE>(f1[k], wy);
            const int rz = axis_weights<SHAPE>(f2[k], wz);
            // first stencil node, tile-local (periodic)
            int lx = ix + rx - ox, ly = iy + ry - oy, lz = iz + rz - oz;
            lx += lx < 0 ? a.nx : 0;
            ly += ly < 0 ? a.ny : 0;
            lz += lz < 0 ? a.nz : 0;
            lx -= lx >= a.nx ? a.nx : 0;
            ly -= ly >= a.ny ? a.ny : 0;
            lz -= lz >= a.nz ? a.nz : 0;
            const bool in_tile = lx >= 0 && ly >= 0 && lz >= 0 && lx + NP <= TE && ly + NP <= TE &&
                                 lz + NP <= TE;
            T dens = T(0);
            if (in_tile) {  // separable: rows along x, then y, then z
                const T *t0 = tile + (lz * TE + ly) * TE + lx;
#pragma unroll
                for (int cz = 0; cz < NP; ++cz) {
                    T dz = T(0);
#pragma unroll
                    for (int cy = 0; cy < NP; ++cy) {
                        const T *row = t0 + (cz * TE + cy) * TE;
                        T dy = wx[0] * row[0];
#pragma unroll
                        for (int cx = 1; cx < NP; ++cx)
                            dy += wx[cx] * row[cx];
                        dz += wy[cy] * dy;
                    }
                    dens += wz[cz] * dz;
                }
            } else {
                int kx[3], ky[3], kz[3];
                axis_nodes(ix, rx, a.nx, kx);
                axis_nodes(iy, ry, a.ny, ky);
                axis_nodes(iz, rz, a.nz, kz);
#pragma unroll
                for (int cz = 0; cz < NP; ++cz)
#pragma unroll
                    for (int cy = 0; cy < NP; ++cy) {
                        const T wyz = wy[cy] * wz[cz];
                        const int64_t row = (int64_t(kz[cz]) * a.ny + ky[cy]) * a.nx;
#pragma unroll
                        for (int cx = 0; cx < NP; ++cx)
                            dens += wx[cx] * wyz * a.nn[row + kx[cx]];
                    }
            }
            a.w[j] = ww[k] * exp(-a.coef * beta * dens);
        }
    }
    if (flag)
        atomicOr(a.status, flag);
}

template <typename T>
cudaError_t losses_binned_dispatch(const LossDesc &d, cudaStream_t s)
{
    LossBinArgs<T> a;
    a.n = d.n;
    a.cell = d.cell;
    a.o0 = static_cast<const T *>(d.off[0]);
    a.o1 = static_cast<const T *>(d.off[1]);
    a.o2 = static_cast<const T *>(d.off[2]);
    a.u0 = static_cast<const T *>(d.u[0]);
    a.u1 = static_cast<const T *>(d.u[1]);
    a.u2 = static_cast<const T *>(d.u[2]);
    a.w = static_cast<T *>(d.w);
    a.nn = static_cast<const T *>(d.nn);
    a.coef = T(d.coef);
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.status = d.status;
    a.g.bin_start = d.bin_start;
    a.g.nbx = d.nbx;
    a.g.nby = d.nby;
    a.g.nbz = d.nbz;
    const unsigned nbins = unsigned(int64_t(d.nbx) * d.nby * d.nbz);
    if (d.shape == 1) {
        if (d.bin == 4) losses_binned_kernel<T, 1, 4><<<nbins, 256, 0, s>>>(a);
        else losses_binned_kernel<T, 1, 8><<<nbins, 256, 0, s>>>(a);
    } else {
        if (d.bin == 4) losses_binned_kernel<T, 2, 4><<<nbins, 256, 0, s>>>(a);
        else losses_binned_kernel<T, 2, 8><<<nbins, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

} // namespace rsol
