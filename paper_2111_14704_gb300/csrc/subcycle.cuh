// Per-packet adaptive timestep with sub-cycling (Sec. 3, timestep
// constraints).  Every CR time derivative carries c~/c, so every CR timestep
// constraint is c/c~ times its usual value:
//   gyration     dt_j < C / Omega~_j,  Omega~_j = (c~/c) |q/m| |B(x_j)| / (gamma_j c)
//   CR Courant   dt_j < C dx / |v_eff|, |v_eff| = c~ beta_j
//   losses       dt_j < C N_j / |dN_j/dt| = C / ((c~/c) sigma n_n c beta_j)
// A packet takes 2^k sub-steps of dt / 2^k (k the smallest level that meets
// its limit, at most max_level) in the fields of the global step, each a full
// packet step whose deposit carries the factor 2^-k, so the feedback grid
// receives the time average over the global step.
//
// Three kernels: levels (and per-level counts), a bucket scan, and the
// sub-cycled push over the packets in level-major order (high levels first),
// so that a warp's lanes run the same number of sub-steps.
#pragma once

#include "push.cuh"
#include "rsol_device.cuh"
#include "rsol_internal.h"

namespace rsol {

constexpr int kMaxLevel = 16;

template <typename T>
struct SubArgs {
    T courant;      // C
    T k_gyro;       // (c~/c) |q/m| / c:  Omega~ = k_gyro |B| / gamma
    T k_cross;      // dx / c~:           crossing-time limit = k_cross / beta
    T k_loss;       // 1 / ((c~/c) sigma n_n c), or 0 for no loss limit
    T dt;
    int max_level;
    uint8_t *level;     // [n] level of each packet
    uint32_t *counts;   // [kMaxLevel + 1] packets per level, then cursors
    uint32_t *order;    // [n] packet indices, level-major
};

// Sub-cycling level of packet j: B gathered with W at x_j (the order of the
// push's gather), the limit formed in the packet's precision with IEEE
// square roots and divisions, then the smallest k with dt / 2^k <= limit.
template <typename T, int SHAPE>
__device__ __forceinline__ int packet_level(const PushArgs<T> &a, const SubArgs<T> &sa, int64_t j)
{
    constexpr int NP = SHAPE == 1 ? 2 : 3;
    const uint32_t c = a.cell[j];
    const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
    if (ix >= a.nx || iy >= a.ny || iz >= a.nz)
        return 0;  // the push flags the packet and skips it
    T wx[3], wy[3], wz[3];
    int kx[3], ky[3], kz[3];
    axis_nodes(ix, axis_weights<SHAPE>(a.off0[j], wx), a.nx, kx);
    axis_nodes(iy, axis_weights<SHAPE>(a.off1[j], wy), a.ny, ky);
    axis_nodes(iz, axis_weights<SHAPE>(a.off2[j], wz), a.nz, kz);
    T B[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int cz = 0; cz < NP; ++cz) {
#pragma unroll
        for (int by = 0; by < NP; ++by) {
            const T wyz = wy[by] * wz[cz];
            const int64_t row = (int64_t(kz[cz]) * a.ny + ky[by]) * a.nx;
#pragma unroll
            for (int ax = 0; ax < NP; ++ax) {
                T F[6];
                load_node(a.fields + (row + kx[ax]) * 8, F);
                const T W = wx[ax] * wyz;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    B[q] += W * F[3 + q];
            }
        }
    }
    const T u[3] = {a.u0[j], a.u1[j], a.u2[j]};
    const T u2 = dot3(u, u);
    const T g = Math<T>::sqrt(T(1) + u2);
    const T beta = Math<T>::sqrt(u2) / g;
    const T bmag = Math<T>::sqrt(dot3(B, B));
    T lim = T(INFINITY);
    const T omega = sa.k_gyro * bmag / g;
    if (omega > T(0))
        lim = T(1) / omega;
    if (beta > T(0)) {
        const T t_cross = sa.k_cross / beta;
        lim = t_cross < lim ? t_cross : lim;
        if (sa.k_loss > T(0)) {
            const T t_loss = sa.k_loss / beta;
            lim = t_loss < lim ? t_loss : lim;
        }
    }
    lim = sa.courant * lim;
    int k = 0;
    T dts = sa.dt;
    while (k < sa.max_level && dts > lim) {
        dts *= T(0.5);
        ++k;
    }
    return k;
}

// Levels of all packets and the number of packets per level (one shared
// histogram per block, then one global add per level).
template <typename T, int SHAPE>
__global__ void __launch_bounds__(256) levels_kernel(PushArgs<T> a, SubArgs<T> sa)
{
    __shared__ uint32_t hist[kMaxLevel + 1];
    if (threadIdx.x <= kMaxLevel)
        hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < a.n; j += stride) {
        const int k = packet_level<T, SHAPE>(a, sa, j);
        sa.level[j] = uint8_t(k);
        atomicAdd(&hist[k], 1u);
    }
    __syncthreads();
    if (threadIdx.x <= kMaxLevel && hist[threadIdx.x])
        atomicAdd(&sa.counts[threadIdx.x], hist[threadIdx.x]);
}

// counts[k] -> cursor[k] = first slot of level k in the level-major order
// (highest level first), in place.  One thread.
static __global__ void level_offsets_kernel(uint32_t *counts, int max_level)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    uint32_t base = 0;
    for (int k = max_level; k >= 0; --k) {
        const uint32_t c = counts[k];
        counts[k] = base;
        base += c;
    }
}

// order[cursor[level]++] = j, one atomic per level present in each warp.
static __global__ void __launch_bounds__(256) bucket_kernel(int64_t n, const uint8_t *level, uint32_t *cursor,
                                                     uint32_t *order)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t n_round = (n + 31) & ~int64_t(31);
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n_round; j += stride) {
        const bool on = j < n;
        const int k = on ? int(level[j]) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (on && lane == leader)
            base = atomicAdd(&cursor[k], uint32_t(__popc(peers)));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (on)
            order[base + __popc(peers & ((1u << lane) - 1u))] = uint32_t(j);
    }
}

// The sub-cycled push: thread t advances packet order[t] by 2^k sub-steps of
// the per-packet body of every push kernel (gather, Boris, feedback, drift),
// with h, adv and the deposit scaled by 2^-k (exact in binary).
template <typename T, int SHAPE, bool DEPOSIT, bool DET>
__global__ void __launch_bounds__(256) push_subcycled_kernel(PushArgs<T> a, SubArgs<T> sa)
{
    int flag = 0;
    auto gather_node = [&](int64_t node, T F[6]) { load_node(a.fields + node * 8, F); };
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < a.n; t += stride) {
        const int64_t j = sa.order[t];
        const int k = sa.level[j];
        PushArgs<T> b = a;
        const T scale = T(1) / T(1u << k);
        b.k.h = a.k.h * scale;
        b.k.adv = a.k.adv * scale;
        b.k.qv = a.k.qv * scale;
        auto deposit_node = [&](int64_t node, T W, const T Q[8]) {
            if (DET)
                red_node_fixed(b.fx + node * 8, W, Q, b.fx_scale);
            else
                red_node(b.fb + node * 8, W, Q);
        };
        for (uint32_t s = 0; s < (1u << k); ++s)
            push_one<T, SHAPE, DEPOSIT>(b, j, gather_node, deposit_node, &flag);
    }
    if (flag)
        atomicOr(a.status, flag);
}

// Keys of the sorted sub-cycled step: level rank r = max_level - k (highest
// level first), then the bin-major key of the packet's stencil anchor (the
// cell for CIC, the nearest node for TSC), the key rsol_sort uses, so that
// each level's packets form bin ranges the binned kernel can tile.
template <typename T, int SHAPE>
__global__ void __launch_bounds__(256) level_keys_kernel(PushArgs<T> a, SubArgs<T> sa, int lb, int nbx,
                                                         int nby, uint32_t nbins,
                                                         uint32_t *__restrict__ keys)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const uint32_t m = (1u << lb) - 1u;
    int flag = 0;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < a.n; j += stride) {
        const uint32_t c = a.cell[j];
        int ax = cell_x(c), ay = cell_y(c), az = cell_z(c);
        if (ax >= a.nx || ay >= a.ny || az >= a.nz) {
            flag |= ST_BADCELL;
            keys[j] = 0xFFFFFFFFu;  // sorts after every bin: never pushed
            continue;
        }
        const int k = packet_level<T, SHAPE>(a, sa, j);
        if (SHAPE == 2) {
            ax += a.off0[j] >= T(0.5) ? 1 : 0;
            ay += a.off1[j] >= T(0.5) ? 1 : 0;
            az += a.off2[j] >= T(0.5) ? 1 : 0;
            ax -= ax == a.nx ? a.nx : 0;
            ay -= ay == a.ny ? a.ny : 0;
            az -= az == a.nz ? a.nz : 0;
        }
        const uint32_t bin_id = ((uint32_t(az) >> lb) * uint32_t(nby) + (uint32_t(ay) >> lb)) * uint32_t(nbx) +
                                (uint32_t(ax) >> lb);
        const uint32_t local = (((uint32_t(az) & m) << lb | (uint32_t(ay) & m)) << lb) | (uint32_t(ax) & m);
        const uint32_t r = uint32_t(sa.max_level - k);
        keys[j] = ((r * nbins + bin_id) << (3 * lb)) | local;
    }
    if (flag)
        atomicOr(a.status, flag);
}

template <typename T>
cudaError_t level_keys_dispatch(const PushDesc &d, const SubDesc &sd, int lb, int nbx, int nby,
                                uint32_t nbins, uint32_t *keys, cudaStream_t s)
{
    const PushArgs<T> a = make_push_args<T>(d);
    SubArgs<T> sa;
    sa.courant = T(sd.courant);
    sa.k_gyro = T(sd.k_gyro);
    sa.k_cross = T(sd.k_cross);
    sa.k_loss = T(sd.k_loss);
    sa.dt = T(sd.dt);
    sa.max_level = sd.max_level;
    sa.level = nullptr;
    sa.counts = nullptr;
    sa.order = nullptr;
    int64_t blocks = (d.n + 255) / 256;
    const int64_t cap = int64_t(d.sm_count) * 8 * 4;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    if (d.shape == 1)
        level_keys_kernel<T, 1><<<unsigned(blocks), 256, 0, s>>>(a, sa, lb, nbx, nby, nbins, keys);
    else
        level_keys_kernel<T, 2><<<unsigned(blocks), 256, 0, s>>>(a, sa, lb, nbx, nby, nbins, keys);
    return cudaGetLastError();
}

template <typename T>
cudaError_t subcycle_dispatch(const PushDesc &d, const SubDesc &sd, cudaStream_t s)
{
    const PushArgs<T> a = make_push_args<T>(d);
    SubArgs<T> sa;
    sa.courant = T(sd.courant);
    sa.k_gyro = T(sd.k_gyro);
    sa.k_cross = T(sd.k_cross);
    sa.k_loss = T(sd.k_loss);
    sa.dt = T(sd.dt);
    sa.max_level = sd.max_level;
    sa.level = sd.level;
    sa.counts = sd.counts;
    sa.order = sd.order;
    const int threads = 256;
    int64_t blocks = (d.n + threads - 1) / threads;
    const int64_t cap = int64_t(d.sm_count) * 8;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    cudaError_t e = cudaMemsetAsync(sd.counts, 0, sizeof(uint32_t) * (kMaxLevel + 1), s);
    if (e != cudaSuccess)
        return e;
    if (d.shape == 1)
        levels_kernel<T, 1><<<unsigned(blocks), threads, 0, s>>>(a, sa);
    else
        levels_kernel<T, 2><<<unsigned(blocks), threads, 0, s>>>(a, sa);
    level_offsets_kernel<<<1, 32, 0, s>>>(sd.counts, sd.max_level);
    bucket_kernel<<<unsigned(blocks), threads, 0, s>>>(d.n, sd.level, sd.counts, sd.order);
    const bool dep = d.fb != nullptr;
    const bool det = d.det != 0;
    // the push: more blocks than the level passes (each thread's work varies)
    int64_t pblocks = (d.n + threads - 1) / threads;
    const int64_t pcap = int64_t(d.sm_count) * 8 * 4;
    pblocks = pblocks > pcap ? pcap : (pblocks < 1 ? 1 : pblocks);
    const unsigned g = unsigned(pblocks);
    if (d.shape == 1) {
        if (!dep) push_subcycled_kernel<T, 1, false, false><<<g, threads, 0, s>>>(a, sa);
        else if (det) push_subcycled_kernel<T, 1, true, true><<<g, threads, 0, s>>>(a, sa);
        else push_subcycled_kernel<T, 1, true, false><<<g, threads, 0, s>>>(a, sa);
    } else {
        if (!dep) push_subcycled_kernel<T, 2, false, false><<<g, threads, 0, s>>>(a, sa);
        else if (det) push_subcycled_kernel<T, 2, true, true><<<g, threads, 0, s>>>(a, sa);
        else push_subcycled_kernel<T, 2, true, false><<<g, threads, 0, s>>>(a, sa);
    }
    return cudaGetLastError();
}

} // namespace rsol
