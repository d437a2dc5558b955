// Push + gather + feedback kernels (Sec. 2: Eq. momentum.alt, v_eff = c~ beta,
// force on the gas), templated on the arithmetic type and the packet kernel W.
// Instantiated once per precision in push_f32.cu / push_f64.cu.
#pragma once

#include "rsol_device.cuh"
#include "rsol_internal.h"

namespace rsol {

template <typename T>
struct PushArgs {
    int64_t n;
    uint32_t *cell;
    T *off0, *off1, *off2;
    T *u0, *u1, *u2;
    const T *w;
    const T *fields;        // [node][8]
    T *fb;                  // [node][8] or null
    long long *fx;          // [node][8] fixed-point accumulators (deterministic mode)
    int nx, ny, nz;
    StepConst<T> k;
    T fx_scale;             // 2^bits for the fixed-point deposit
    int *status;
    uint32_t *perm;         // binned kernel: per-bin visiting order scratch (n), or null
};

// Six field values of one node (E then B) from the node-major grid.
__device__ __forceinline__ void load_node(const float *p, float F[6])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float2 b = __ldg(reinterpret_cast<const float2 *>(p + 4));
    F[0] = a.x; F[1] = a.y; F[2] = a.z; F[3] = a.w; F[4] = b.x; F[5] = b.y;
}
__device__ __forceinline__ void load_node(const double *p, double F[6])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
    const double2 c = __ldg(reinterpret_cast<const double2 *>(p + 4));
    F[0] = a.x; F[1] = a.y; F[2] = b.x; F[3] = b.y; F[4] = c.x; F[5] = c.y;
}

// Add W * Q[0..7] to one node of the global feedback grid.
__device__ __forceinline__ void red_node(float *p, float W, const float Q[8])
{
    atomicAdd(reinterpret_cast<float4 *>(p), make_float4(W * Q[0], W * Q[1], W * Q[2], W * Q[3]));
    atomicAdd(reinterpret_cast<float4 *>(p + 4), make_float4(W * Q[4], W * Q[5], W * Q[6], W * Q[7]));
}
__device__ __forceinline__ void red_node(double *p, double W, const double Q[8])
{
#pragma unroll
    for (int q = 0; q < 8; ++q)
        atomicAdd(p + q, W * Q[q]);
}

__device__ __forceinline__ long long to_fixed(float v) { return __float2ll_rn(v); }
__device__ __forceinline__ long long to_fixed(double v) { return __double2ll_rn(v); }

template <typename T>
__device__ __forceinline__ void red_node_fixed(long long *p, T W, const T Q[8], T scale)
{
#pragma unroll
    for (int q = 0; q < 8; ++q)
        atomicAdd(reinterpret_cast<unsigned long long *>(p + q),
                  static_cast<unsigned long long>(to_fixed(W * Q[q] * scale)));
}

// Per-packet body shared by every push kernel: gather through `gather_node`,
// Boris, feedback (deposited through `deposit_node` when DEPOSIT), drift.
template <typename T, int SHAPE, bool DEPOSIT, typename Gather, typename Deposit>
__device__ __forceinline__ void push_one(const PushArgs<T> &a, int64_t j, Gather gather_node,
                                         Deposit deposit_node, int *flag)
{
    constexpr int NP = SHAPE == 1 ? 2 : 3;
    const uint32_t c = a.cell[j];
    const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
    if (ix >= a.nx || iy >= a.ny || iz >= a.nz) {  // caller passed a cell off the grid
        *flag |= ST_BADCELL;
        return;
    }
    T fx = a.off0[j], fy = a.off1[j], fz = a.off2[j];
    const T u0[3] = {a.u0[j], a.u1[j], a.u2[j]};
    T wx[3], wy[3], wz[3];
    int kx[3], ky[3], kz[3];
    axis_nodes(ix, axis_weights<SHAPE>(fx, wx), a.nx, kx);
    axis_nodes(iy, axis_weights<SHAPE>(fy, wy), a.ny, ky);
    axis_nodes(iz, axis_weights<SHAPE>(fz, wz), a.nz, kz);

    T E[3] = {T(0), T(0), T(0)}, B[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int cz = 0; cz < NP; ++cz) {
#pragma unroll
        for (int by = 0; by < NP; ++by) {
            const T wyz = wy[by] * wz[cz];
            const int64_t row = (int64_t(kz[cz]) * a.ny + ky[by]) * a.nx;
#pragma unroll
            for (int ax = 0; ax < NP; ++ax) {
                const T W = wx[ax] * wyz;
                T F[6];
                gather_node(row + kx[ax], F);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    E[q] += W * F[q];
                    B[q] += W * F[3 + q];
                }
            }
        }
    }

    const BorisOut<T> b = boris(a.k.h, E, B, u0);

    if (DEPOSIT) {
        const T g0 = Math<T>::sqrt(T(1) + dot3(u0, u0));
        T Q[8];
        feedback(a.k, a.w[j], E, B, b, g0, Q);
#pragma unroll
        for (int cz = 0; cz < NP; ++cz) {
#pragma unroll
            for (int by = 0; by < NP; ++by) {
                const T wyz = wy[by] * wz[cz];
                const int64_t row = (int64_t(kz[cz]) * a.ny + ky[by]) * a.nx;
#pragma unroll
                for (int ax = 0; ax < NP; ++ax)
                    deposit_node(row + kx[ax], wx[ax] * wyz, Q);
            }
        }
    }

    if (!(Math<T>::finite(b.u1[0]) && Math<T>::finite(b.u1[1]) && Math<T>::finite(b.u1[2]))) {
        *flag |= ST_NONFINITE;
        return;
    }
    const T s = a.k.adv * b.inv_g1;
    const int nx_ = drift_axis(ix, fx, s * b.u1[0], a.nx, flag);
    const int ny_ = drift_axis(iy, fy, s * b.u1[1], a.ny, flag);
    const int nz_ = drift_axis(iz, fz, s * b.u1[2], a.nz, flag);
    a.cell[j] = pack_cell(nx_, ny_, nz_);
    a.off0[j] = fx;
    a.off1[j] = fy;
    a.off2[j] = fz;
    a.u0[j] = b.u1[0];
    a.u1[j] = b.u1[1];
    a.u2[j] = b.u1[2];
}

// Order-free kernel: one packet per thread (grid-stride), gathers through the
// read-only cache, deposits with global vector atomics (or 64-bit fixed-point
// atomics in deterministic mode).
template <typename T, int SHAPE, bool DEPOSIT, bool DET>
__global__ void __launch_bounds__(256) push_unbinned_kernel(PushArgs<T> a)
{
    int flag = 0;
    auto gather_node = [&](int64_t node, T F[6]) { load_node(a.fields + node * 8, F); };
    auto deposit_node = [&](int64_t node, T W, const T Q[8]) {
        if (DET)
            red_node_fixed(a.fx + node * 8, W, Q, a.fx_scale);
        else
            red_node(a.fb + node * 8, W, Q);
    };
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < a.n; j += stride)
        push_one<T, SHAPE, DEPOSIT>(a, j, gather_node, deposit_node, &flag);
    if (flag)
        atomicOr(a.status, flag);
}

// Fixed-point accumulators -> feedback grid: fb += fx / scale, then fx = 0.
template <typename T>
__global__ void fixed_to_grid_kernel(long long *fx, T *fb, int64_t count, T inv_scale)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
        const long long v = fx[i];
        if (v != 0) {
            fb[i] += T(v) * inv_scale;
            fx[i] = 0;
        }
    }
}

template <typename T, int SHAPE, bool DEPOSIT, bool DET>
cudaError_t launch_unbinned(const PushArgs<T> &a, int sm_count, cudaStream_t s)
{
    const int threads = 256;
    int64_t blocks = (a.n + threads - 1) / threads;
    const int64_t cap = int64_t(sm_count) * 8 * 4;
    if (blocks > cap)
        blocks = cap;
    if (blocks < 1)
        blocks = 1;
    push_unbinned_kernel<T, SHAPE, DEPOSIT, DET><<<unsigned(blocks), threads, 0, s>>>(a);
    return cudaGetLastError();
}

} // namespace rsol

namespace rsol {

template <typename T>
struct MomArgs {
    int64_t n;
    const uint32_t *cell;
    const T *off0, *off1, *off2, *u0, *u1, *u2, *w;
    T *grid;
    long long *fx;
    int nx, ny, nz;
    T inv_vol, mc, mc2, qc, fx_scale;
};

// State moments (Sec. 2 packet totals per unit volume): n, N m c u, N gamma m c^2,
// N q c beta, deposited with the packet kernel W at the current positions.
template <typename T, int SHAPE, bool DET>
__global__ void __launch_bounds__(256) moments_grid_kernel(MomArgs<T> a)
{
    constexpr int NP = SHAPE == 1 ? 2 : 3;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < a.n; j += stride) {
        const uint32_t c = a.cell[j];
        if (cell_x(c) >= a.nx || cell_y(c) >= a.ny || cell_z(c) >= a.nz)
            continue;  // off-grid cells are reported by the push; skipped here
        const T u[3] = {a.u0[j], a.u1[j], a.u2[j]};
        const T g = Math<T>::sqrt(T(1) + dot3(u, u));
        const T N = a.w[j] * a.inv_vol;
        T Q[8];
        Q[0] = N;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            Q[1 + q] = N * a.mc * u[q];
        Q[4] = N * g * a.mc2;
        const T ig = Math<T>::div(T(1), g);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            Q[5 + q] = N * a.qc * (u[q] * ig);
        T wx[3], wy[3], wz[3];
        int kx[3], ky[3], kz[3];
        axis_nodes(cell_x(c), axis_weights<SHAPE>(a.off0[j], wx), a.nx, kx);
        axis_nodes(cell_y(c), axis_weights<SHAPE>(a.off1[j], wy), a.ny, ky);
        axis_nodes(cell_z(c), axis_weights<SHAPE>(a.off2[j], wz), a.nz, kz);
#pragma unroll
        for (int cz = 0; cz < NP; ++cz)
#pragma unroll
            for (int by = 0; by < NP; ++by) {
                const T wyz = wy[by] * wz[cz];
                const int64_t row = (int64_t(kz[cz]) * a.ny + ky[by]) * a.nx;
#pragma unroll
                for (int ax = 0; ax < NP; ++ax) {
                    const int64_t node = row + kx[ax];
                    if (DET)
                        red_node_fixed(a.fx + node * 8, wx[ax] * wyz, Q, a.fx_scale);
                    else
                        red_node(a.grid + node * 8, wx[ax] * wyz, Q);
                }
            }
    }
}

// FP64 totals, first level: block b reduces a fixed contiguous chunk of packets
// (and of feedback nodes) in a fixed order into partials[b][16].
template <typename T>
__global__ void __launch_bounds__(256) totals_kernel(const T *u0, const T *u1, const T *u2,
                                                     const T *w, int64_t n, const T *fb,
                                                     int64_t n_nodes, double mc, double mc2,
                                                     double qc, double vol, double *partials)
{
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q)
        acc[q] = 0.0;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = int64_t(blockIdx.x) * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        // gamma and beta in the packets' own precision (exact inputs, one
        // rounding each), every product and sum in FP64
        const T uf[3] = {u0[j], u1[j], u2[j]};
        const T gf = Math<T>::sqrt(T(1) + dot3(uf, uf));
        const T igf = T(1) / gf;
        const double N = double(w[j]);
        const double Nmc = N * mc, Nqc = N * qc;
        acc[0] += N;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            acc[1 + q] += Nmc * double(uf[q]);
        acc[4] += N * mc2 * double(gf);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            acc[5 + q] += Nqc * double(uf[q] * igf);
    }
    if (fb) {
        const int64_t cn = (n_nodes + gridDim.x - 1) / gridDim.x;
        const int64_t nlo = int64_t(blockIdx.x) * cn;
        const int64_t nhi = nlo + cn < n_nodes ? nlo + cn : n_nodes;
        for (int64_t i = nlo + threadIdx.x; i < nhi; i += blockDim.x)
#pragma unroll
            for (int q = 0; q < 8; ++q)
                acc[8 + q] += double(fb[i * 8 + q]) * vol;
    }
    __shared__ double red[256][17];
#pragma unroll
    for (int q = 0; q < 16; ++q)
        red[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < 16; ++q)
                red[threadIdx.x][q] += red[threadIdx.x + s][q];
        __syncthreads();
    }
    if (threadIdx.x < 16)
        partials[int64_t(blockIdx.x) * 16 + threadIdx.x] = red[0][threadIdx.x];
}

// Second level: one block sums the partials in a fixed order.
static __global__ void __launch_bounds__(256) totals_final_kernel(const double *partials, int blocks,
                                                          double *out)
{
    __shared__ double red[256][17];
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q)
        acc[q] = 0.0;
    for (int b = threadIdx.x; b < blocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 16; ++q)
            acc[q] += partials[int64_t(b) * 16 + q];
#pragma unroll
    for (int q = 0; q < 16; ++q)
        red[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < 16; ++q)
                red[threadIdx.x][q] += red[threadIdx.x + s][q];
        __syncthreads();
    }
    if (threadIdx.x < 16)
        out[threadIdx.x] = red[0][threadIdx.x];
}

// Catastrophic losses (Sec. 2 collisional terms): w *= exp(-(c~/c) sigma c beta n_n dt),
// beta at the packet's current momentum, n_n gathered with W from a node grid
// (one value per node) or uniform when nn is null.
template <typename T, int SHAPE>
__global__ void __launch_bounds__(256) losses_kernel(int64_t n, const uint32_t *__restrict__ cell,
                                                     const T *__restrict__ o0,
                                                     const T *__restrict__ o1,
                                                     const T *__restrict__ o2,
                                                     const T *__restrict__ u0,
                                                     const T *__restrict__ u1,
                                                     const T *__restrict__ u2, T *__restrict__ w,
                                                     const T *__restrict__ nn, T nn_uniform,
                                                     T coef, int nx, int ny, int nz, int *status)
{
    constexpr int NP = SHAPE == 1 ? 2 : 3;
    int flag = 0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride) {
        const T u[3] = {u0[j], u1[j], u2[j]};
        const T uu = dot3(u, u);
        const T beta = Math<T>::sqrt(uu) * Math<T>::rsqrt(T(1) + uu);
        T dens = nn_uniform;
        if (nn) {
            const uint32_t c = cell[j];
            const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
            if (ix >= nx || iy >= ny || iz >= nz) {
                flag |= ST_BADCELL;
                continue;
            }
            T wx[3], wy[3], wz[3];
            int kx[3], ky[3], kz[3];
            axis_nodes(ix, axis_weights<SHAPE>(o0[j], wx), nx, kx);
            axis_nodes(iy, axis_weights<SHAPE>(o1[j], wy), ny, ky);
            axis_nodes(iz, axis_weights<SHAPE>(o2[j], wz), nz, kz);
            dens = T(0);
#pragma unroll
            for (int cz = 0; cz < NP; ++cz)
#pragma unroll
                for (int cy = 0; cy < NP; ++cy) {
                    const T wyz = wy[cy] * wz[cz];
                    const int64_t row = (int64_t(kz[cz]) * ny + ky[cy]) * nx;
#pragma unroll
                    for (int cx = 0; cx < NP; ++cx)
                        dens += wx[cx] * wyz * nn[row + kx[cx]];
                }
        }
        w[j] *= exp(-coef * beta * dens);
    }
    if (flag)
        atomicOr(status, flag);
}

template <typename T>
cudaError_t losses_dispatch(const LossDesc &d, cudaStream_t s)
{
    int64_t blocks = (d.n + 255) / 256;
    const int64_t cap = int64_t(d.sm_count) * 16;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    auto go = [&](auto kern) {
        kern<<<unsigned(blocks), 256, 0, s>>>(
            d.n, d.cell, static_cast<const T *>(d.off[0]), static_cast<const T *>(d.off[1]),
            static_cast<const T *>(d.off[2]), static_cast<const T *>(d.u[0]),
            static_cast<const T *>(d.u[1]), static_cast<const T *>(d.u[2]), static_cast<T *>(d.w),
            static_cast<const T *>(d.nn), T(d.nn_uniform), T(d.coef), d.nx, d.ny, d.nz, d.status);
    };
    if (d.shape == 1)
        go(losses_kernel<T, 1>);
    else
        go(losses_kernel<T, 2>);
    return cudaGetLastError();
}

template <typename T>
PushArgs<T> make_push_args(const PushDesc &d)
{
    PushArgs<T> a;
    a.n = d.n;
    a.cell = d.cell;
    a.off0 = static_cast<T *>(d.off[0]);
    a.off1 = static_cast<T *>(d.off[1]);
    a.off2 = static_cast<T *>(d.off[2]);
    a.u0 = static_cast<T *>(d.u[0]);
    a.u1 = static_cast<T *>(d.u[1]);
    a.u2 = static_cast<T *>(d.u[2]);
    a.w = static_cast<const T *>(d.w);
    a.fields = static_cast<const T *>(d.fields);
    a.fb = static_cast<T *>(d.fb);
    a.fx = d.fx;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.k.h = T(d.h);
    a.k.adv = T(d.adv);
    a.k.qv = T(d.qv);
    a.k.c = T(d.c);
    a.fx_scale = T(d.fx_scale);
    a.status = d.status;
    a.perm = d.perm;
    return a;
}

template <typename T>
cudaError_t push_binned_dispatch(const PushDesc &d, cudaStream_t s);

template <typename T>
cudaError_t push_dispatch(const PushDesc &d, cudaStream_t s)
{
    if (d.tile_mode == 1 && d.fb != nullptr && d.bin_start != nullptr && (d.bin == 4 || d.bin == 8))
        return push_binned_dispatch<T>(d, s);
    const PushArgs<T> a = make_push_args<T>(d);
    const bool dep = d.fb != nullptr;
    const bool det = d.det != 0;
    if (d.shape == 1) {
        if (!dep) return launch_unbinned<T, 1, false, false>(a, d.sm_count, s);
        if (det) return launch_unbinned<T, 1, true, true>(a, d.sm_count, s);
        return launch_unbinned<T, 1, true, false>(a, d.sm_count, s);
    }
    if (!dep) return launch_unbinned<T, 2, false, false>(a, d.sm_count, s);
    if (det) return launch_unbinned<T, 2, true, true>(a, d.sm_count, s);
    return launch_unbinned<T, 2, true, false>(a, d.sm_count, s);
}

template <typename T>
cudaError_t moments_dispatch(const MomentsDesc &d, cudaStream_t s)
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
    a.fx = d.fx;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.inv_vol = T(d.inv_vol);
    a.mc = T(d.mc);
    a.mc2 = T(d.mc2);
    a.qc = T(d.qc);
    a.fx_scale = T(d.fx_scale);
    const int threads = 256;
    int64_t blocks = (d.n + threads - 1) / threads;
    const int64_t cap = int64_t(d.sm_count) * 8 * 4;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    if (d.shape == 1) {
        if (d.det) moments_grid_kernel<T, 1, true><<<unsigned(blocks), threads, 0, s>>>(a);
        else moments_grid_kernel<T, 1, false><<<unsigned(blocks), threads, 0, s>>>(a);
    } else {
        if (d.det) moments_grid_kernel<T, 2, true><<<unsigned(blocks), threads, 0, s>>>(a);
        else moments_grid_kernel<T, 2, false><<<unsigned(blocks), threads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t totals_dispatch(const TotalsDesc &d, cudaStream_t s)
{
    totals_kernel<T><<<d.blocks, 256, 0, s>>>(
        static_cast<const T *>(d.u[0]), static_cast<const T *>(d.u[1]),
        static_cast<const T *>(d.u[2]), static_cast<const T *>(d.w), d.n,
        static_cast<const T *>(d.fb), d.n_nodes, d.mc, d.mc2, d.qc, d.vol, d.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    totals_final_kernel<<<1, 256, 0, s>>>(d.partials, d.blocks, d.out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fixed_dispatch(long long *fx, void *grid, int64_t count, double inv_scale,
                           int sm_count, cudaStream_t s)
{
    int64_t blocks = (count + 255) / 256;
    const int64_t cap = int64_t(sm_count) * 16;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    fixed_to_grid_kernel<T><<<unsigned(blocks), 256, 0, s>>>(fx, static_cast<T *>(grid), count,
                                                             T(inv_scale));
    return cudaGetLastError();
}

} // namespace rsol
