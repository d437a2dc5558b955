// Reverse-mode (adjoint) step of the packet push for the loss
//     L = || sum_n S^n ||_2,
// S^n the momentum source deposited on the nodes in step n (Sec. 2, force on
// the gas).  With Gbar = dL/d(sum_n S^n) = (sum_n S^n) / L the same grid for
// every step, the reverse of one step n needs the packet state at its start
// (x^n, u^n), the fields F^n and the adjoint state (xbar, ubar) of
// (x^{n+1}, u^{n+1}); it returns (xbar, ubar) of (x^n, u^n) and adds
// dL/dF^n to a node-major grid.  The forward quantities are recomputed
// from (x^n, u^n) in the same order as the forward step.
#pragma once

#include "push.cuh"
#include "rsol_device.cuh"
#include "rsol_internal.h"

namespace rsol {

template <typename T>
struct AdjArgs {
    int64_t n;
    const uint32_t *cell;
    const T *off0, *off1, *off2;
    const T *u0, *u1, *u2;
    const T *w;
    const T *fields;        // [node][8]: E, B at step n
    const T *fb;            // [node][8]: sum_n of the feedback; S in components 4..6
    const double *loss;     // device: L, 1/L
    T *xb0, *xb1, *xb2;     // dL/dx (cell units), in: step n+1, out: step n
    T *ub0, *ub1, *ub2;     // dL/du,               in: step n+1, out: step n
    T *fbar;                // [node][8]: dL/dF^n added to components 0..5
    int nx, ny, nz;
    StepConst<T> k;
    int *status;
};

// Derivatives of the one-axis factors of axis_weights with respect to f
// (the same branch for the anchor).
template <int SHAPE, typename T>
__device__ __forceinline__ void axis_dweights(T f, T dw[3])
{
    if (SHAPE == 1) {
        dw[0] = T(-1);
        dw[1] = T(1);
        dw[2] = T(0);
    } else {
        const T d = f >= T(0.5) ? f - T(1) : f;
        dw[0] = d - T(0.5);
        dw[1] = T(-2) * d;
        dw[2] = T(0.5) + d;
    }
}

__device__ __forceinline__ void load_s(const float *p, float S[3])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p + 4));
    S[0] = a.x; S[1] = a.y; S[2] = a.z;
}
__device__ __forceinline__ void load_s(const double *p, double S[3])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p + 4));
    S[0] = a.x; S[1] = a.y; S[2] = __ldg(p + 6);
}

__device__ __forceinline__ void red_field_bar(float *p, float W, const float Eb[3], const float Bb[3])
{
    atomicAdd(reinterpret_cast<float4 *>(p), make_float4(W * Eb[0], W * Eb[1], W * Eb[2], W * Bb[0]));
    atomicAdd(reinterpret_cast<float2 *>(p + 4), make_float2(W * Bb[1], W * Bb[2]));
}
__device__ __forceinline__ void red_field_bar(double *p, double W, const double Eb[3], const double Bb[3])
{
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        atomicAdd(p + q, W * Eb[q]);
        atomicAdd(p + 3 + q, W * Bb[q]);
    }
}

// a[i] for a runtime i in {0, 1, 2} without indexing a local array.
template <typename V>
__device__ __forceinline__ V sel3(const V a[3], int i)
{
    return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]);
}

// One packet: recompute gather, Boris and S at (x^n, u^n), then propagate the
// adjoint backwards through drift, deposit, Boris and gather.  The stencil's
// node values come from load(cz, by, ax, F[6], S[3]) (fields and the
// accumulated momentum source) and its share of dL/dF goes to
// scatter(cz, by, ax, W, Ebar, Bbar), so that the same arithmetic serves the
// global-memory and the tiled kernels.  xb, ub: adjoints of (x^{n+1}, u^{n+1})
// in, of (x^n, u^n) out.
template <typename T, int SHAPE, typename Load, typename Scatter>
__device__ __forceinline__ void adjoint_packet(const StepConst<T> &kc, T wj, T inv_L, T fx, T fy,
                                               T fz, const T u0[3], T xb[3], T ub[3], Load load,
                                               Scatter scatter, int *flag)
{
    constexpr int NP = SHAPE == 1 ? 2 : 3;
    T wx[3], wy[3], wz[3], dx[3], dy[3], dz[3];
    axis_weights<SHAPE>(fx, wx);
    axis_weights<SHAPE>(fy, wy);
    axis_weights<SHAPE>(fz, wz);
    axis_dweights<SHAPE>(fx, dx);
    axis_dweights<SHAPE>(fy, dy);
    axis_dweights<SHAPE>(fz, dz);

    // pass 1: E, B and Gbar at the packet (same order as the forward gather)
    // and their gradients with respect to the packet position, so that the
    // position adjoint needs no second pass over the nodes' values
    T E[3] = {T(0), T(0), T(0)}, B[3] = {T(0), T(0), T(0)}, G[3] = {T(0), T(0), T(0)};
    T dE[3][3] = {}, dB[3][3] = {}, dG[3][3] = {};   // [direction][component]
    // z planes one at a time (not unrolled: keeps the loads in flight to one
    // plane's nodes instead of all of them, and the registers below 128)
#pragma unroll 1
    for (int cz = 0; cz < NP; ++cz) {
        const T wzc = sel3(wz, cz), dzc = sel3(dz, cz);
#pragma unroll
        for (int by = 0; by < NP; ++by) {
            const T wyz = wy[by] * wzc;
            const T dyz = dy[by] * wzc;
            const T ydz = wy[by] * dzc;
#pragma unroll
            for (int ax = 0; ax < NP; ++ax) {
                const T W = wx[ax] * wyz;
                const T Wd[3] = {dx[ax] * wyz, wx[ax] * dyz, wx[ax] * ydz};
                T F[6], S[3];
                load(cz, by, ax, F, S);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    E[q] += W * F[q];
                    B[q] += W * F[3 + q];
                    G[q] += W * S[q];
                }
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        dE[d][q] += Wd[d] * F[q];
                        dB[d][q] += Wd[d] * F[3 + q];
                        dG[d][q] += Wd[d] * S[q];
                    }
            }
        }
    }

    // forward Boris with its intermediates (as boris())
    const T h = kc.h;
    T um[3], t[3], s[3], upr[3], up[3], u1[3], cr[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        um[q] = u0[q] + h * E[q];
    const T inv_gm = Math<T>::rsqrt(T(1) + dot3(um, um));
    const T hg = h * inv_gm;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        t[q] = hg * B[q];
    const T sf = Math<T>::div(T(2), T(1) + dot3(t, t));
#pragma unroll
    for (int q = 0; q < 3; ++q)
        s[q] = sf * t[q];
    cross3(um, t, cr);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        upr[q] = um[q] + cr[q];
    cross3(upr, s, cr);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        up[q] = um[q] + cr[q];
        u1[q] = up[q] + h * E[q];
    }
    const T inv_g1 = Math<T>::rsqrt(T(1) + dot3(u1, u1));
    const T wq = wj * kc.qv;
    const T half_ig = T(0.5) * inv_gm;
    T bb[3], Sj[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        bb[q] = (up[q] + um[q]) * half_ig;
    cross3(bb, B, cr);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        Sj[q] = -wq * (E[q] + cr[q]);

    // reverse: drift x^{n+1} = x^n + adv u1 / g1
    T u1b[3];
    {
        const T vb[3] = {kc.adv * xb[0], kc.adv * xb[1], kc.adv * xb[2]};
        const T uv = dot3(u1, vb) * inv_g1 * inv_g1;
        u1b[0] = ub[0] + inv_g1 * (vb[0] - u1[0] * uv);
        u1b[1] = ub[1] + inv_g1 * (vb[1] - u1[1] * uv);
        u1b[2] = ub[2] + inv_g1 * (vb[2] - u1[2] * uv);
    }
    // deposit: L depends on S_j through Gbar(x^n) . S_j
    T Sb[3], Eb[3], Bb[3], bbb[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        Sb[q] = inv_L * G[q];
    cross3(B, Sb, bbb);
    cross3(Sb, bb, Bb);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        Eb[q] = -wq * Sb[q];
        bbb[q] = -wq * bbb[q];
        Bb[q] = -wq * Bb[q];
    }
    // bb = (u+ + u-) / (2 g-)
    T upb[3], umb[3];
    T gmb = -dot3(bbb, bb) * inv_gm;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        upb[q] = bbb[q] * half_ig + u1b[q];   // u1 = u+ + h E
        umb[q] = bbb[q] * half_ig;
        Eb[q] += h * u1b[q];
    }
    // u+ = u- + u' x s
    T uprb[3], sb[3], tb[3];
    cross3(s, upb, uprb);
    cross3(upb, upr, sb);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        umb[q] += upb[q];
    // s = sf t, sf = 2 / (1 + t.t)
    const T ts = dot3(t, sb) * sf * sf;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        tb[q] = sf * sb[q] - t[q] * ts;
    // u' = u- + u- x t
    cross3(t, uprb, cr);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        umb[q] += uprb[q] + cr[q];
    cross3(uprb, um, cr);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        tb[q] += cr[q];
    // t = h B / g-
    gmb -= dot3(tb, t) * inv_gm;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        Bb[q] += hg * tb[q];
    // g- = sqrt(1 + u-.u-), u- = u0 + h E
    const T gk = gmb * inv_gm;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        umb[q] += gk * um[q];
        Eb[q] += h * umb[q];
    }

    // position adjoint: xbar^n = xbar^{n+1} + grad(E).Ebar + grad(B).Bbar
    // + grad(Gbar_raw).S_j / L  (the last from the x^n deposit weights)
    const T Sn[3] = {inv_L * Sj[0], inv_L * Sj[1], inv_L * Sj[2]};
    const T px = xb[0] + dot3(dE[0], Eb) + dot3(dB[0], Bb) + dot3(dG[0], Sn);
    const T py = xb[1] + dot3(dE[1], Eb) + dot3(dB[1], Bb) + dot3(dG[1], Sn);
    const T pz = xb[2] + dot3(dE[2], Eb) + dot3(dB[2], Bb) + dot3(dG[2], Sn);

    // pass 2: scatter dL/dF^n = W (Ebar, Bbar)
#pragma unroll
    for (int cz = 0; cz < NP; ++cz) {
#pragma unroll
        for (int by = 0; by < NP; ++by) {
            const T wyz = wy[by] * wz[cz];
#pragma unroll
            for (int ax = 0; ax < NP; ++ax)
                scatter(cz, by, ax, wx[ax] * wyz, Eb, Bb);
        }
    }
    if (!(Math<T>::finite(px) && Math<T>::finite(py) && Math<T>::finite(pz) &&
          Math<T>::finite(umb[0]) && Math<T>::finite(umb[1]) && Math<T>::finite(umb[2])))
        *flag |= ST_NONFINITE;
    xb[0] = px;
    xb[1] = py;
    xb[2] = pz;
    ub[0] = umb[0];
    ub[1] = umb[1];
    ub[2] = umb[2];
}

// One packet of the order-free kernel: stencil nodes read from and reduced
// into global memory.
template <typename T, int SHAPE>
__device__ __forceinline__ void adjoint_one(const AdjArgs<T> &a, int64_t j, T inv_L, int *flag)
{
    const uint32_t c = a.cell[j];
    const int ix = cell_x(c), iy = cell_y(c), iz = cell_z(c);
    if (ix >= a.nx || iy >= a.ny || iz >= a.nz) {
        *flag |= ST_BADCELL;
        return;
    }
    const T fx = a.off0[j], fy = a.off1[j], fz = a.off2[j];
    const T u0[3] = {a.u0[j], a.u1[j], a.u2[j]};
    T w3[3];
    int kx[3], ky[3], kz[3];
    axis_nodes(ix, axis_weights<SHAPE>(fx, w3), a.nx, kx);
    axis_nodes(iy, axis_weights<SHAPE>(fy, w3), a.ny, ky);
    axis_nodes(iz, axis_weights<SHAPE>(fz, w3), a.nz, kz);
    auto node = [&](int cz, int by, int ax) {
        return (int64_t(sel3(kz, cz)) * a.ny + ky[by]) * a.nx + kx[ax];
    };
    auto load = [&](int cz, int by, int ax, T F[6], T S[3]) {
        const int64_t nd = node(cz, by, ax);
        load_node(a.fields + nd * 8, F);
        load_s(a.fb + nd * 8, S);
    };
    auto scatter = [&](int cz, int by, int ax, T W, const T Eb[3], const T Bb[3]) {
        red_field_bar(a.fbar + node(cz, by, ax) * 8, W, Eb, Bb);
    };
    T xb[3] = {a.xb0[j], a.xb1[j], a.xb2[j]};
    T ub[3] = {a.ub0[j], a.ub1[j], a.ub2[j]};
    adjoint_packet<T, SHAPE>(a.k, a.w[j], inv_L, fx, fy, fz, u0, xb, ub, load, scatter, flag);
    a.xb0[j] = xb[0];
    a.xb1[j] = xb[1];
    a.xb2[j] = xb[2];
    a.ub0[j] = ub[0];
    a.ub1[j] = ub[1];
    a.ub2[j] = ub[2];
}


template <typename T, int SHAPE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) adjoint_kernel(AdjArgs<T> a)
{
    int flag = 0;
    const T inv_L = T(a.loss[1]);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < a.n; j += stride)
        adjoint_one<T, SHAPE>(a, j, inv_L, &flag);
    if (flag)
        atomicOr(a.status, flag);
}

// L^2 = sum over nodes of |S|^2 (components 4..6), FP64, fixed order:
// block partials, then one block for the total.
template <typename T>
__global__ void __launch_bounds__(256) loss_partials_kernel(const T *fb, int64_t n_nodes, double *partials)
{
    __shared__ double sh[256];
    double acc = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_nodes; i += stride) {
        const T *p = fb + i * 8 + 4;
        const double a = double(p[0]), b = double(p[1]), c = double(p[2]);
        acc += a * a + b * b + c * c;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        partials[blockIdx.x] = sh[0];
}

template <typename T>
AdjArgs<T> make_adj_args(const AdjDesc &d)
{
    AdjArgs<T> a;
    a.n = d.n;
    a.cell = d.cell;
    a.off0 = static_cast<const T *>(d.off[0]);
    a.off1 = static_cast<const T *>(d.off[1]);
    a.off2 = static_cast<const T *>(d.off[2]);
    a.u0 = static_cast<const T *>(d.u[0]);
    a.u1 = static_cast<const T *>(d.u[1]);
    a.u2 = static_cast<const T *>(d.u[2]);
    a.w = static_cast<const T *>(d.w);
    a.fields = static_cast<const T *>(d.fields);
    a.fb = static_cast<const T *>(d.fb);
    a.loss = d.loss;
    a.xb0 = static_cast<T *>(d.xb[0]);
    a.xb1 = static_cast<T *>(d.xb[1]);
    a.xb2 = static_cast<T *>(d.xb[2]);
    a.ub0 = static_cast<T *>(d.ub[0]);
    a.ub1 = static_cast<T *>(d.ub[1]);
    a.ub2 = static_cast<T *>(d.ub[2]);
    a.fbar = static_cast<T *>(d.fbar);
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.k.h = T(d.h);
    a.k.adv = T(d.adv);
    a.k.qv = T(d.qv);
    a.k.c = T(d.c);
    a.status = d.status;
    return a;
}

template <typename T>
cudaError_t launch_adjoint(const AdjDesc &d, cudaStream_t s)
{
    const AdjArgs<T> a = make_adj_args<T>(d);
    const int threads = 256;
    int64_t blocks = (d.n + threads - 1) / threads;
    const int64_t cap = int64_t(d.sm_count) * 8 * 4;
    blocks = blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
    if (d.shape == 1)
        adjoint_kernel<T, 1><<<unsigned(blocks), threads, 0, s>>>(a);
    else
        adjoint_kernel<T, 2><<<unsigned(blocks), threads, 0, s>>>(a);
    return cudaGetLastError();
}

static __global__ void __launch_bounds__(256) loss_final_kernel(const double *partials, int blocks, double *loss)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < blocks; i += blockDim.x)
        acc += partials[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double L = sqrt(sh[0]);
        loss[0] = L;
        loss[1] = L > 0.0 ? 1.0 / L : 0.0;
    }
}

} // namespace rsol
