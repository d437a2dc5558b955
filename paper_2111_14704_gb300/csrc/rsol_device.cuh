// Device-side building blocks of the RSOL packet step (Ji & Hopkins,
// arXiv:2111.14704, Sec. 2), templated on the arithmetic type.  Every kernel
// of librsol composes these; nothing here touches memory layout policy beyond
// the packed cell index and the node-major grids described in rsol.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsol {

// Device status bits (combined with atomicOr, read by rsol_check).
enum : int { ST_NONFINITE = 1, ST_COURANT = 2, ST_TIMEOUT = 4, ST_BADCELL = 8 };

constexpr int CELL_BITS = 10;
constexpr uint32_t CELL_MASK = (1u << CELL_BITS) - 1u;

__host__ __device__ __forceinline__ uint32_t pack_cell(int ix, int iy, int iz)
{
    return uint32_t(ix) | (uint32_t(iy) << CELL_BITS) | (uint32_t(iz) << (2 * CELL_BITS));
}
__device__ __forceinline__ int cell_x(uint32_t c) { return int(c & CELL_MASK); }
__device__ __forceinline__ int cell_y(uint32_t c) { return int((c >> CELL_BITS) & CELL_MASK); }
__device__ __forceinline__ int cell_z(uint32_t c) { return int(c >> (2 * CELL_BITS)); }

// Packed pairs of FP32 values for the f32x2 arithmetic of this GPU: one
// instruction performs two independent operations, each rounded exactly like
// the scalar instruction (fma.rn.f32x2 is two IEEE fused multiply-adds), so
// code written with them gives the same bits as the scalar code.
using f32x2 = unsigned long long;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// a * b + c, per half
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// a * b, per half
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Scalars of one step, precomputed on the host in double and rounded once.
template <typename T>
struct StepConst {
    T h;        // Boris half-step (c~/c)(q/m)/c * dt / 2   (Eq. momentum.alt)
    T adv;      // dt c~ / dx: cells moved per unit beta     (v_eff = c~ beta)
    T qv;       // q / dx^3: charge density of a unit-weight packet
    T c;        // true speed of light (current and energy source)
};

// Arithmetic policy: FP32 uses the fast hardware reciprocal square root; the
// FP64 build uses correctly rounded sqrt and division.
template <typename T> struct Math;
template <> struct Math<float> {
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float floor(float x) { return floorf(x); }
    static __device__ __forceinline__ bool finite(float x) { return isfinite(x); }
};
template <> struct Math<double> {
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double floor(double x) { return ::floor(x); }
    static __device__ __forceinline__ bool finite(double x) { return isfinite(x); }
};

// One-axis factors of the packet kernel W for x = i + f, f in [0, 1).
// Nodes are i + first + {0, 1, 2}.  CIC: (1 - f, f) on i, i+1.  TSC: around
// the nearest node j (j = i + 1 when f >= 1/2), d = x - j in [-1/2, 1/2):
// (1/2 - d)^2 / 2, 3/4 - d^2, (1/2 + d)^2 / 2 on j-1, j, j+1.
template <int SHAPE, typename T>
__device__ __forceinline__ int axis_weights(T f, T w[3])
{
    if (SHAPE == 1) {
        w[0] = T(1) - f;
        w[1] = f;
        w[2] = T(0);
        return 0;
    } else {
        const bool hi = f >= T(0.5);
        const T d = hi ? f - T(1) : f;
        const T a = T(0.5) - d;
        const T b = T(0.5) + d;
        w[0] = T(0.5) * a * a;
        w[1] = T(0.75) - d * d;
        w[2] = T(0.5) * b * b;
        return hi ? 0 : -1;
    }
}

// Wrapped node indices i + first + {0, 1, 2} on a periodic axis of n nodes.
__device__ __forceinline__ void axis_nodes(int i, int first, int n, int k[3])
{
    int k0 = i + first;
    k0 += (k0 < 0) ? n : 0;
    int k1 = k0 + 1;
    k1 -= (k1 >= n) ? n : 0;
    int k2 = k1 + 1;
    k2 -= (k2 >= n) ? n : 0;
    k[0] = k0;
    k[1] = k1;
    k[2] = k2;
}

template <typename T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Result of the Boris update of one packet.
template <typename T>
struct BorisOut {
    T u1[3];     // u^{n+1/2}
    T sum[3];    // u+ + u-
    T inv_gm;    // 1 / gamma at u-
    T inv_g1;    // 1 / gamma^{n+1/2}
};

// Boris kick-rotate-kick for d(gamma beta)/dt = (c~/c)(q/(m c))[E + beta x B]
// with h = (c~/c)(q/m)/c dt/2: u- = u0 + hE; t = hB/g-; s = 2t/(1+t^2);
// u' = u- + u- x t; u+ = u- + u' x s; u1 = u+ + hE.
template <typename T>
__device__ __forceinline__ BorisOut<T> boris(T h, const T E[3], const T B[3], const T u0[3])
{
    BorisOut<T> r;
    T um[3], t[3], s[3], up[3], cr[3], uprime[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        um[q] = u0[q] + h * E[q];
    r.inv_gm = Math<T>::rsqrt(T(1) + dot3(um, um));
    const T hg = h * r.inv_gm;
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
        uprime[q] = um[q] + cr[q];
    cross3(uprime, s, cr);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        up[q] = um[q] + cr[q];
        r.u1[q] = up[q] + h * E[q];
        r.sum[q] = up[q] + um[q];
    }
    r.inv_g1 = Math<T>::rsqrt(T(1) + dot3(r.u1, r.u1));
    return r;
}

// The eight feedback densities of one packet (weight w), per unit volume:
// rho = w q; J = w q c u1/g1; S = -w q [E + beta_bar x B], beta_bar = (u+ + u-)/(2 g-);
// H = -w q c E.(u+ + u-) / (g1 + g0).
template <typename T>
__device__ __forceinline__ void feedback(const StepConst<T> &k, T w, const T E[3], const T B[3],
                                         const BorisOut<T> &b, T g0, T Q[8])
{
    const T wq = w * k.qv;
    const T wqc = wq * k.c;
    Q[0] = wq;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        Q[1 + q] = wqc * (b.u1[q] * b.inv_g1);
    const T half_ig = T(0.5) * b.inv_gm;
    T bbar[3], bxB[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        bbar[q] = b.sum[q] * half_ig;
    cross3(bbar, B, bxB);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        Q[4 + q] = -wq * (E[q] + bxB[q]);
    const T g1 = Math<T>::div(T(1), b.inv_g1);
    Q[7] = -wqc * Math<T>::div(dot3(E, b.sum), g1 + g0);
}

// Drift of one axis with carry into the integer cell (periodic, n cells).
// Returns the new cell index; sets *flag on a non-finite or >1-cell move
// (the packet is then left where it was).
template <typename T>
__device__ __forceinline__ int drift_axis(int i, T &off, T delta, int n, int *flag)
{
    T o = off + delta;
    if (!Math<T>::finite(o)) {
        *flag |= ST_NONFINITE;
        return i;
    }
    T kf = Math<T>::floor(o);
    o = o - kf;
    int k = int(kf);
    if (o >= T(1)) {
        o = T(0);
        k += 1;
    }
    if (k < -1 || k > 1) {
        *flag |= ST_COURANT;
        k = ((k % n) + n) % n;
    }
    int j = i + k;
    j += (j < 0) ? n : 0;
    j -= (j >= n) ? n : 0;
    off = o;
    return j;
}

} // namespace rsol
