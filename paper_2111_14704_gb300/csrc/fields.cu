// Analytic field source standing in for the MHD solver (out of scope of the
// packet step): B0 x-hat plus a superposition of Alfven modes, and the
// ideal-MHD electric field E = -(u/c) x B of Sec. 2 (below Eq. momentum).
//
// cos(2 pi n.r/L - omega t + phi) is evaluated as Re(Tx * Ty * Tz) with
// per-mode, per-axis phase tables T_a[m][i] = exp(2 pi i n_a i / N_a) built in
// double from exactly reduced integer phases; the time-dependent phase
// psi_m = phi_m - sigma_m k_x vA t (reduced on the host) is folded into Tx by
// the table kernel.  One block per (y, z) row of nodes.
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "rsol_device.cuh"
#include "rsol_internal.h"

namespace rsol {

namespace {

struct ModeCoef {
    double cB[3];   // A_m e_m
    double cu[3];   // -sigma_m vA A_m e_m / B0
    double psi;     // phi_m - omega_m t, reduced to [0, 2 pi)
    int n[3];
};

constexpr int MAX_MODES = 256;

// Mode table passed by value as a kernel parameter (no host staging buffer,
// so the launch can be captured in a CUDA graph).
struct ModeSet {
    ModeCoef m[MAX_MODES];
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Per-mode coefficients (cB, cu as T) and phase tables: for mode m the complex
// entries (re, im) of axis x (nx), then y (ny), then z (nz).
// When tabx_t is given, the x entries are also written mode-fastest:
// tabx_t[(i * n_modes + m) * 2 + {0, 1}].
template <typename T>
__global__ void tables_kernel(const ModeSet modes, int n_modes, int nx, int ny, int nz,
                              T *__restrict__ coef, T *__restrict__ tab, T *__restrict__ tabx_t = nullptr)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_modes; m += gridDim.x * blockDim.x)
        for (int q = 0; q < 3; ++q) {
            coef[6 * m + q] = T(modes.m[m].cB[q]);
            coef[6 * m + 3 + q] = T(modes.m[m].cu[q]);
        }
    const int len = nx + ny + nz;
    const int64_t total = int64_t(n_modes) * len;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int m = int(t / len);
        int i = int(t % len);
        int axis = 0, N = nx;
        if (i >= nx) {
            i -= nx;
            axis = 1;
            N = ny;
            if (i >= ny) {
                i -= ny;
                axis = 2;
                N = nz;
            }
        }
        const ModeCoef &mc = modes.m[m];
        // exact integer phase reduction: turns = (n_a * i mod N) / N
        long long r = (static_cast<long long>(mc.n[axis]) * i) % N;
        if (r < 0)
            r += N;
        double ang = 2.0 * double(r) / double(N);  // in units of pi
        double s, c;
        sincospi(ang, &s, &c);
        if (axis == 0) {
            double sp, cp;
            sincos(mc.psi, &sp, &cp);
            const double re = c * cp - s * sp;
            const double im = s * cp + c * sp;
            c = re;
            s = im;
        }
        tab[2 * t] = T(c);
        tab[2 * t + 1] = T(s);
        if (tabx_t && axis == 0) {
            tabx_t[(int64_t(i) * n_modes + m) * 2] = T(c);
            tabx_t[(int64_t(i) * n_modes + m) * 2 + 1] = T(s);
        }
    }
}

// FP64: one block per (iy, iz) row: the per-mode product Ty * Tz is formed
// once per row in shared memory, packed with the mode's coefficients into
// words {cB, cu_x} {cu_y, cu_z, w_re, w_im}; each thread then needs only Tx at
// its node.  The sum runs over the modes in order (one chain per component).
template <typename T>
struct alignas(16) ModePack {
    T v[8];
};

template <typename T>
__device__ __forceinline__ void load_pack(const ModePack<T> &p, T v[8])
{
    if constexpr (sizeof(T) == 4) {
        const float4 a = reinterpret_cast<const float4 *>(p.v)[0];
        const float4 b = reinterpret_cast<const float4 *>(p.v)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            const double2 a = reinterpret_cast<const double2 *>(p.v)[k / 2];
            v[k] = a.x;
            v[k + 1] = a.y;
        }
    }
}

// the eight field values of one node (E, B, two zero pads) with 16-byte stores
__device__ __forceinline__ void store_node8(float *f, const float v[6])
{
    reinterpret_cast<float4 *>(f)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4 *>(f)[1] = make_float4(v[4], v[5], 0.f, 0.f);
}
__device__ __forceinline__ void store_node8(double *f, const double v[6])
{
    reinterpret_cast<double2 *>(f)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(f)[1] = make_double2(v[2], v[3]);
    reinterpret_cast<double2 *>(f)[2] = make_double2(v[4], v[5]);
    reinterpret_cast<double2 *>(f)[3] = make_double2(0.0, 0.0);
}

template <typename T>
__global__ void __launch_bounds__(128) alfven_kernel(const T *__restrict__ coef,
                                                     int n_modes, const T *__restrict__ tab,
                                                     int nx, int ny, int nz, T B0, T ugx, T ugy,
                                                     T ugz, T inv_c, T *__restrict__ fields)
{
    __shared__ ModePack<T> s_p[MAX_MODES];
    const int iy = blockIdx.y;
    const int iz = blockIdx.z;
    const int len = nx + ny + nz;
    for (int m = threadIdx.x; m < n_modes; m += blockDim.x) {
        ModePack<T> p;
        for (int q = 0; q < 6; ++q)
            p.v[q] = coef[6 * m + q];
        const T *t = tab + int64_t(m) * len * 2;
        const T yr = t[2 * (nx + iy)], yi = t[2 * (nx + iy) + 1];
        const T zr = t[2 * (nx + ny + iz)], zi = t[2 * (nx + ny + iz) + 1];
        p.v[6] = yr * zr - yi * zi;
        p.v[7] = yr * zi + yi * zr;
        s_p[m] = p;
    }
    __syncthreads();
    for (int ix = blockIdx.x * blockDim.x + threadIdx.x; ix < nx; ix += gridDim.x * blockDim.x) {
        T B[3] = {B0, T(0), T(0)};
        T u[3] = {ugx, ugy, ugz};
        const T *t = tab + 2 * ix;
#pragma unroll 4
        for (int m = 0; m < n_modes; ++m, t += int64_t(len) * 2) {
            const T xr = t[0], xi = t[1];
            T c[8];
            load_pack(s_p[m], c);
            const T cs = xr * c[6] - xi * c[7];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                B[q] += c[q] * cs;
                u[q] += c[3 + q] * cs;
            }
        }
        // E = -(u / c) x B
        const T v[6] = {-(u[1] * B[2] - u[2] * B[1]) * inv_c, -(u[2] * B[0] - u[0] * B[2]) * inv_c,
                        -(u[0] * B[1] - u[1] * B[0]) * inv_c, B[0], B[1], B[2]};
        store_node8(fields + ((int64_t(iz) * ny + iy) * nx + ix) * 8, v);
    }
}

// FP32: a block of AF_ROWS warps takes AF_ROWS (y, z) rows of one z plane;
// lane l of warp w takes the nodes x = l + 32 k of row w, AF_NODES of them at
// a time, so that each mode's coefficients and row phase (shared-memory
// broadcasts) are read once per AF_NODES nodes instead of once per node: a
// kernel with one node per thread is bound by L1/shared-memory throughput,
// not arithmetic.  Only the first node's x phase is read per mode; the other
// nodes' (32, 64, 96 nodes on) follow by complex rotation, a few float
// roundings from the table's values.  Each node's six sums run over the modes
// in order, in f32x2 pairs {Bx, By}, {Bz, ux}, {uy, uz}.
constexpr int AF_ROWS = 4, AF_NODES = 4;

__global__ void __launch_bounds__(32 * AF_ROWS) alfven_rows_kernel(
    const float *__restrict__ coef, int n_modes, const float *__restrict__ tab, int nx, int ny,
    int nz, float B0, float ugx, float ugy, float ugz, float inv_c, float *__restrict__ fields)
{
    // dynamic shared memory, n_modes entries each: {cB_x, cB_y, cB_z, cu_x},
    // {cu_y, cu_z}, the rotation Tx(x + 32) / Tx(x), then Ty * Tz of each of
    // the AF_ROWS rows
    extern __shared__ float4 af_smem[];
    float4 *s_c0 = af_smem;
    float2 *s_c1 = reinterpret_cast<float2 *>(s_c0 + n_modes);
    float2 *s_r = s_c1 + n_modes;
    float2 *s_w = s_r + n_modes;  // [row][mode]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int iz = blockIdx.z, iy0 = blockIdx.y * AF_ROWS;
    const int len = nx + ny + nz;
    for (int m = threadIdx.x; m < n_modes; m += blockDim.x) {
        s_c0[m] = make_float4(coef[6 * m], coef[6 * m + 1], coef[6 * m + 2], coef[6 * m + 3]);
        s_c1[m] = make_float2(coef[6 * m + 4], coef[6 * m + 5]);
        const float *t = tab + int64_t(m) * len * 2;
        // |Tx| = 1: Tx(32) conj(Tx(0)) = exp(2 pi i n_x 32 / nx), the step of 32 nodes
        s_r[m] = nx > 32 ? make_float2(t[64] * t[0] + t[65] * t[1], t[65] * t[0] - t[64] * t[1])
                         : make_float2(1.f, 0.f);
        const float zr = t[2 * (nx + ny + iz)], zi = t[2 * (nx + ny + iz) + 1];
        for (int r = 0; r < AF_ROWS && iy0 + r < ny; ++r) {
            const float yr = t[2 * (nx + iy0 + r)], yi = t[2 * (nx + iy0 + r) + 1];
            s_w[r * n_modes + m] = make_float2(yr * zr - yi * zi, yr * zi + yi * zr);
        }
    }
    __syncthreads();
    const int iy = iy0 + warp;
    if (iy >= ny)
        return;
    for (int x0 = 0; x0 < nx; x0 += 32 * AF_NODES) {
        f32x2 s01[AF_NODES], s23[AF_NODES], s45[AF_NODES];
#pragma unroll
        for (int k = 0; k < AF_NODES; ++k) {
            s01[k] = f2_pack(B0, 0.f);
            s23[k] = f2_pack(0.f, ugx);
            s45[k] = f2_pack(ugy, ugz);
        }
        // node x0 + lane's phase is read from the table, the next ones (32 nodes
        // apart) are rotated from it; nodes past the row's end are not stored
        const bool any = x0 + lane < nx;
        const float *t = tab + 2 * (any ? x0 + lane : 0);
#pragma unroll 2
        for (int m = 0; m < n_modes; ++m, t += int64_t(len) * 2) {
            const ulonglong2 c0 = *reinterpret_cast<const ulonglong2 *>(&s_c0[m]);
            const float2 c1 = s_c1[m];
            const float2 w = s_w[warp * n_modes + m];
            const float2 rot = s_r[m];
            const f32x2 cu = f2_pack(c1.x, c1.y);
            float2 x = *reinterpret_cast<const float2 *>(t);
#pragma unroll
            for (int k = 0; k < AF_NODES; ++k) {
                if (k > 0)
                    x = make_float2(x.x * rot.x - x.y * rot.y, x.x * rot.y + x.y * rot.x);
                const float cs = x.x * w.x - x.y * w.y;
                const f32x2 cs2 = f2_pack(cs, cs);
                s01[k] = f2_fma(c0.x, cs2, s01[k]);
                s23[k] = f2_fma(c0.y, cs2, s23[k]);
                s45[k] = f2_fma(cu, cs2, s45[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < AF_NODES; ++k) {
            const int ix = x0 + lane + 32 * k;
            if (ix >= nx)
                continue;
            float B[3], u[3];
            f2_unpack(s01[k], B[0], B[1]);
            f2_unpack(s23[k], B[2], u[0]);
            f2_unpack(s45[k], u[1], u[2]);
            // E = -(u / c) x B
            const float v[6] = {-(u[1] * B[2] - u[2] * B[1]) * inv_c, -(u[2] * B[0] - u[0] * B[2]) * inv_c,
                                -(u[0] * B[1] - u[1] * B[0]) * inv_c, B[0], B[1], B[2]};
            store_node8(fields + ((int64_t(iz) * ny + iy) * nx + ix) * 8, v);
        }
    }
}

struct AdjModeSet {
    double a[MAX_MODES * 4];
};

template <typename T>
__global__ void acoef_kernel(const AdjModeSet set, int n_modes, T *__restrict__ acoef)
{
    for (int i = threadIdx.x; i < 4 * n_modes; i += blockDim.x)
        acoef[i] = T(set.a[i]);
}

// Adjoint of alfven_kernel with respect to the amplitudes A_m, one block per
// (iy, iz) row.  Given Fbar = dL/dF at each node: with E = -(u/c) x B,
//   ubar = -(1/c) B x Ebar,   Bbar_tot = Bbar - (1/c) Ebar x u,
// and since dB/dA_m = e_m cos_m, du/dA_m = kk_m e_m cos_m (kk_m = -sigma_m vA / B0),
//   dL/dA_m = sum over nodes of cos_m e_m . (Bbar_tot + kk_m ubar).
// Phase A (a thread per node) forms Bbar_tot and ubar of up to 128 nodes in
// shared memory; phase B (a thread per mode) sums its mode's terms over them
// in node order, reading the x phase table mode-fastest (coalesced).  The
// block writes one FP64 partial per mode; amp_reduce_kernel adds the
// partials in row order, so the result does not depend on scheduling.  When
// fbar_total is given, Fbar is also added into it and zeroed.
template <typename T>
__global__ void __launch_bounds__(128) alfven_adjoint_kernel(
    const T *__restrict__ coef, const T *__restrict__ acoef, int n_modes,
    const T *__restrict__ tab, const T *__restrict__ tabx_t, int nx, int ny, int nz, T B0, T ugx,
    T ugy, T ugz, T inv_c, T *__restrict__ fbar, T *__restrict__ fbar_total,
    double *__restrict__ partials)
{
    constexpr int CH = 128;
    // per mode {cB, cu, Ty Tz} in 16-byte words (phase A reads a mode in two
    // vector loads), and {e_m, kk_m} for phase B
    __shared__ ModePack<T> s_p[MAX_MODES];
    __shared__ T s_a[MAX_MODES][4];
    __shared__ T s_v[CH][6];
    const int iy = blockIdx.y;
    const int iz = blockIdx.z;
    const int len = nx + ny + nz;
    for (int m = threadIdx.x; m < n_modes; m += blockDim.x) {
        ModePack<T> p;
        for (int q = 0; q < 6; ++q)
            p.v[q] = coef[6 * m + q];
        for (int q = 0; q < 4; ++q)
            s_a[m][q] = acoef[4 * m + q];
        const T *t = tab + int64_t(m) * len * 2;
        const T yr = t[2 * (nx + iy)], yi = t[2 * (nx + iy) + 1];
        const T zr = t[2 * (nx + ny + iz)], zi = t[2 * (nx + ny + iz) + 1];
        p.v[6] = yr * zr - yi * zi;
        p.v[7] = yr * zi + yi * zr;
        s_p[m] = p;
    }
    // per-mode accumulators: thread threadIdx.x owns modes threadIdx.x + k * blockDim.x
    constexpr int MPT = (MAX_MODES + 127) / 128;
    // phase-B layout: modes rounded up to a warp, R node phases per mode
    const int nm_r = (n_modes + 31) & ~31;
    const int R = nm_r >= int(blockDim.x) ? 1 : int(blockDim.x) / nm_r;
    T acc[MPT];
#pragma unroll
    for (int k = 0; k < MPT; ++k)
        acc[k] = T(0);
    __syncthreads();
    for (int x0 = 0; x0 < nx; x0 += CH) {
        const int cnt = nx - x0 < CH ? nx - x0 : CH;
        // phase A
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int ix = x0 + i;
            // two interleaved chains over the modes (independent FMAs in flight)
            T B[3] = {B0, T(0), T(0)}, B2[3] = {T(0), T(0), T(0)};
            T u[3] = {ugx, ugy, ugz}, u2[3] = {T(0), T(0), T(0)};
            using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
            int m = 0;
            for (; m + 1 < n_modes; m += 2) {
                const T *t = tab + int64_t(m) * len * 2;
                const T2 x = *reinterpret_cast<const T2 *>(t + 2 * ix);
                const T2 x2 = *reinterpret_cast<const T2 *>(t + int64_t(len) * 2 + 2 * ix);
                T c[8], c2[8];
                load_pack(s_p[m], c);
                load_pack(s_p[m + 1], c2);
                const T cs = x.x * c[6] - x.y * c[7];
                const T cs2 = x2.x * c2[6] - x2.y * c2[7];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    B[q] += c[q] * cs;
                    u[q] += c[3 + q] * cs;
                    B2[q] += c2[q] * cs2;
                    u2[q] += c2[3 + q] * cs2;
                }
            }
            if (m < n_modes) {
                const T *t = tab + int64_t(m) * len * 2;
                const T2 x = *reinterpret_cast<const T2 *>(t + 2 * ix);
                T c[8];
                load_pack(s_p[m], c);
                const T cs = x.x * c[6] - x.y * c[7];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    B[q] += c[q] * cs;
                    u[q] += c[3 + q] * cs;
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                B[q] += B2[q];
                u[q] += u2[q];
            }
            T *f = fbar + ((int64_t(iz) * ny + iy) * nx + ix) * 8;
            const T Eb[3] = {f[0], f[1], f[2]};
            const T Bb[3] = {f[3], f[4], f[5]};
            if (fbar_total) {
                T *ft = fbar_total + ((int64_t(iz) * ny + iy) * nx + ix) * 8;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    ft[q] += f[q];
                    f[q] = T(0);
                }
            }
            s_v[i][0] = Bb[0] - (Eb[1] * u[2] - Eb[2] * u[1]) * inv_c;
            s_v[i][1] = Bb[1] - (Eb[2] * u[0] - Eb[0] * u[2]) * inv_c;
            s_v[i][2] = Bb[2] - (Eb[0] * u[1] - Eb[1] * u[0]) * inv_c;
            s_v[i][3] = -(B[1] * Eb[2] - B[2] * Eb[1]) * inv_c;
            s_v[i][4] = -(B[2] * Eb[0] - B[0] * Eb[2]) * inv_c;
            s_v[i][5] = -(B[0] * Eb[1] - B[1] * Eb[0]) * inv_c;
        }
        __syncthreads();
        // phase B: thread (m, r) sums nodes r, r + R, ... of the chunk for mode m
#pragma unroll
        for (int k = 0; k < MPT; ++k) {
            const int slot_id = threadIdx.x + k * blockDim.x;
            const int m = slot_id % nm_r, r = slot_id / nm_r;
            if (m < n_modes && r < R) {
                const T wr = s_p[m].v[6], wi = s_p[m].v[7];
                const T e0 = s_a[m][0], e1 = s_a[m][1], e2 = s_a[m][2], kk = s_a[m][3];
                T a = acc[k];
                for (int i = r; i < cnt; i += R) {
                    const T *tx = tabx_t + (int64_t(x0 + i) * n_modes + m) * 2;
                    const T cs = tx[0] * wr - tx[1] * wi;
                    a += cs * (e0 * (s_v[i][0] + kk * s_v[i][3]) + e1 * (s_v[i][1] + kk * s_v[i][4]) +
                               e2 * (s_v[i][2] + kk * s_v[i][5]));
                }
                acc[k] = a;
            }
        }
        __syncthreads();
    }
    // the R partial sums of each mode, added in r order
    __shared__ double s_part[128 * MPT];
#pragma unroll
    for (int k = 0; k < MPT; ++k)
        s_part[threadIdx.x + k * blockDim.x] = double(acc[k]);
    __syncthreads();
    const int64_t row = int64_t(iz) * ny + iy;
    for (int m = threadIdx.x; m < n_modes; m += blockDim.x) {
        double sum = 0.0;
        for (int r = 0; r < R; ++r)
            sum += s_part[r * nm_r + m];
        partials[row * n_modes + m] = sum;
    }
}

// amp_bar[m] += sum over rows of partials[row][m], in row order (one block per mode).
__global__ void __launch_bounds__(256) amp_reduce_kernel(const double *__restrict__ partials,
                                                         int64_t rows, int n_modes,
                                                         double *__restrict__ amp_bar)
{
    __shared__ double sh[256];
    const int m = blockIdx.x;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x)
        acc += partials[r * n_modes + m];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        amp_bar[m] += sh[0];
}

} // namespace

namespace {

// Host-side mode coefficients: integer wave numbers, A e, -sigma vA A e / B0 and
// the time-dependent phase psi = phi - sigma k_x vA t reduced to [0, 2 pi).
void fill_modes(ModeSet &hm, const double *h_modes, const double *h_sigma, int n_modes, double t,
                double B0, double vA, double dx, int nx)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < n_modes; ++m) {
        const double *r = h_modes + 8 * m;
        ModeCoef &mc = hm.m[m];
        for (int q = 0; q < 3; ++q) {
            mc.n[q] = int(std::lround(r[q]));
            mc.cB[q] = r[6] * r[3 + q];
            mc.cu[q] = -h_sigma[m] * vA * r[6] * r[3 + q] / B0;
        }
        const double kx = two_pi * mc.n[0] / (nx * dx);
        const double omega = h_sigma[m] * kx * vA;
        double psi = std::fmod(r[7] - omega * t, two_pi);
        if (psi < 0)
            psi += two_pi;
        mc.psi = psi;
    }
}

} // namespace

size_t alfven_scratch_bytes(int nx, int ny, int nz, int n_modes)
{
    return align_up(size_t(n_modes) * 6 * sizeof(double)) +
           align_up(size_t(n_modes) * (nx + ny + nz) * 2 * sizeof(double));
}

cudaError_t alfven_fields(const double *h_modes, const double *h_sigma, int n_modes, double t,
                          double B0, double vA, const double *u_gas, double c, double dx,
                          int nx, int ny, int nz, int precision, void *fields, void *scratch,
                          cudaStream_t s)
{
    if (n_modes < 0 || n_modes > MAX_MODES)
        return cudaErrorInvalidValue;
    static thread_local ModeSet hm;
    fill_modes(hm, h_modes, h_sigma, n_modes, t, B0, vA, dx, nx);
    const size_t esz = precision == 32 ? sizeof(float) : sizeof(double);
    void *coef = scratch;
    void *tab = static_cast<char *>(scratch) + align_up(size_t(n_modes) * 6 * esz);
    const int64_t entries = int64_t(n_modes) * (nx + ny + nz);
    const int tb = int((entries + 255) / 256) > 0 ? int((entries + 255) / 256) : 1;
    const dim3 grid(1, ny, nz);
    if (precision == 32) {
        tables_kernel<float><<<tb, 256, 0, s>>>(hm, n_modes, nx, ny, nz,
                                                static_cast<float *>(coef),
                                                static_cast<float *>(tab));
        const dim3 rows(1, unsigned((ny + AF_ROWS - 1) / AF_ROWS), unsigned(nz));
        const size_t smem = size_t(n_modes) * (sizeof(float4) + sizeof(float2) * (2 + AF_ROWS));
        alfven_rows_kernel<<<rows, 32 * AF_ROWS, smem, s>>>(
            static_cast<const float *>(coef), n_modes, static_cast<const float *>(tab), nx, ny,
            nz, float(B0), float(u_gas[0]), float(u_gas[1]), float(u_gas[2]), float(1.0 / c),
            static_cast<float *>(fields));
    } else {
        tables_kernel<double><<<tb, 256, 0, s>>>(hm, n_modes, nx, ny, nz,
                                                 static_cast<double *>(coef),
                                                 static_cast<double *>(tab));
        alfven_kernel<double><<<grid, 128, 0, s>>>(
            static_cast<const double *>(coef), n_modes, static_cast<const double *>(tab), nx,
            ny, nz, B0, u_gas[0], u_gas[1], u_gas[2], 1.0 / c, static_cast<double *>(fields));
    }
    return cudaGetLastError();
}

} // namespace rsol

namespace rsol {

size_t alfven_adjoint_scratch_bytes(int nx, int ny, int nz, int n_modes)
{
    return alfven_scratch_bytes(nx, ny, nz, n_modes) + align_up(size_t(n_modes) * 4 * sizeof(double)) +
           align_up(size_t(ny) * nz * n_modes * sizeof(double)) +
           align_up(size_t(n_modes) * nx * 2 * sizeof(double));
}

cudaError_t alfven_adjoint(const double *h_modes, const double *h_sigma, int n_modes, double t,
                           double B0, double vA, const double *u_gas, double c, double dx, int nx,
                           int ny, int nz, int precision, void *fbar, void *fbar_total,
                           double *amp_bar, void *scratch, cudaStream_t s)
{
    if (n_modes < 1 || n_modes > MAX_MODES)
        return cudaErrorInvalidValue;
    static thread_local ModeSet hm;
    fill_modes(hm, h_modes, h_sigma, n_modes, t, B0, vA, dx, nx);
    // d/dA coefficients: e_m and kk_m = -sigma_m vA / B0 (kernel parameter, so
    // that the call can be captured in a CUDA graph)
    static thread_local AdjModeSet ac;
    for (int m = 0; m < n_modes; ++m) {
        for (int q = 0; q < 3; ++q)
            ac.a[4 * m + q] = h_modes[8 * m + 3 + q];
        ac.a[4 * m + 3] = -h_sigma[m] * vA / B0;
    }
    const size_t esz = precision == 32 ? sizeof(float) : sizeof(double);
    char *base = static_cast<char *>(scratch);
    void *coef = base;
    void *tab = base + align_up(size_t(n_modes) * 6 * esz);
    char *after = base + alfven_scratch_bytes(nx, ny, nz, n_modes);
    void *acoef = after;
    double *partials = reinterpret_cast<double *>(after + align_up(size_t(n_modes) * 4 * sizeof(double)));
    void *tabx_t = after + align_up(size_t(n_modes) * 4 * sizeof(double)) +
                   align_up(size_t(ny) * nz * n_modes * sizeof(double));
    const int64_t entries = int64_t(n_modes) * (nx + ny + nz);
    const int tb = int((entries + 255) / 256) > 0 ? int((entries + 255) / 256) : 1;
    const dim3 grid(1, ny, nz);
    if (precision == 32) {
        acoef_kernel<float><<<1, 256, 0, s>>>(ac, n_modes, static_cast<float *>(acoef));
        tables_kernel<float><<<tb, 256, 0, s>>>(hm, n_modes, nx, ny, nz, static_cast<float *>(coef),
                                                static_cast<float *>(tab), static_cast<float *>(tabx_t));
        alfven_adjoint_kernel<float><<<grid, 128, 0, s>>>(
            static_cast<const float *>(coef), static_cast<const float *>(acoef), n_modes,
            static_cast<const float *>(tab), static_cast<const float *>(tabx_t), nx, ny, nz, float(B0), float(u_gas[0]), float(u_gas[1]),
            float(u_gas[2]), float(1.0 / c), static_cast<float *>(fbar), static_cast<float *>(fbar_total),
            partials);
    } else {
        acoef_kernel<double><<<1, 256, 0, s>>>(ac, n_modes, static_cast<double *>(acoef));
        tables_kernel<double><<<tb, 256, 0, s>>>(hm, n_modes, nx, ny, nz, static_cast<double *>(coef),
                                                 static_cast<double *>(tab), static_cast<double *>(tabx_t));
        alfven_adjoint_kernel<double><<<grid, 128, 0, s>>>(
            static_cast<const double *>(coef), static_cast<const double *>(acoef), n_modes,
            static_cast<const double *>(tab), static_cast<const double *>(tabx_t), nx, ny, nz, B0, u_gas[0], u_gas[1], u_gas[2], 1.0 / c,
            static_cast<double *>(fbar), static_cast<double *>(fbar_total), partials);
    }
    amp_reduce_kernel<<<n_modes, 256, 0, s>>>(partials, int64_t(ny) * nz, n_modes, amp_bar);
    return cudaGetLastError();
}

} // namespace rsol
