// Internal launch descriptors shared by the C-ABI layer (rsol_api.cu) and the
// per-precision kernel translation units.  Precision-independent: pointers
// are untyped, scalars are double (rounded once to the kernel's type).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsol {

struct PushDesc {
    int64_t n;
    uint32_t *cell;
    void *off[3];
    void *u[3];
    const void *w;
    const void *fields;
    void *fb;               // may be null: no deposit
    long long *fx;          // fixed-point accumulators (deterministic mode) or null
    int nx, ny, nz, shape, det;
    double h, adv, qv, c, fx_scale;
    int *status;
    int sm_count;
    // binned path (null bin_start: order-free kernel)
    const uint32_t *bin_start;  // nbins + 1 packet offsets of the last sort
    int bin, nbx, nby, nbz;
    int warps;              // binned kernel CTA width: 8, or 0 / 16 for the widest that fits
    int tile_mode;          // 0 = order-free kernel; 1 = binned shared-memory kernel
    uint32_t *perm;         // binned kernel scratch (n entries): local visiting order, or null
};

struct MomentsDesc {
    int64_t n;
    const uint32_t *cell;
    const void *off[3];
    const void *u[3];
    const void *w;
    void *grid;             // [node][8] state moments (accumulated)
    long long *fx;
    int nx, ny, nz, shape, det;
    double inv_vol, mc, mc2, qc, q, fx_scale;
    int sm_count;
    // the binned kernel (set when the packets are the last sort's output)
    const uint32_t *bin_start;
    int bin, nbx, nby, nbz;
};

struct TotalsDesc {
    int64_t n;
    const void *u[3];
    const void *w;
    const void *fb;         // may be null
    int64_t n_nodes;
    double mc, mc2, qc, vol;
    double *partials;       // scratch: blocks * 16 doubles
    double *out;            // device: 16 doubles
    int blocks;
};

struct LossDesc {
    int64_t n;
    const uint32_t *cell;
    const void *off[3];
    const void *u[3];
    void *w;
    const void *nn;         // node grid of n_n (one value per node) or null
    double nn_uniform, coef;  // coef = (c~/c) sigma c dt
    int nx, ny, nz, shape;
    int *status;
    int sm_count;
    // gathered n_n on the last sort's output: per-bin n_n tiles (else null)
    const uint32_t *bin_start;
    int bin, nbx, nby, nbz;
};

cudaError_t losses_f32(const LossDesc &d, cudaStream_t s);
cudaError_t losses_f64(const LossDesc &d, cudaStream_t s);
cudaError_t push_f32(const PushDesc &d, cudaStream_t s);
// Batched push over the bins of many boxes (boxes: device array of BatchBox<T>;
// work: device scratch of batch_work_words(total_bins) words, overwritten).
cudaError_t push_batch_f32(const PushDesc &d, const void *boxes, int n_boxes, uint32_t total_bins,
                           int warps, uint32_t *work, cudaStream_t s);
cudaError_t push_batch_f64(const PushDesc &d, const void *boxes, int n_boxes, uint32_t total_bins,
                           int warps, uint32_t *work, cudaStream_t s);
inline size_t batch_work_words(uint32_t total_bins) { return 3 + size_t(total_bins); }
size_t batch_box_size(int precision);
void fill_batch_box_f32(void *dst, int nx, int ny, int nz, int nbx, int nby, int nbz,
                        int64_t node_off, uint32_t bin_base, double h, double adv, double qv, double c);
void fill_batch_box_f64(void *dst, int nx, int ny, int nz, int nbx, int nby, int nbz,
                        int64_t node_off, uint32_t bin_base, double h, double adv, double qv, double c);
cudaError_t push_f64(const PushDesc &d, cudaStream_t s);
cudaError_t fixed_to_grid_f32(long long *fx, void *grid, int64_t count, double inv_scale,
                              int sm_count, cudaStream_t s);
cudaError_t fixed_to_grid_f64(long long *fx, void *grid, int64_t count, double inv_scale,
                              int sm_count, cudaStream_t s);
cudaError_t moments_grid_f32(const MomentsDesc &d, cudaStream_t s);
cudaError_t moments_grid_f64(const MomentsDesc &d, cudaStream_t s);
cudaError_t totals_f32(const TotalsDesc &d, cudaStream_t s);
cudaError_t totals_f64(const TotalsDesc &d, cudaStream_t s);

// Sort (sort.cu): stable LSD radix sort of 32-bit keys with a 32-bit index
// payload, then a gather of the packet arrays.
struct SortScratch {
    uint32_t *keys[2];
    uint32_t *idx[2];
    uint32_t *counts;       // 256 * max_blocks
    uint32_t *block_sums;   // scan partials
    uint32_t *bin_start;    // nbins + 1
    int64_t capacity;       // packets
    int64_t max_blocks;
};
size_t sort_scratch_bytes(int64_t n, int64_t nbins);
// Box-major keys of a batch: packet j of box b (packet offsets off[b] .. off[b+1])
// gets ((bin_base[b] + its bin in box b) << 3 lb) | (its anchor within the bin).
struct BatchKeyBox {
    int nx, ny, nz, nbx, nby;
    uint32_t bin_base;
};
cudaError_t sort_particles_batch(const SortScratch &s, int64_t n, int elem_bytes,
                                 const uint32_t *cell_in, void *const off_in[3],
                                 void *const u_in[3], const void *w_in, uint32_t *cell_out,
                                 void *const off_out[3], void *const u_out[3], void *w_out,
                                 const int64_t *d_offsets, const BatchKeyBox *d_boxes,
                                 int n_boxes, int bin, int shape, int key_bits, int64_t nbins,
                                 cudaStream_t st);
void sort_scratch_carve(void *base, int64_t n, int64_t nbins, SortScratch *s);
// Radix passes over the keys in s.keys[0] (key_bits bits, starting from the
// identity order), payload gather and bin ranges (bin = key >> 3 lb, nbins
// bins) into s.bin_start.
cudaError_t sort_from_keys(const SortScratch &s, int64_t n, int elem_bytes,
                           const uint32_t *cell_in, void *const off_in[3], void *const u_in[3],
                           const void *w_in, uint32_t *cell_out, void *const off_out[3],
                           void *const u_out[3], void *w_out, int lb, int key_bits,
                           int64_t nbins, cudaStream_t st);
cudaError_t sort_particles(const SortScratch &s, int64_t n, int elem_bytes,
                           const uint32_t *cell_in, void *const off_in[3], void *const u_in[3],
                           const void *w_in, uint32_t *cell_out, void *const off_out[3],
                           void *const u_out[3], void *w_out, int nx, int ny, int nz, int bin,
                           int shape, int key_bits, int64_t nbins, cudaStream_t st);

// Counting sort by key (same permutation as sort_particles): counters for
// nkeys + 1 buckets and their chunk sums.  It leaves its permutation in
// s.idx[((key_bits + 7) / 8) & 1], where the radix sort leaves it, and the bin
// ranges in s.bin_start; the input keys go to s.keys of the other parity and
// the other index buffer is scratch.  The sorted keys are not formed.
struct CountScratch {
    uint32_t *cursor;      // nbuckets counters
    uint32_t *sums;        // per scan chunk
    int64_t nbuckets;      // nkeys + 1
    int64_t capacity;      // packets
};
// True where the counting sort is used: 2 <= nkeys <= 2^26 and nkeys <= 2 n.
// With d_boxes (a batch), keys are box-major as in sort_particles_batch, nbins
// the batch's total bins; nx, ny, nz are then unused.
bool count_sort_applies(int64_t n, int64_t nkeys);
size_t count_scratch_bytes(int64_t n, int64_t nkeys);
int count_sort_launches(int64_t nkeys);  // kernels one counting sort launches
void count_scratch_carve(void *base, int64_t n, int64_t nkeys, CountScratch *c);
cudaError_t count_sort_particles(const SortScratch &s, const CountScratch &c, int64_t n,
                                 int elem_bytes, const uint32_t *cell_in, void *const off_in[3],
                                 void *const u_in[3], const void *w_in, uint32_t *cell_out,
                                 void *const off_out[3], void *const u_out[3], void *w_out, int nx,
                                 int ny, int nz, int bin, int shape, int key_bits, int64_t nbins,
                                 cudaStream_t st,
                                 const int64_t *d_offsets = nullptr,
                                 const BatchKeyBox *d_boxes = nullptr, int n_boxes = 0);

// Per-packet adaptive timestep with sub-cycling (subcycle.cuh).
struct SubDesc {
    double courant, k_gyro, k_cross, k_loss, dt;
    int max_level;
    uint8_t *level;         // [n] per-packet level (output)
    uint32_t *counts;       // [17] scratch
    uint32_t *order;        // [n] scratch: level-major packet order
};
cudaError_t push_subcycled_f32(const PushDesc &d, const SubDesc &sd, cudaStream_t s);
cudaError_t push_subcycled_f64(const PushDesc &d, const SubDesc &sd, cudaStream_t s);
// Level-major anchor keys (rank max_level - k, then the rsol_sort key) for the
// sorted sub-cycled step (the radix passes start from the identity order).
cudaError_t level_keys_f32(const PushDesc &d, const SubDesc &sd, int lb, int nbx, int nby,
                          uint32_t nbins, uint32_t *keys, cudaStream_t s);
cudaError_t level_keys_f64(const PushDesc &d, const SubDesc &sd, int lb, int nbx, int nby,
                          uint32_t nbins, uint32_t *keys, cudaStream_t s);

// Reverse-mode step of the differentiable run (adjoint.cu).
struct AdjDesc {
    int64_t n;
    const uint32_t *cell;
    const void *off[3];
    const void *u[3];
    const void *w;
    const void *fields;     // [node][8] E, B at the step
    const void *fb;         // [node][8] accumulated feedback (S in 4..6)
    const double *loss;     // device: L, 1/L
    void *xb[3];            // position adjoint (in/out)
    void *ub[3];            // momentum adjoint (in/out)
    void *fbar;             // [node][8] field adjoint (accumulated)
    int nx, ny, nz, shape;
    double h, adv, qv, c;
    int *status;
    int sm_count;
    // tiled kernel: bin ranges of the last sort of this packet order, or null
    const uint32_t *bin_start;
    int bin, nbx, nby, nbz;
};
cudaError_t adjoint_step_f32(const AdjDesc &d, cudaStream_t s);
cudaError_t adjoint_step_f64(const AdjDesc &d, cudaStream_t s);
cudaError_t loss_norm(const void *fb, int64_t n_nodes, int precision, double *partials, int blocks,
                      double *loss, cudaStream_t s);
// Adjoints back to the order before a sort: out[perm[t]] = in[t] (es: element bytes).
cudaError_t unpermute6(int64_t n, int es, const uint32_t *perm, void *const xb_in[3],
                       void *const ub_in[3], void *const xb_out[3], void *const ub_out[3],
                       int sm_count, cudaStream_t s);

// Field source (fields.cu)
cudaError_t alfven_fields(const double *h_modes, const double *h_sigma, int n_modes, double t,
                          double B0, double vA, const double *u_gas, double c, double dx,
                          int nx, int ny, int nz, int precision, void *fields, void *scratch,
                          cudaStream_t s);
size_t alfven_scratch_bytes(int nx, int ny, int nz, int n_modes);
// Adjoint of the field source with respect to the mode amplitudes.
size_t alfven_adjoint_scratch_bytes(int nx, int ny, int nz, int n_modes);
cudaError_t alfven_adjoint(const double *h_modes, const double *h_sigma, int n_modes, double t,
                           double B0, double vA, const double *u_gas, double c, double dx, int nx,
                           int ny, int nz, int precision, void *fbar, void *fbar_total,
                           double *amp_bar, void *scratch, cudaStream_t s);

} // namespace rsol
