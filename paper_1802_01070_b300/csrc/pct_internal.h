// pct_internal.h -- private interface between the C ABI (pct_api.cu) and the
// kernel launchers (pct_kernels.cu).  Not installed, not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pct_bins.cuh"
#include "pct_device.cuh"

namespace pct {

// Device pointers of one loaded history set (12 SoA columns, stride floats apart):
// in_x, in_y, in_z, out_x, out_y, out_z, theta_in, psi_in, theta_out, psi_out, phi, wepl.
enum HistField { H_INX = 0, H_INY, H_INZ, H_OUTX, H_OUTY, H_OUTZ, H_THI, H_PSI, H_THO, H_PSO, H_PHI,
                 H_WEPL, H_NF };

struct Launch {
    cudaStream_t stream;
    int cta;              // threads per block for per-proton kernels
    int64_t* launches;    // launch counter to bump
};

// How the DROP block step and the row writer walk a proton's path: lane ranges
// (pct_warp.cuh) or rounds of one segment per lane (pct_round.cuh).
constexpr int kWalkLanes = 0;
constexpr int kWalkRounds = 1;

struct Geo {
    GridC g;
    MlpC mc;
    const uint8_t* mask;  // device, nx*ny*nz bytes
    const uint8_t* dist;  // device, nx*ny*nz bytes: chessboard distance to the hull (or null)
    unsigned* flags;      // device error word
    int walk = kWalkLanes;
    unsigned long long* fallbacks = nullptr;   // device: protons the round walk passed to the lane walk
};

// 1/(beta^2 p^2) of a 200 MeV proton in water as a polynomial in depth (cm),
// MeV^-2: the energy-loss fit used with the most-likely-path formalism (host).
extern const double kCoef200[6];
// MLP table tab[k] = Sigma(0, k du) (S00, S01, S11, 2 S01) in cm / rad for
// k = 0..kmax (tab[0] = 0), evaluated in FP64 on the host.
void mlp_sigma_table(double du_mm, int kmax, float4* tab);

// dist = chessboard distance of each voxel to the nearest hull voxel (capped at
// 255); tmp is scratch of the same size.
cudaError_t launch_hull_dist(const Launch& L, const uint8_t* mask, int nx, int ny, int nz, uint8_t* tmp,
                             uint8_t* dist);
cudaError_t launch_prepare(const Launch& L, const Geo& G, const float* hist, int64_t stride,
                           int64_t n, float* rec);
// out[i] = the record kernel's tangent of the angle t[i] (diagnostic)
cudaError_t launch_tan_angle(const Launch& L, const double* t, double* out, int64_t n);
// records of protons [first, first + count) only
cudaError_t launch_prepare_range(const Launch& L, const Geo& G, const float* hist, int64_t stride,
                                 int64_t first, int64_t count, float* rec);
cudaError_t launch_hull_states(const Launch& L, const float* rec, int64_t stride, int64_t first,
                               int64_t count, float* out);
cudaError_t launch_mlp_points(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              int64_t first, int64_t count, int32_t max_pts, float* out_xyz,
                              int32_t* out_npts);
cudaError_t launch_rows(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                        int64_t first, int64_t count, int32_t max_nnz, int32_t* out_idx,
                        float* out_len, int32_t* out_nnz);
// y = A x and g += A^T y (g cleared by the caller); `next` is a device work
// counter, cleared by the launcher.
cudaError_t launch_forward(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                           int64_t n, const float* x, float* y, unsigned long long* next);
cudaError_t launch_adjoint(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                           int64_t n, const float* y, float* g_out, unsigned long long* next);
// Lists of the protons whose path crosses the hull, per DROP block of size B:
// block k's protons are vidx[boff[k] .. boff[k+1]) (proton order).  chunk is
// scratch of compact_chunks(n) values; vidx holds n values, boff
// ceil(n / B) + 1.
constexpr int64_t kCompactChunk = 8192;   // protons per compaction chunk
int64_t compact_chunks(int64_t n);
cudaError_t launch_compact(const Launch& L, const float* rec, int64_t stride, int64_t n, int64_t B,
                           int64_t* chunk, int64_t* vidx, int64_t* boff);
// DROP block step of block k (at most `count` protons) over its valid list;
// `next` is a device work counter that must be zero at launch (the block
// apply that follows resets it).
cudaError_t launch_drop_fused(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              const int64_t* vidx, const int64_t* boff, int64_t k, int64_t count,
                              const float* x, float2* acc, unsigned long long* next);
// Block apply over the hull voxels (mask != 0); resets the work counter
// `next` when not null.
cudaError_t launch_drop_apply(const Launch& L, int64_t n_vox, const uint8_t* mask, float* x, float2* acc,
                              float lambda, unsigned long long* next);

// data cleaning (pct_clean.cu): bins of (gantry angle, t, v) and the cut
struct CleanBins {
    ProtonBins bins;
    double k_sigma;
};
// keep[i] = 1 for the protons within k_sigma of their bin's mean in WEPL and
// both angle changes; bin (n), cnt (nbins), sum and dev2 (3 nbins) are scratch
cudaError_t launch_clean(const Launch& L, const CleanBins& P, const float* hist, int64_t stride, int64_t n,
                         int* bin, unsigned* cnt, double* sum, double* dev2, uint8_t* keep);
// kept protons' 12 columns written in order to out (column stride out_stride);
// *total (device) = their number; chunk holds clean_chunks(n) values
int64_t clean_chunks(int64_t n);
cudaError_t launch_keep_compact(const Launch& L, const uint8_t* keep, int64_t n, int64_t* chunk,
                                int64_t* total, const float* hist, int64_t stride, float* out,
                                int64_t out_stride);
// the same compaction of any ncols float columns; column shift_col (>= 0) gets
// `shift` added.  In two parts: count (chunk offsets and *total), then fill.
cudaError_t launch_flag_count(const Launch& L, const uint8_t* flag, int64_t n, int64_t* chunk, int64_t* total);
cudaError_t launch_flag_fill(const Launch& L, const uint8_t* flag, int64_t n, const int64_t* chunk,
                             const float* src, int64_t stride, int ncols, int shift_col, float shift, float* out,
                             int64_t out_stride);
cudaError_t launch_flag_compact(const Launch& L, const uint8_t* flag, int64_t n, int64_t* chunk,
                                int64_t* total, const float* src, int64_t stride, int ncols, int shift_col,
                                float shift, float* out, int64_t out_stride);

// image regions of Algorithm 1 (pct_regions.cu): flag[i] = proton i has a
// hull path whose entry or exit slice lies in [lo, hi)
cudaError_t launch_region_flags(const Launch& L, const float* rec, int64_t stride, int64_t n, const GridC& g,
                                int lo, int hi, uint8_t* flag);

// filtered back-projection (pct_fbp.cu): x = the FBP image inside the hull, 0
// outside; cnt, sum (nbins) scratch, q (nbins) the filtered sinogram
int fbp_max_angles();
cudaError_t launch_fbp(const Launch& L, const ProtonBins& P, const GridC& g, const uint8_t* hull,
                       const float* hist, int64_t stride, int64_t n, unsigned* cnt, double* sum, float* q,
                       float* x);

// gradient-based reconstruction (pct_grad.cu)
cudaError_t launch_tv(const Launch& L, const float* x, int nx, int ny, int nz, float eps, float* grad,
                      double* value);
cudaError_t launch_adam(const Launch& L, float* x, const float* g, float* m, float* v, int64_t n,
                        float lr, float b1, float b2, float eps, int step);

// stored rows (pct_rows.cu)
int64_t scan_chunks(int64_t m);
cudaError_t launch_csr_count(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                             int64_t m, int32_t* cnt);
cudaError_t launch_csr_fill(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                            int64_t m, const int64_t* rowptr, int32_t* idx, float* len);
cudaError_t launch_pack_count(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              int64_t m, int32_t* cnt, short4* start);
// chord_unit > 0: 16-bit fixed-point chords in units of chord_unit mm; 0: FP16
cudaError_t launch_pack_fill(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                             int64_t m, const int64_t* rowptr, uint8_t* codes, uint16_t* lens,
                             float chord_unit);
cudaError_t launch_row_scan(const Launch& L, const int32_t* cnt, int64_t m, int64_t* rowptr,
                            int64_t* chunk_sum);
cudaError_t launch_drop_csr(const Launch& L, unsigned* flags, const int64_t* rowptr, const int32_t* idx,
                            const float* len, const float* b, int64_t first, int64_t count,
                            const float* x, float2* acc);
cudaError_t launch_drop_packed(const Launch& L, const GridC& g, unsigned* flags, const int64_t* rowptr,
                               const short4* start, const uint8_t* codes, const uint16_t* lens,
                               float chord_unit, const float* b, int64_t first, int64_t count,
                               const float* x, float2* acc);

}  // namespace pct
