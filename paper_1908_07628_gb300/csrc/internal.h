// Internal launchers shared between the host orchestration (api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct eels_ctx;

namespace eels {

// Tile hook of a context: called between tiles of work with phase 0 (build: `done` of
// `total` slices stepped) or 1 (map: `done` of `total` depths contracted), after the
// tile's work is queued on the call's stream.  A non-zero return abandons the call with
// EELS_ERR_CANCELLED.  The map server installs one on each of its contexts.
typedef int (*TileHook)(void* user, int phase, int done, int total);
void set_tile_hook(eels_ctx* ctx, TileHook fn, void* user);
// Flops of the context's last map contraction as grouped (8 per complex product).
double last_map_flops(const eels_ctx* ctx);

// True if the multislice kernels are compiled for grid side n.
bool grid_supported(int n);

// Number of float2 values in the twiddle table of a length-n transform, and the host
// routine that fills one (exp(-2 pi i k / n) and the second-stage factor tables of the
// two-stage plans, each rounded from FP64).  Every FFT kernel takes such a table.
int twiddle_table_size(int n);
void fill_twiddle_tables(int n, float2* h);

// t[i][y][x] = exp(i sigma v[i][y][x]) with the phase in FP64 (Eqs. 3-4).
cudaError_t launch_transmission(const float* v, double sigma, float2* t, int64_t count,
                                cudaStream_t s);

// Ptab[kx'][ky'] = B(k) exp(-i pi lambda dz |k|^2) * scale on the N/2 x N/2 box
// (box order: index i < N/4 is frequency i, else i - N/2).  Phase argument in FP64.
cudaError_t launch_propagator_table(float2* ptab, int n, double cell, double lam, double dz,
                                    float scale, cudaStream_t s);

// W[b][y][kx'] = amp[b] exp(2 pi i py[b] y / N) at kx' = box(px[b]), zero elsewhere:
// the row-spectrum form of the plane wave amp * exp(2 pi i (px x + py y)/N) / N.
cudaError_t launch_init_plane_waves(float2* W, int n, int n_waves, const int* px, const int* py,
                                    const float2* amp, const float2* tw, cudaStream_t s);

// Row pass of one slice step for n_waves waves (see multislice.cu).
//   store_mode 0: none; 1: store Dec(t psi) (S_in); 2: store Dec(psi) before the
//   transmission (S_out).  Only waves < s_waves are stored, at S + wave*s_stride.
cudaError_t launch_row_pass(int n, int n_waves, const float2* W, float2* Phi, const float2* t_slice,
                            int conj_t, int store_mode, float2* S, int s_waves, int64_t s_stride,
                            int fft_out, const float2* tw, cudaStream_t s);

// Column pass: FFT_y, crop to the band box, multiply by Ptab (or conj), and then
//   mode 0: zero-pad and inverse FFT_y back into W;
//   mode 1: accumulate det_scale * sum |.|^2 over det_mask bins into det_acc[wave_out[w]].
cudaError_t launch_col_pass(int n, int n_waves, const float2* Phi, float2* W, const float2* ptab,
                            int conj_p, int mode, const uint8_t* det_mask, const int* wave_out,
                            double* det_acc, double det_scale, const float2* tw, cudaStream_t s);

// Quadratic baseline: elastic probe waves in row-spectrum form.
//   coef[b][j] = c exp(-2 pi i f (p_j Rx_b + q_j Ry_b)/L) computed in FP64 phase.
cudaError_t launch_probe_init(float2* W, int n, int n_probes, const double* rx, const double* ry,
                              const int* bp, const int* bq, int n_beams, int f, double cell,
                              double c, const float2* tw, cudaStream_t s);

// Quadratic baseline: new inelastic waves in row-pass output form from the
// stored decimated transmitted elastic waves D (Eq. Hn0Psi on the N/2 grid).
struct SpawnList {
  const int* src;     // elastic wave index
  const int* site;    // site index
  const int* type;    // transition type
  int count;
  int first_wave;     // output wave index of the first spawn
};
// H is [S][T][w][w], or [T][w][w] shared by every site when h_mul = 0.
cudaError_t launch_spawn(int n, const SpawnList& sp, const float2* D, const float2* H, int n_types,
                         int h_mul, int w, const int* win_x0, const int* win_y0, float2* Phi,
                         const float2* tw, cudaStream_t s);

// Contraction (CUDA cores, FP32).
struct TransitionBatch {
  const int* site;    // [count] site index of each transition
  const int* type;    // [count]
  int count;
};
struct WindowLists {
  const int* xoff; const int* xcnt; const int* xlist;   // per site: scan columns in the PRISM window
  const int* yoff; const int* ycnt; const int* ylist;   // per site: scan rows
  int max_nr;                                           // max over sites of xcnt*ycnt
};
cudaError_t launch_gemm1_fp32(const float2* Sout, const float2* Sin, int nh, int n_out, int n_in,
                              int w, const float2* H, int n_types, int h_mul,
                              const TransitionBatch& tb, const int* win_x0, const int* win_y0,
                              float2* M, int64_t m_stride, cudaStream_t s);
cudaError_t launch_gemm2_abs2_fp32(const float2* M, int64_t m_stride, int n_out, int n_in,
                                   const float2* ax, const float2* ay, int n_sx, int n_sy,
                                   const TransitionBatch& tb, const WindowLists& wl, double* map,
                                   cudaStream_t s);
// ax[j][ix] = exp(-2 pi i f p_j Rx(ix) / L) (FP64 phase); same for ay with q_j, Ry.  Row
// ix holds position Rx = r0 + (r_first + ix) step (a window of a longer scan line).
// transposed = 1 writes out[pos][j] instead (coalesced reads along the beams).
cudaError_t launch_phase_table(float2* out, const int* bidx, int n_beams, int f, double cell,
                               double r0, double step, int n_pos, cudaStream_t s,
                               int transposed = 0, int r_first = 0);
cudaError_t launch_scale(double* a, int64_t count, double scale, cudaStream_t s);
// a *= scale; bit 2 of *flag is set if any result is NaN or Inf (the map's sentinel)
cudaError_t launch_scale_check(double* a, int64_t count, double scale, int* flag,
                               cudaStream_t s);
// Bounds-checked debug build: each collector moves its translation unit's check flag into
// bit 4 of *status (and clears it); in the normal build they do nothing.
cudaError_t collect_checks_tc(int* status, cudaStream_t s);        // contract_tc.cu
cudaError_t collect_checks_fp32(int* status, cudaStream_t s);      // contract_fp32.cu
cudaError_t collect_checks_ms(int* status, cudaStream_t s);        // multislice.cu
cudaError_t collect_checks_elastic(int* status, cudaStream_t s);   // elastic.cu
// acc[i] += x[i]
cudaError_t launch_accumulate(double* acc, const double* x, int64_t count, cudaStream_t s);

// Elastic images (elastic.cu).  Cut pass: out[r][sx][y'][x'] for scan rows iy0 ..
// iy0 + n_rows - 1 = sum_j ax[j][sx] ay[j][iy] S[j][(wy[iy] + y') % nh][(wx[sx] + x') % nh].
constexpr int kMaxDetectors = 8;
bool cut_supported(int m);
cudaError_t launch_exit_cut(const float2* S, int n_in, int nh, int m, const float2* ax,
                            const float2* ay, int n_sx, int n_sy, const int* wx, const int* wy,
                            int iy0, int n_rows, float2* out, cudaStream_t s);
// map[m][p] /= bf[p] for m < n_types, p < n_pix.
cudaError_t launch_divide(double* map, const double* bf, int n_types, int64_t n_pix,
                          cudaStream_t s);
// 2-D DFT of n_cut cuts of M x M (in place), then img[d][iy0 * n_sx + cut] += sum of
// |X|^2 over the bins with bit d set in mask[ky][kx].
cudaError_t launch_cut_detect(int m, float2* X, int n_cut, const uint8_t* mask, int n_det,
                              int n_sx, int iy0, int64_t img_stride, double* img,
                              const float2* tw, cudaStream_t s);

// Tensor-core (tcgen05) contraction of a batch of sites of one slice: gathers the
// windowed operands, runs GEMM 1 (M = Sout^H diag(H) Sin) and GEMM 2 with the fused
// sum_d |.|^2 epilogue into map.  All pointers are device memory.  Operand buffers
// hold tc_value_bytes(prec) bytes per value: hi + lo planes of TF32 (8) or BF16 (4).
#define EELS_TC_TF32 0
#define EELS_TC_BF16X3 1
int tc_k_align(int prec);   // K padding (elements) of the operand buffers
int tc_value_bytes(int prec);   // bytes per operand value, both planes
int tc_tile_width(int narrow);   // output tile columns of the GEMMs: 128 (narrow) or 256
struct TcBatch {
  int prec;                               // EELS_TC_TF32 or EELS_TC_BF16X3
  const float2* Sout; const float2* Sin;  // depth planes [beam][nh][nh]
  int nh, n_out, n_in, w, n_types;
  const float2* H;                        // [S][T][w][w] or shared [T][w][w]
  int h_mul;                              // 1: per-site H, 0: shared
  const int* wx; const int* wy;           // per site window origin
  const int* slot_site;                   // [n_sites] site of each slot of this batch
  const int* z_site; const int* z_type;   // [n_sites * T] transition z = slot*T + type
  int n_sites, slots_cap;                 // sites in this batch, buffer capacity in sites
  int k1p, k2p;                           // padded K of GEMM 1 (2 w^2) and GEMM 2 (2 n_in)
  void* A1; void* B1; void* M1; void* B2;
  const float2* ax; const float2* ay; int n_sx, n_sy;
  const int* xoff; const int* xcnt; const int* xlist;
  const int* yoff; const int* ycnt; const int* ylist;
  int nr_cap;                             // max scan positions of a site
  const int* a_batch1; const int* b_batch1; const int* n_valid1;
  const int* a_batch2; const int* b_batch2; const int* n_valid2;
  double* map;
  int* status;                            // set to 1 if a bounded wait timed out
  long long wait_cycles;                  // limit of the pipeline waits, clock cycles (0: default)
  int withhold;                           // 1: TMA producers issue no load (failure test)
  // association with the probe sum first (GEMM-Y then per-channel GEMM-V)
  void* AY; void* BY; void* BV;           // a rows, S_in window transposed, H_t . Y rows
  const int* a_batch_y; const int* n_valid_y;   // identity map and k1p per site
  const int* m_valid_y;                         // scan positions of the site of each slot
  const float2* axT; const float2* ayT;         // phase tables [pos][n_in] (transposed)
  // prefix sums of the tiles with work per problem (the persistent TF32 GEMMs walk only
  // those): tiles_v over the transitions for GEMM 2 / GEMM-V (column tiles of 2 n_R rows x
  // all row tiles of n_out), tiles_y over the sites for GEMM-Y (row tiles of n_R x all
  // column tiles); n_tiles_* = the batch's total
  const int* tiles_v; int n_tiles_v;
  const int* tiles_y; int n_tiles_y;
  // output tile width (columns, tc_tile_width) of the grouping's first GEMM (GEMM 1 /
  // GEMM-Y) and second GEMM (GEMM 2 / GEMM-V); tiles_y and tiles_v list tiles of these widths
  int bn_first, bn_second;
};
cudaError_t tc_gather(const TcBatch& b, cudaStream_t s);   // A1, B1, B2 operand buffers
cudaError_t tc_gemm1(const TcBatch& b, cudaStream_t s);    // M1 = GEMM 1
cudaError_t tc_gemm2(const TcBatch& b, cudaStream_t s);    // map += sum_d |GEMM 2|^2
cudaError_t tc_gather_y(const TcBatch& b, cudaStream_t s); // A1, AY, BY
cudaError_t tc_gemm_y(const TcBatch& b, cudaStream_t s);   // BV = H_t . (a rows x Sin window)
cudaError_t tc_gemm_v(const TcBatch& b, cudaStream_t s);   // map += sum_d |A1 x BV|^2

}  // namespace eels
