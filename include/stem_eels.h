/*
 * stem_eels.h -- C ABI of the GB300 STEM-EELS library (libstemeels.so).
 *
 * Linear-scaling (PRISM) STEM-EELS maps after Brown, Ciston & Ophus,
 * arXiv 1908.07628.  The library builds the probe-side scattering matrix S_in
 * (Sec. III: "S_1 ... propagate the plane wave components that fall within the
 * probe forming aperture"), carries the detector plane waves backwards to make
 * S_out (Eq. MSTop, used as its complex conjugate), contracts
 * M_n = S_out^H diag(H_n) S_in per transition (Eqs. Hn0op, SHn0) and
 * accumulates f^2 sum_d |M_n a(R)|^2 into an FP64 map (second algorithm
 * listing of Sec. III).  It also runs the conventional quadratic algorithm
 * (first listing of Sec. III) on the GPU as the same-hardware baseline.
 *
 * Conventions shared by every call
 * - Square cell L x L (Angstrom) sampled on an N x N grid, N = 2^a 3^b with
 *   N in {64, 128, 256, 384, 512, 768, 1024}.  Real-space arrays are row-major
 *   [y][x]; pixel (ix, iy) sits at (ix L/N, iy L/N).
 * - Forward transform exp(-2 pi i r.g) (footnote to Eq. 4); the propagator is
 *   band-limited to p^2 + q^2 < (N/4)^2 (Sec. III, "bandwidth limited ... to 1/2").
 * - Probe beams: k = f(p, q)/L with lambda |k| <= alpha; detector beams the same
 *   with beta.  Transition windows live on the N/2 grid.
 * - Complex data are interleaved float pairs (re, im) -- "complex64".
 * - Every pointer argument is borrowed for the duration of the call only.  A
 *   flag next to each array says whether it is host or device memory; device
 *   pointers must belong to the context's device.  Handles are owned by the
 *   library and released by the matching _free / _destroy call.
 * - Work is issued on the CUDA stream passed as `stream` (a cudaStream_t, NULL
 *   for the legacy default stream).  Calls that return results to host memory
 *   synchronise that stream before returning; calls that write device memory
 *   return once the work is queued.
 * - Errors: every call returns an eels_status; no call aborts or throws.  The
 *   text of the last error of a context is available from eels_last_error().
 */
#ifndef STEM_EELS_H
#define STEM_EELS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EELS_OK = 0,
  EELS_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, beam outside band limit) */
  EELS_ERR_UNSUPPORTED = 2,  /* grid size or option not built into this library */
  EELS_ERR_OOM = 3,          /* device allocation failed */
  EELS_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
  EELS_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  EELS_ERR_CANCELLED = 6,    /* a map server request was cancelled or passed its deadline */
  EELS_ERR_NONFINITE = 7,    /* the computed map holds NaN or Inf (non-finite inputs or an
                                overflow); the map is still written */
  EELS_ERR_BOUNDS = 8        /* bounds-checked debug build only (compiled with -DSTEM_CHECK):
                                a kernel found an index it derives from a device list (window
                                origin, beam or scan index, tile decode, TMA box coordinate)
                                out of range and skipped that access; the result is invalid */
} eels_status;

/* Arithmetic of the inelastic contraction (Eq. SHn0 and the |.|^2 scan sum).
 * The multislice always runs in FP32 with FP64 propagator phases; the map is
 * always accumulated in FP64. */
typedef enum {
  EELS_PREC_FP32 = 0,        /* FP32 CUDA-core complex GEMMs */
  EELS_PREC_TF32 = 1,        /* tcgen05 TF32 hi+lo split (3 products), FP32 accumulate: about
                                21 significant bits per operand, the FP32-class tensor path */
  EELS_PREC_BF16X3 = 2       /* tcgen05 BF16 hi+lo split (3 products), FP32 accumulate: about
                                16 significant bits per operand, the reduced-precision path */
} eels_precision;

typedef struct eels_ctx eels_ctx;
typedef struct eels_smatrix eels_smatrix;

/* Specimen: the projected potential of each slice (Eq. 3-4, v_i(r) in V*A). */
typedef struct {
  int n;                  /* grid side N */
  int n_z;                /* number of slices */
  double cell;            /* L, Angstrom */
  const float* vproj;     /* [n_z][n][n] V*A */
  int vproj_on_device;    /* 1: device pointer, 0: host pointer */
} eels_specimen;

/* Electron optics of the probe and the PRISM interpolation (Sec. II-III). */
typedef struct {
  double lambda;          /* relativistic wavelength, Angstrom */
  double sigma;           /* interaction constant, rad / (V A) */
  double dz;              /* slice thickness, Angstrom */
  int f;                  /* PRISM interpolation factor, >= 1 */
  double alpha;           /* probe convergence semi-angle, rad */
} eels_optics;

/* Ionising sites and their transition potentials H_n0 (Eq. Hn0def), sampled on
 * a w x w window of the N/2 grid whose origin (win_x0, win_y0) is periodic.
 * (x, y) is the site position used for the PRISM window rule: a site counts
 * for probe R iff the minimum-image r_s - R lies in [-L/2f, L/2f) on both axes. */
typedef struct {
  int n_sites;
  int n_types;            /* channels per site (e.g. m = -1, 0, 1) */
  int w;                  /* window side on the N/2 grid, 1 <= w <= N/2 */
  const float* H;         /* complex64 [n_sites][n_types][w][w] */
  const int32_t* slice;   /* [n_sites] slice index of each site */
  const int32_t* win_x0;  /* [n_sites] window origin column on the N/2 grid */
  const int32_t* win_y0;  /* [n_sites] window origin row */
  const double* x;        /* [n_sites] Angstrom */
  const double* y;        /* [n_sites] Angstrom */
  int on_device;          /* 1: H is a device pointer (the small per-site arrays are always host) */
  int h_shared;           /* 1: H is [n_types][w][w], the same transition potentials at every
                             site (windows still placed per site); 0: per-site H as above */
} eels_transitions;

/* Scan raster: R(ix, iy) = (x0 + ix*step_x, y0 + iy*step_y), Angstrom. */
typedef struct {
  int n_sx, n_sy;
  double x0, y0, step_x, step_y;
} eels_scan;

/* Create a context on CUDA device `device`.  Owns twiddle tables, options, the grouping
 * choices of the autotuner and the profiling records.  A context serves one host thread
 * at a time; threads that compute concurrently each use their own context (as the map
 * server's workers do).  Different contexts may run concurrently on one device. */
eels_status eels_create(int device, eels_ctx** out);
void eels_destroy(eels_ctx* ctx);
/* Text of the last error raised on this context ("" if none).  Owned by ctx. */
const char* eels_last_error(const eels_ctx* ctx);

/* Build S_in (Sec. III second listing, "Advance S_1 one slice"): the plane
 * waves of the probe aperture on the f-lattice carried through slices
 * 0..n_z-1; S_in(i) = Dec(t_i psi_j(i)) is stored for every depth on the N/2
 * grid as complex64 [n_z][n_in][N/2][N/2] (beam-major planes), scaled by N.
 * Also keeps the transmission functions t_i for inelastic_map.  The returned
 * handle owns all of it; free it with eels_smatrix_free.  Returns
 * EELS_ERR_ARG if a probe beam lies outside the band limit, EELS_ERR_OOM if the
 * device cannot hold n_z * n_in * (N/2)^2 * 8 bytes plus the transmissions. */
eels_status eels_build_smatrix(eels_ctx* ctx, const eels_specimen* spec, const eels_optics* optics,
                               void* stream, eels_smatrix** out);
/* Releases the handle in stream order on the stream it was built on, which must
 * still exist; the call waits for that stream's queued work first.  The context the
 * handle was built on may already be destroyed (language bindings whose garbage
 * collector finalises objects in any order rely on this). */
void eels_smatrix_free(eels_smatrix* sm);

/* Shape of a built S-matrix: grid, slices and number of probe beams. */
eels_status eels_smatrix_info(const eels_smatrix* sm, int* n, int* n_z, int* n_in);

/* Copy the probe beam list (integer f-lattice indices p, q; k = f(p,q)/L) to host
 * arrays of length n_in, in the column order of S_in. */
eels_status eels_smatrix_beams(const eels_smatrix* sm, int32_t* p, int32_t* q);

/* Copy S_in(depth) (complex64 [n_in][N/2][N/2], values scaled by N so that a
 * unit-norm plane wave has unit-modulus samples) to device memory `dst`. */
eels_status eels_smatrix_copy_depth(const eels_smatrix* sm, int depth, float* dst, void* stream);

/* EELS map of the linear algorithm (Sec. III second listing, realised exactly
 * with S_out streamed backwards one depth at a time):
 *   map[m][iy][ix] = f^2 sum_{sites s in window(R)} sum_d |sum_j M_{s,m}[d,j] a_j(R)|^2
 * map_out is FP64 [n_types][n_sy][n_sx], caller-owned, host or device
 * (map_on_device); it is overwritten.  beta is the EELS collection semi-angle.
 * The call waits for its work to finish before it returns (it reads a device status
 * word): EELS_ERR_TIMEOUT if a bounded tensor-core wait gave up, EELS_ERR_NONFINITE if a
 * map value is NaN or Inf, EELS_ERR_BOUNDS (bounds-checked build only) if a kernel's
 * index check failed.  EELS_ERR_UNSUPPORTED if the precision is not built. */
eels_status eels_inelastic_map(eels_ctx* ctx, const eels_smatrix* sm, const eels_transitions* tr,
                               const eels_scan* scan, double beta, int precision,
                               double* map_out, int map_on_device, void* stream);

/* The same map computed per scan tile, resumable (not in the paper: a map of a long scan
 * can be stopped and picked up again without redoing finished positions).  The scan is
 * cut into tiles of tile_nx x tile_ny positions (edge tiles smaller), tile k = ty * gx + tx
 * with gx = ceil(n_sx / tile_nx), gy = ceil(n_sy / tile_ny); tile_done is caller-owned
 * host memory of gx * gy bytes.  Tiles with tile_done[k] != 0 are skipped; every other
 * tile is mapped, as eels_inelastic_map does over that rectangle of the scan (the stored
 * S_in of sm is reused, the detector beams are carried backwards again per tile), its
 * values are written into map_out (host, FP64 [n_types][n_sy][n_sx]) and tile_done[k] is
 * set to 1.  Positions outside finished tiles are not touched.  At most max_tiles tiles
 * are mapped per call (<= 0: no limit); *remaining (may be null) receives the number of
 * tiles left.  On an error the tiles finished before it stay written and marked, so a
 * later call with the same map_out and tile_done resumes there; the error codes are
 * those of eels_inelastic_map, plus EELS_ERR_ARG for a null tile_done or a tile size
 * below 1.  A position's value does not depend on the tiling beyond FP64 summation
 * order when the grouping and tile width are fixed (EELS_OPT_ASSOCIATION,
 * EELS_OPT_TILE_WIDTH); the autotuner may choose differently for differently shaped
 * tiles (differences at the precision's rounding level). */
eels_status eels_inelastic_map_tiles(eels_ctx* ctx, const eels_smatrix* sm,
                                     const eels_transitions* tr, const eels_scan* scan,
                                     double beta, int precision, int tile_nx, int tile_ny,
                                     double* map_out, uint8_t* tile_done, int max_tiles,
                                     int* remaining, void* stream);

/* Elastic STEM images from the same S-matrix (Sec. IV D: the annular dark-field image
 * with a 60 mrad inner angle and the incoherent bright-field image whose detector has
 * the extent of the EELS aperture, by which the EELS map is divided).
 *
 * Needs a handle built while EELS_OPT_EXIT_PLANE was 1 (S_in at the exit surface);
 * otherwise EELS_ERR_ARG.  For probe R the exit wave sum_j c a_j(R) S_exit[j] (Sec. III)
 * is cut to the L/f cell around R on the N/2 grid: the M = N/(2f) pixels per axis whose
 * minimum-image offset from R lies in [-L/2f, L/2f) (the rule of the site windows),
 * starting at the in-rule pixel whose cyclic predecessor is out of rule (pixel 0 at f = 1).
 * Detector d integrates over the cut's DFT lattice k = f(a, b)/L:
 *   out[d][iy][ix] = (16 f^2 / N^2) sum_{k in D_d} |sum_{p in cut} psi(x_p) e^{-2 pi i k.x_p}|^2
 * with D_d = {k : inner_d <= lambda |k| (<= outer_d if outer_d > 0), 16 f^2 (a^2 + b^2) < N^2}.
 * For a wave that lies inside the cut this is the EELS detector's f^2 sum over f-lattice
 * beams.  1 <= n_det <= 8.  out is FP64 [n_det][n_sy][n_sx], caller-owned, host or device
 * (out_on_device), overwritten.  EELS_ERR_UNSUPPORTED if N/2 is not divisible by f or
 * M is not one of 16, 32, 48, 64, 96, 128, 192, 256, 384, 512. */
typedef struct {
  double inner;   /* semi-angle (rad), lambda |k| >= inner */
  double outer;   /* semi-angle (rad), lambda |k| <= outer; <= 0: up to the band limit */
} eels_detector;
eels_status eels_elastic_images(eels_ctx* ctx, const eels_smatrix* sm, const eels_scan* scan,
                                const eels_detector* detectors, int n_det, double* out,
                                int out_on_device, void* stream);

/* Frozen-phonon average of the EELS map: the mean over n_configs passes, each a full
 * build + map of one configuration of thermally displaced atoms (specs[c], trs[c]; the
 * displacements are the caller's), with the same optics, scan, beta and precision
 * (Sec. IV A / IV D speak of frozen phonon passes).  Configurations must share the grid
 * and the channel count (EELS_ERR_ARG otherwise); each may have its own sites.  The FP64
 * sum runs on the device in configuration order, then is divided by n_configs.  Options
 * of the context (grouping, S_out scheme, shards) apply to every pass.  map_out as for
 * eels_inelastic_map. */
eels_status eels_phonon_map(eels_ctx* ctx, const eels_specimen* specs,
                            const eels_transitions* trs, int n_configs,
                            const eels_optics* optics, const eels_scan* scan, double beta,
                            int precision, double* map_out, int map_on_device, void* stream);

/* The bright-field correction of Sec. IV D: map[m][p] /= bf[p] in place for every
 * channel m < n_types and pixel p < n_pix (FP64; both host or both device per
 * on_device; a zero bright-field pixel gives inf or nan there, as IEEE division does). */
eels_status eels_divide_map(eels_ctx* ctx, double* map, const double* bf, int n_types,
                            int64_t n_pix, int on_device, void* stream);

/* The conventional quadratic algorithm (Sec. III first listing) on the GPU,
 * batched over probes and inelastic waves, same FFT kernels.  If positions is
 * non-NULL only the n_pos scan points positions[2k] = iy, positions[2k+1] = ix
 * (host int32) are computed and the rest of the map is zero.  Returns in
 * *steps (if non-NULL) the number of multislice operations performed, which
 * equals the paper's count sum_i n_states,i (n_z - i) + n_z per probe. */
eels_status eels_quadratic_reference_map(eels_ctx* ctx, const eels_specimen* spec,
                                         const eels_optics* optics, const eels_transitions* tr,
                                         const eels_scan* scan, double beta,
                                         const int32_t* positions, int n_pos, double* map_out,
                                         int map_on_device, void* stream, int64_t* steps);

/* Context options.
 * EELS_OPT_ASSOCIATION selects how the tensor-core contraction groups the triple
 * product sum_p conj(S_out[d,p]) H_n[p] sum_j S_in[j,p] a_j(R) (Eq. SHn0 applied to
 * the probes): EELS_ASSOC_AUTO (default) times both groupings (and, with them, both
 * tile widths of each GEMM, EELS_OPT_TILE_WIDTH) once per contraction shape on the first
 * slice that has sites and keeps the fastest choice for that shape in the context; EELS_ASSOC_TRANSITION_FIRST forms
 * M_n = S_out^H diag(H_n) S_in and then M_n a(R) (the paper's order);
 * EELS_ASSOC_PROBE_FIRST forms Y = S_in a(R) once per site (the elastic wave inside the
 * window) and then S_out^H (H_n . Y) per channel.  Both give the same map up to rounding.
 * EELS_ASSOC_MODEL picks, per call, the grouping with fewer complex products over the
 * call's sites (transition first: T (n_out w^2 n_in + n_out n_in n_R) per site; probe
 * first: n_R n_in w^2 + T n_out w^2 n_R), without timing anything, so that the choice and
 * with it the rounding of the map never depend on what else runs on the device (the map
 * server uses it).
 *
 * EELS_OPT_SHARD_COUNT (G >= 1, default 1) and EELS_OPT_SHARD_INDEX (0 <= g < G,
 * default 0) restrict eels_inelastic_map to one shard of the detector beams: beam d
 * (in the enumeration order of the aperture: rows q ascending, then p ascending)
 * belongs to shard d mod G.  The map is a sum of |.|^2 over detector beams (Alg. 2,
 * the detector sum of Eq. SHn0 applied to a probe), so the maps of the G shards add up
 * to the full map; each shard needs the full S_in but only its share of S_out.  A shard
 * with no beam returns a zero map.  eels_inelastic_map returns EELS_ERR_ARG if the
 * index is not below the count.  The paper has no sharding; this serves one process per
 * GPU, each computing one shard, with one FP64 sum of the maps at the end.
 * Returns EELS_ERR_ARG for an unknown option or value. */
#define EELS_OPT_ASSOCIATION 1
#define EELS_ASSOC_AUTO 0
#define EELS_ASSOC_TRANSITION_FIRST 1
#define EELS_ASSOC_PROBE_FIRST 2
#define EELS_ASSOC_MODEL 3
#define EELS_OPT_SHARD_COUNT 2
#define EELS_OPT_SHARD_INDEX 3
/* EELS_OPT_SOUT_SCHEME selects how eels_inelastic_map brings the detector-side
 * matrix S_out (the paper's S_2) to each depth; S_in always comes from the handle.
 *   EELS_SOUT_STREAM (default): carried backwards from the exit surface once, the
 *     contraction of each depth running as the sweep passes it; exact, n_z n_out
 *     beam-steps.
 *   EELS_SOUT_RECOMPUTE: recalculated from the exit surface for every depth that holds
 *     transitions, as the Sec. III listing does ("Re-calculate S_2"); exact, up to
 *     n_z (n_z + 1)/2 n_out beam-steps.
 *   EELS_SOUT_INVERSE: carried back to depth 0 once, then retreated one slice per depth
 *     with the inverse multislice operator (Sec. IV C, Eq. MSinvop): propagate with P,
 *     multiply by t_{i+1}, project onto the band.  Approximate: what the backward sweep
 *     scattered outside the band limit is not recovered; exact at depth 0 and in free
 *     space.  2 n_z n_out beam-steps plus one band projection per depth. */
/* EELS_OPT_EXIT_PLANE (0 default, 1): eels_build_smatrix also stores S_in at the exit
 * surface (one more depth of n_in N/2 x N/2 planes and one more half slice step), which
 * eels_elastic_images needs. */
#define EELS_OPT_EXIT_PLANE 5
/* EELS_OPT_SIN_CHECKPOINT (K >= 0, default 0): a build with K >= 2 does not store S_in at
 * every depth; it keeps the probe waves at every K-th depth (ceil(n_z / K) copies of n_in
 * N x N/2 row spectra) and eels_inelastic_map recomputes S_in one segment of K depths at a
 * time as the backward sweep reaches it (one more forward pass: n_z n_in more beam-steps).
 * The map is the same bit for bit up to the order of the FP64 sums.  K near sqrt(2 n_z)
 * minimises the memory, about (2 n_z / K + K) instead of n_z planes of (N/2)^2 per probe
 * beam; this runs specimens whose S_in does not fit in HBM.  Needs the stream S_out scheme
 * (EELS_ERR_UNSUPPORTED otherwise); eels_smatrix_copy_depth returns EELS_ERR_UNSUPPORTED
 * for such a handle.  0 and 1 store every depth. */
#define EELS_OPT_SIN_CHECKPOINT 8
/* EELS_OPT_BATCH_SITES (>= 0, default 0): at most this many sites of one slice are
 * contracted per batch of tensor-core launches; 0 sizes the batch by the operand budget
 * (EELS_OPT_OPERAND_MIB).  The map does not depend on it (up to FP64 summation order);
 * smaller batches use less device memory and more launches. */
#define EELS_OPT_BATCH_SITES 6
/* EELS_OPT_OPERAND_MIB (>= 64, default 8192): device memory, in MiB, for the tensor-core
 * operand buffers of one batch of sites; the batch holds as many sites of a slice as
 * fit (at least one).  Larger batches mean fewer, longer launches. */
#define EELS_OPT_OPERAND_MIB 9
/* EELS_OPT_TILE_WIDTH (0 default, 128 or 256): columns of the output tiles of the
 * tensor-core GEMMs (the tiles are 128 rows high).  0 lets the library choose per GEMM:
 * EELS_ASSOC_AUTO times both widths of each GEMM together with the groupings, once per
 * contraction shape, and keeps the faster; otherwise the narrow tile is taken where it
 * covers the GEMM's columns with at least 5 % fewer padded columns.  The map does not
 * depend on the width beyond rounding order. */
#define EELS_OPT_TILE_WIDTH 10
/* EELS_OPT_WAIT_TEST (>= 0, default 0), for failure-detection tests only: a value v > 0
 * limits every pipeline wait of the tensor-core kernels to 1000 v clock cycles and makes
 * their TMA producers issue no load, so that the consumers' bounded waits run out with
 * nothing in flight; each kernel then records the timeout, frees its tensor memory and
 * returns, and eels_inelastic_map returns EELS_ERR_TIMEOUT.  The context stays usable;
 * set 0 to return to normal operation. */
#define EELS_OPT_WAIT_TEST 7
/* EELS_OPT_CHECK_TEST (0 default, 1), for tests of the bounds-checked debug build only:
 * eels_inelastic_map sets the window origin of the first site that some probe reaches to
 * N/2, one past its range.
 * Every kernel that walks a window checks the origin, records the violation and skips its
 * work, and the call returns EELS_ERR_BOUNDS; an unchecked periodic walk from N/2 would
 * still stay inside the plane.  The normal build returns EELS_ERR_UNSUPPORTED. */
#define EELS_OPT_CHECK_TEST 11
/* eels_checked_build: 1 if this library was compiled with -DSTEM_CHECK, else 0. */
int eels_checked_build(void);
#define EELS_OPT_SOUT_SCHEME 4
#define EELS_SOUT_STREAM 0
#define EELS_SOUT_RECOMPUTE 1
#define EELS_SOUT_INVERSE 2
eels_status eels_set_option(eels_ctx* ctx, int option, int value);

/* Per-kernel device timing.  While enabled, every kernel launch made by calls on
 * this context is bracketed by CUDA events recorded on the launch stream.
 * eels_profile_read synchronises those events, folds them into running totals
 * and returns the number of bytes the JSON text {"kernel": {"launches": L,
 * "ms": T}, ...} needs (with its NUL).  If buf holds at least that many bytes
 * the text is written there and the totals are reset; otherwise nothing is
 * lost and the call can be repeated with a larger buffer.  Disabled by default. */
eels_status eels_profile_enable(eels_ctx* ctx, int on);
int eels_profile_read(eels_ctx* ctx, char* buf, int cap);

/* The autotuner's choices kept in the context (EELS_ASSOC_AUTO): a JSON list with one
 * object per contraction shape {"precision", "n", "n_out", "n_in", "w", "nr_max",
 * "n_types", "grouping", "tile_first", "tile_second"} (tile widths of the grouping's
 * first and second GEMM).  Returns the bytes the text needs with its NUL; writes it if
 * buf holds that many. */
int eels_tuning_read(eels_ctx* ctx, char* buf, int cap);

/* Size of the static device work array used by eels_build_smatrix_static. */
#define EELS_STATIC_SCRATCH_BYTES (64ull << 20)

/* S_in build that allocates nothing (the paper has no counterpart: this is a
 * deployment variant of eels_build_smatrix).  Some callers cannot call cudaMalloc:
 * plug-ins whose host application owns (or has reserved) all of the device memory,
 * and real-time acquisition loops that must not take the time of, or risk the
 * failure of, an allocation in the middle of a run.  This call writes what
 * eels_build_smatrix stores, S_in(i) for every depth as complex64
 * [n_z][n_in][N/2][N/2] scaled by N, into the caller's device buffer s_in
 * (s_in_bytes long), and keeps all its work arrays in one static device array of
 * EELS_STATIC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
 * vproj may be host or device memory (a host vproj is copied slice by slice into
 * the static array); it takes no context and reports errors as a status plus text
 * in err (err_cap bytes).  *n_in_out receives the number of probe beams once every
 * check has passed; a rejected call leaves it untouched.
 * - The first call on a device looks up the device address of the static array
 *   (cudaGetSymbolAddress) and keeps it for the process; make that first call
 *   before any stream capture.  The address is not looked up again, so a call
 *   after cudaDeviceReset on that device is undefined.
 * - Every call on a device shares the array and leaves its contents behind;
 *   calls whose GPU work overlaps (different streams or threads) race.
 * - Waves are processed in chunks sized to the static array (at N = 512 about 30
 *   waves per chunk, at N = 1024 six).
 * - EELS_ERR_ARG if s_in_bytes < n_z n_in (N/2)^2 * 8 or if not even one N x N/2
 *   complex64 work wave pair plus one slice of tables fits in the static array;
 *   EELS_ERR_UNSUPPORTED for an unbuilt grid size. */
eels_status eels_build_smatrix_static(const eels_specimen* spec, const eels_optics* optics,
                                      float* s_in, int64_t s_in_bytes, int* n_in_out,
                                      void* stream, char* err, int err_cap);

/* ---------------------------------------------------------------------------
 * Map server (not in the paper: a serving loop around the calls above).
 * A request is one complete map: S-matrix build plus inelastic map.  Requests are
 * queued in arrival order and admitted as soon as the request's device footprint
 * (eels_request_footprint) fits in what is left of hbm_budget bytes; admission is
 * first-fit in arrival order, and a request bypassed eight times stops further
 * bypassing until it is admitted.  Each admitted request runs on its own context and
 * non-blocking stream, and its S_in stays resident until its map is done.
 * Work is issued in tiles of four slices of the build or four depths of the map (the
 * backward S_out step and the contraction of the sites at those depths).  `slots` issue
 * tokens gate the device: a request holds a token while it issues one tile, lets that
 * tile finish, hands the token to the request that has waited longest and queues again,
 * so the tiles of admitted requests interleave and overlap on the device.  A cancelled
 * request, or one past its deadline, is dropped at its next tile boundary (or before
 * admission) with EELS_ERR_CANCELLED and its memory released.  Contexts of the server
 * use EELS_ASSOC_MODEL, so a request's map does not depend on the other requests.
 * --------------------------------------------------------------------------- */
typedef struct eels_server eels_server;

typedef struct {
  eels_specimen spec;        /* host vproj */
  eels_optics optics;
  eels_transitions tr;       /* host arrays */
  eels_scan scan;
  double beta;
  int precision;             /* eels_precision */
  double deadline_s;         /* > 0: dropped once this many seconds have passed since
                                submission (checked at tile boundaries); 0: no deadline */
  int sin_checkpoint;        /* as EELS_OPT_SIN_CHECKPOINT; -1: the server picks
                                K = ceil(sqrt(2 n_z)) if storing every depth would take more
                                than half its budget, else stores every depth */
} eels_request;

typedef struct {
  int64_t submitted, completed, failed, cancelled;
  double p50_ms, p99_ms, mean_ms, max_ms;   /* submit -> done latency of completed requests */
  double mean_wait_ms;                      /* submit -> first tile issued */
  double makespan_s;                        /* first submit -> last completion */
  double pixel_slices_per_s;                /* sum of n_scan n_z of completed requests / makespan */
  int64_t peak_bytes;                       /* largest sum of admitted footprints */
} eels_server_stats;

/* Progress of one request; times in seconds since the server was created, -1 if the
 * event has not happened. */
typedef struct {
  int done;                 /* 1 once finished (completed, failed or cancelled) */
  int status;               /* eels_status once done */
  double t_submit, t_admit, t_first_tile, t_done;
  int tiles;                /* tiles issued */
  int64_t footprint;        /* device bytes reserved while admitted */
  int n_in, n_out;          /* probe beams (alpha) and detector beams (beta) on the f-lattice */
  int64_t pixel_slices;     /* n_sx n_sy n_z */
  int64_t wave_steps;       /* multislice wave-slice steps issued for the request: n_in n_z
                               (build) + n_out n_z (S_out stream) + n_in n_z again when S_in
                               is checkpointed (segment recompute) */
  double contraction_flops; /* flops of the map's contraction as grouped, 8 per complex
                               product (once finished; 0 before) */
} eels_request_info;

/* Device bytes the server reserves for a request while it runs: transmissions, S_in (or
 * its checkpoints when sin_checkpoint >= 2), the larger of the build's work arrays and the
 * map's (backward work arrays, one S_out depth, a 4 GiB cap for contraction buffers, the
 * transition potentials and, with checkpoints, the forward work arrays and one segment of
 * S_in).  sin_checkpoint = -1 counts as 0.  -1 for invalid sizes. */
int64_t eels_request_footprint(const eels_request* req);
/* Start a server on `device` with `slots` issue tokens and an HBM budget of hbm_budget
 * bytes. */
eels_status eels_server_create(int device, int64_t hbm_budget, int slots, eels_server** out);
/* Queue a request; its input arrays are BORROWED until eels_server_wait has returned
 * for it.  *id identifies it.  EELS_ERR_OOM if its footprint exceeds the whole budget,
 * EELS_ERR_ARG for device inputs, a negative deadline or invalid sizes. */
eels_status eels_server_submit(eels_server* sv, const eels_request* req, int64_t* id);
/* Ask for request id to be dropped: at once if it is not admitted yet, else at its next
 * tile boundary.  Its wait then returns EELS_ERR_CANCELLED.  No effect once it is done. */
eels_status eels_server_cancel(eels_server* sv, int64_t id);
/* Block until request id is done (timeout_s <= 0: no limit) and copy its FP64 map
 * [n_types][n_sy][n_sx] to host map_out (may be NULL); *latency_s (if non-NULL) gets its
 * submit-to-completion time.  Returns the request's own status, or EELS_ERR_TIMEOUT. */
eels_status eels_server_wait(eels_server* sv, int64_t id, double* map_out, double timeout_s,
                             double* latency_s);
eels_status eels_server_request_info(eels_server* sv, int64_t id, eels_request_info* out);
eels_status eels_server_stats_get(eels_server* sv, eels_server_stats* out);
/* Stop admitting; requests not yet admitted are dropped, admitted ones run to completion. */
void eels_server_destroy(eels_server* sv);

/* Measured FP32 FMA rate of device `device` (flop/s, 2 per FMA), the denominator of
 * the CUDA-core ALU roofline (no counterpart in the paper: a measurement aid).  Runs
 * one launch of independent FMA chains, `iters` FMAs per chain, timed with CUDA
 * events on the legacy default stream (about 1e9 iters take a few hundred ms). */
eels_status eels_fp32_fma_rate(int device, int iters, double* flops_per_s);

/* Number of f-lattice beams with lambda |k| <= angle (Sec. III, pi alpha^2 L^2 / f^2). */
int eels_count_beams(int n, double cell, double lambda, int f, double angle);

/* The paper's memory model (Sec. III memory paragraph), in bytes of
 * single-precision complex arrays: out[0] = conventional minimum, 4 N^2;
 * out[1] = transmission functions, n_z N^2; out[2] = both scattering matrices,
 * (planes_in + planes_out) (N/2)^2.  Returns EELS_ERR_ARG for invalid sizes. */
eels_status eels_memory_model(int n, int n_z, int planes_in, int planes_out, int64_t out[3]);

/* Device bytes of a request (Sec. III memory paragraph):
 * transmissions n_z N^2 + S_in n_z n_in (N/2)^2 + one S_out depth n_out (N/2)^2
 * complex64 values, plus two multislice work arrays of chunk * N * N/2 values.
 * Returns -1 for invalid arguments. */
int64_t eels_footprint_bytes(int n, int n_z, int n_in, int n_out, int chunk);

#ifdef __cplusplus
}
#endif
#endif /* STEM_EELS_H */
