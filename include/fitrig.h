/*
 * fitrig.h -- C ABI of the GB300 (sm_103a) FITrig trigger library.
 *
 * FITrig (arXiv 2509.21754) flags ultra-long-period pulsars in a stack of
 * radio dirty snapshots.  For every three-snapshot unit (s, s+1, s+2) and every
 * tile t of the image it computes tLISI (Sec. 2.2.4, Eq. tLISI with Eq. 3-5),
 * turns the tile values of one unit into z-scores and keeps the tiles with
 * z > tau (Sec. 2.4.1, the image-domain branch).  The image-frequency branch
 * (Sec. 2.4.2) transforms each tile's tLISI series over the units, takes the
 * largest spectral magnitude eta_t (Eq. eta with h = maximum magnitude), and
 * thresholds the z-score of eta.  Selected tiles are merged into 8-connected
 * components and reported as candidates.
 *
 * Conventions for every call:
 *   - The return value is a fitrig_status; no call throws or aborts.
 *   - Outputs go through out-parameters; the caller owns every buffer it
 *     passes.  A plan owns all device memory it allocates and frees it in
 *     fitrig_plan_destroy.
 *   - Images are row-major, ny rows of nx pixels, x = column, y = row, both
 *     0-based.  Tiles are w x w, tile (ty, tx) covers rows ty*w .. ty*w+w-1 and
 *     columns tx*w .. tx*w+w-1; tile index t = ty * Tx + tx.
 *   - Units are 0-based: unit s spans snapshots s, s+1, s+2 (the paper's
 *     s = 1..L-2 shifted by one).
 *   - A plan is not thread-safe: use one plan per host thread.
 *   - All device work is issued on the plan's stream (FITRIG_OPT_STREAM);
 *     calls that return host-visible results synchronise that stream.  The
 *     plan's own stream (the default) is a blocking stream: it is ordered with
 *     the legacy default stream, so device buffers written there are complete
 *     before a push reads them.  With another stream the caller orders the
 *     producer of a pushed device buffer before the push.
 */
#ifndef FITRIG_H_
#define FITRIG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FITRIG_API __attribute__((visibility("default")))
#else
#define FITRIG_API
#endif

typedef struct fitrig_plan_s* fitrig_plan_t;
typedef struct fitrig_batch_s* fitrig_batch_t;
typedef struct fitrig_server_s* fitrig_server_t;

/* One serving result: the trigger of one unit of one field. */
typedef struct {
  int32_t field;         /* field id from fitrig_server_admit                       */
  int32_t unit;          /* unit s: the field's snapshots s, s+1, s+2 (s+2 arrived)  */
  int32_t ncand;         /* candidates delivered with it                             */
  int32_t status;        /* fitrig_status of the unit                                */
  int64_t t_arrival_ns;  /* the caller's stamp of snapshot s+2 (CLOCK_MONOTONIC ns)  */
  int64_t t_done_ns;     /* CLOCK_MONOTONIC ns when the result reached host memory   */
  int64_t cand_offset;   /* index of its first candidate in the poll's candidates    */
  /* where the latency t_done_ns - t_arrival_ns went (64-byte record):           */
  int64_t t_push_ns;     /* CLOCK_MONOTONIC ns when fitrig_server_push was entered   */
  int64_t t_enqueued_ns; /* ... when the unit's device work had been enqueued        */
  float copy_ms;         /* device: the snapshot's copy into the ring, from the time
                            the field's stream reached it (includes waiting for a
                            copy engine) to its end (GPU global timer)              */
  float trigger_ms;      /* device: the unit's trigger, from the end of the copy to
                            the candidates in host memory (includes SM sharing with
                            other fields' streams)                                   */
} fitrig_result;

/* One trigger candidate (32 bytes). */
typedef struct {
  int32_t x, y;          /* pixel column and row (0-based)                        */
  int32_t snapshot;      /* unit s (first snapshot of s, s+1, s+2); -1 = freq     */
  float significance;    /* z-score of the component's peak tile                  */
  int32_t branch;        /* FITRIG_BRANCH_IMAGE or FITRIG_BRANCH_FREQ             */
  int32_t freq_bin;      /* DFT bin k of eta (freq branch), -1 otherwise          */
  float xf, yf;          /* sub-tile position (freq branch), = x, y otherwise     */
} fitrig_candidate;

typedef enum {
  FITRIG_OK = 0,
  FITRIG_EINVAL = 1,       /* invalid argument                                     */
  FITRIG_ENOMEM = 2,       /* device or pinned-host allocation failed              */
  FITRIG_ESTATE = 3,       /* call not valid in the plan's current state           */
  FITRIG_ECUDA = 4,        /* a CUDA runtime call failed                           */
  FITRIG_ETIMEOUT = 5,     /* a bounded device wait gave up                        */
  FITRIG_ETRUNC = 6,       /* output buffer too small; *n holds the full count     */
  FITRIG_ENONFINITE = 7,   /* warning: non-finite pixels invalidated some tiles    */
  FITRIG_EBUSY = 8,        /* resource busy (serving admission)                    */
  FITRIG_EUNSUPPORTED = 9  /* valid but not implemented combination                */
} fitrig_status;

enum { FITRIG_BRANCH_IMAGE = 1, FITRIG_BRANCH_FREQ = 2, FITRIG_BRANCH_BOTH = 3 };
enum { FITRIG_F32 = 0, FITRIG_BF16 = 1, FITRIG_F16 = 2 };

/* Options for fitrig_plan_set. */
enum {
  FITRIG_OPT_STORAGE = 1,    /* FITRIG_F32 (default) | FITRIG_BF16 | FITRIG_F16       */
  FITRIG_OPT_NOISE = 2,      /* FITRIG_NOISE_MEANSTD (default) | FITRIG_NOISE_MEDMAD  */
  FITRIG_OPT_RMODE = 3,      /* FITRIG_RMODE_ABS (default) | FITRIG_RMODE_SIGNED      */
  FITRIG_OPT_MMODE = 4,      /* FITRIG_MMODE_GLOBAL (default) | FITRIG_MMODE_RUNNING  */
  FITRIG_OPT_EDGE = 5,       /* FITRIG_EDGE_PARTIAL (default) | FITRIG_EDGE_DROP      */
  FITRIG_OPT_STRIDE = 6,     /* FITRIG_STRIDE_TILE (default) | FITRIG_STRIDE_SLIDING  */
  FITRIG_OPT_STREAM = 8,     /* cudaStream_t cast to int64; 0 = the plan's own stream */
  FITRIG_OPT_TIMEOUT_NS = 9, /* bound of every device-side wait (default 2e9 ns)      */
  FITRIG_OPT_AUTOTUNE = 10,  /* 1: use the autotuned stack-march shape (tunes once)    */
  FITRIG_OPT_MAX_SELECTED = 11, /* selected-tile capacity of one detect; 0 = default   */
  FITRIG_OPT_GRAPH = 12,      /* 1 (default): replay repeated detects from a graph     */
  FITRIG_OPT_ACCUMULATE = 13, /* K >= 1: each K pushed snapshots are summed into one   */
  FITRIG_OPT_HARMONICS = 14,  /* m_max of the frequency branch's harmonic sum (1..32)  */
  FITRIG_OPT_REFINE = 15,     /* FITRIG_REFINE_PARABOLIC (default) | FITRIG_REFINE_CUBIC */
  FITRIG_OPT_CODING = 16      /* FITRIG_CODING_VALUE (default) | FITRIG_CODING_DELTA    */
};
/* CODING (not in the paper; half-precision storage that keeps the statistic
 * accurate): with FITRIG_CODING_DELTA and BF16 or F16 storage the plan keeps
 * snapshot 0 in FP32 (the key frame) and stores every later snapshot s as the
 * half-rounded difference from the previous *decoded* snapshot:
 *   q^(s)  = round_to_nearest_even_half(fl32(x^(s) - xt^(s-1)))
 *   xt^(s) = fl32(xt^(s-1) + q^(s)),      xt^(0) = x^(0)
 * The trigger runs on the decoded FP32 snapshots xt (the stack march decodes
 * them in registers, so D, Delta and r of Eq. 3-5 see steady sky that is
 * exact to FP32 instead of rounded to 8 or 11 significant bits).  The coder is
 * closed-loop: each decoded snapshot carries the rounding of one difference
 * only.  A non-finite input pixel (or a difference that overflows the half
 * format) makes that pixel NaN/inf in every later decoded snapshot (there is
 * no key frame to restart from).  F16 differences below 2^-14 are subnormal:
 * scale the data so that pixel differences are well above that.
 * Pushes: the first pushed snapshot (any dtype) becomes the key frame; a
 * later push of FP32 (or the other half type) is encoded on the device; a
 * later push of the storage's own half type is taken as already-encoded
 * differences q (a producer that ran the same coder), after which FP32 pushes
 * return ESTATE until fitrig_plan_reset (the device coder's running xt is
 * not updated by them).  Requires FITRIG_STRIDE_TILE, a window of 3..6 or
 * 8, 16, 32 or 64, ACCUMULATE = 1 and BF16/F16 storage (EUNSUPPORTED on the
 * first push otherwise); not in batches or serving fields.
 * fitrig_stack_device_ptr(plan, 0, ..) returns the FP32 key frame and its
 * pitch in FP32 elements; slots 1.. hold the differences.  Settable before
 * the first push; EINVAL for other values. */
enum { FITRIG_CODING_VALUE = 0, FITRIG_CODING_DELTA = 1 };
/* REFINE: the sub-tile position (xf, yf) of a frequency candidate.  Sec. 2.4.2
 * and the real-data evaluation of Sec. 3 interpolate the eta map (spline, bicubic or Makima) without a
 * formula.  PARABOLIC (default): per axis, the vertex of the parabola through
 * the peak tile's eta and its two neighbours.  CUBIC: per axis, the maximum of
 * the Catmull-Rom cubic spline through the peak tile and two neighbours on
 * each side (a missing outer sample extended linearly), within half a tile;
 * ties keep, in order, the centre, the right side, the left side.  Settable at
 * any time; EINVAL for other values. */
enum { FITRIG_REFINE_PARABOLIC = 0, FITRIG_REFINE_CUBIC = 1 };
/* HARMONICS (Sec. 2.4.2 names harmonic summing as a choice of the spectral
 * function h; the real-data evaluation of Sec. 3 applies it to the real data; the paper gives no
 * formula): with m_max > 1 (a power of two <= 32) eta_t is the largest
 * incoherent harmonic sum (|X_k| + |X_2k| + .. + |X_mk|) / sqrt(m) over
 * m = 1, 2, 4, .., m_max and the fundamentals k with m k <= floor(n/2), and
 * the reported bin is that k (ties: smaller m, then smaller k).  1 (the
 * default) is the maximum magnitude of Sec. 3.4.3.  Settable at any time;
 * EINVAL for other values. */
/* ACCUMULATE (Sec. 3.3.2, Fig. "Snapshots accumulation"): with sampling
 * periods so short that adjacent snapshots are nearly identical, the trigger
 * runs on sums of adjacent snapshots.  With K > 1 every fitrig_push_snapshot
 * adds one raw snapshot to a running FP32 sum on the device (raw snapshots
 * added in push order, the first of a block copied); the K-th raw push of a
 * block stores the sum, rounded to the plan's storage type, as the next
 * snapshot of the stack.  nsnap (fitrig_plan_create) counts these stored
 * sums, so nsnap * K raw pushes fill the stack; a detect uses the complete
 * sums only.  The paper grows the block until adjacent sums differ enough
 * but gives no criterion, so K is fixed by the caller.  Default 1 (no sums);
 * only before the first push; not for serving fields.  Costs an FP32 image of
 * device memory. */
/* GRAPH: the second fitrig_detect of an unchanged plan state (same pushed
 * snapshots count and ring position, same selection lists) captures that
 * detect's device work into a CUDA graph, which it and later detects of the
 * state replay with one launch instead of a few dozen.  Results are the same
 * either way.  0 turns this off (every detect launches its kernels one by
 * one); settable at any time. */
/* MAX_SELECTED bounds the tiles (pixels in sliding mode) that pass the
 * threshold in one detect, over all units and both branches, and so also the
 * candidates.  0 (the default) is automatic: the lists start at 4 Mi +
 * units * T / 12 entries (at most units * T; about 100 bytes of device memory
 * each) and grow when a detect selects more, in which case that detect runs
 * its post-processing (noise, selection, components, candidates) once more on
 * the same tile statistics.  A value > 0 is a hard limit: a detect that
 * selects more returns FITRIG_ETRUNC.  Set after the first push, it resizes
 * the lists at once (synchronising the plan's stream; the pushed snapshots
 * stay); a batch that holds the plan must then be created again. */
enum { FITRIG_NOISE_MEANSTD = 0, FITRIG_NOISE_MEDMAD = 1 };
enum { FITRIG_RMODE_ABS = 0, FITRIG_RMODE_SIGNED = 1 };
/* MMODE: the normaliser M of Eq. tLISI.  GLOBAL: one M, the maximum over
 * every finite pixel of the stack.  RUNNING: the real-time reading of Sec.
 * 2.2.4, unit s divided by M_s, the maximum over snapshots 0..s+2 only.  The
 * image-branch z-scores are unchanged (each unit's tiles share one M_s); the
 * reported tLISI (fitrig_tlisi) and the frequency branch's series (tLISI of
 * one tile over the units) follow the reading.  Costs one warp reduction per
 * snapshot in the march and one small kernel. */
enum { FITRIG_MMODE_GLOBAL = 0, FITRIG_MMODE_RUNNING = 1 };
enum { FITRIG_EDGE_PARTIAL = 0, FITRIG_EDGE_DROP = 1 };
/* STRIDE_SLIDING evaluates the tile statistic over the odd window centred on
 * every pixel (clipped at the border) instead of on the paper's disjoint tiles;
 * every pixel then acts as a 1 x 1 tile (Ty = ny, Tx = nx) for the noise,
 * selection, components and candidates.  Needs an odd window <= 31. */
enum { FITRIG_STRIDE_TILE = 0, FITRIG_STRIDE_SLIDING = 1 };

/* Kernels whose last device time fitrig_kernel_ms reports. */
enum { FITRIG_KERNEL_STACK = 0, FITRIG_KERNEL_NOISE = 1, FITRIG_KERNEL_SELECT = 2,
       FITRIG_KERNEL_SPECTRUM = 3, FITRIG_KERNEL_DETECT = 4, FITRIG_KERNEL_COUNT = 5 };

/*
 * fitrig_plan_create -- a plan for one field: nsnap snapshots of ny x nx
 * pixels, square tiles of `window` pixels (the paper's N_T, Sec. 2.1), z-score
 * threshold `nsigma` (tau, Sec. 2.4.1/2.4.2, strict z > tau) and `branch`.
 * Validates: window in [1, min(nx, ny)], nsnap >= 3 (>= 4 with the frequency
 * branch, whose series has nsnap-2 >= 2 points), nsigma > 0.  Device memory
 * is allocated at the first push.  EINVAL on bad arguments, EUNSUPPORTED for a
 * window above 128 or a frequency-branch series (nsnap - 2) above 4096 points.
 */
FITRIG_API int fitrig_plan_create(int nx, int ny, int nsnap, int window, double nsigma,
                                  int branch, fitrig_plan_t* out);

/* fitrig_plan_set -- set an option (see the enum).  STORAGE, NOISE, RMODE,
 * EDGE, STRIDE and AUTOTUNE are accepted only before the first push (ESTATE
 * after); STREAM, TIMEOUT_NS, MAX_SELECTED, GRAPH, HARMONICS and REFINE at any time.
 * EINVAL for an unknown option or value. */
FITRIG_API int fitrig_plan_set(fitrig_plan_t plan, int option, int64_t value);

/*
 * fitrig_push_snapshot -- copy the next snapshot (slot = number pushed so far)
 * into the plan's device stack.  `data` holds ny rows of `row_pitch_elems`
 * elements (0 means nx) of type `dtype`; it is a device pointer when
 * `on_device` is non-zero, else host memory.  A dtype different from the
 * storage type is converted on the device (round to nearest even); with
 * FITRIG_CODING_DELTA it is coded on the device instead (see
 * FITRIG_OPT_CODING).  The
 * buffer is borrowed: a host buffer may be reused when the call returns; a
 * device buffer once the plan's stream has passed this point.  ESTATE when
 * nsnap snapshots were already pushed.  Host snapshots of 32 MB or more are
 * copied in four row bands on internal side streams (ordered after the work
 * already on the plan's stream; the plan's stream waits for them), so that
 * several copy engines share the transfer; pinned host memory is fastest.
 */
FITRIG_API int fitrig_push_snapshot(fitrig_plan_t plan, const void* data, int dtype,
                                    int on_device, int64_t row_pitch_elems);

/*
 * fitrig_push_snapshots -- push `count` snapshots in one call, the same as
 * `count` calls of fitrig_push_snapshot in order: snapshot i starts
 * `snap_stride_elems` elements after snapshot i-1 (0 means row_pitch * ny) and
 * holds ny rows of `row_pitch_elems` elements (0 means nx).  A host buffer is
 * borrowed until the call returns (one synchronisation at the end, not one per
 * snapshot).  When the host snapshots are contiguous rows of the storage type
 * and the plan's rows are unpadded (nx * element size a multiple of 128 bytes),
 * the block goes as one transfer split into four row bands on the side
 * streams.  With FITRIG_OPT_ACCUMULATE = K they are raw snapshots (K per slot).
 * EINVAL for count < 0 or a stride shorter than one snapshot; ESTATE (nothing
 * pushed) when they do not fit into the remaining slots.
 */
FITRIG_API int fitrig_push_snapshots(fitrig_plan_t plan, const void* data, int32_t count,
                                     int dtype, int on_device, int64_t row_pitch_elems,
                                     int64_t snap_stride_elems);

/* fitrig_plan_reset -- forget the pushed snapshots (keeps the memory) so a new
 * stack of the same shape can be pushed. */
FITRIG_API int fitrig_plan_reset(fitrig_plan_t plan);

/*
 * fitrig_detect -- run the trigger over the pushed snapshots: tLISI for every
 * unit and tile (Sec. 2.2.4, 2.3), the noise estimate and selection of the
 * chosen branch(es) (Sec. 2.4.1, 2.4.2), components and candidates.  The
 * image branch needs >= 3 pushed snapshots, the frequency branch all nsnap.
 * Synchronises the stream and writes the number of candidates to *ncand.
 * Returns ENONFINITE (results valid) when non-finite pixels invalidated tiles,
 * ETIMEOUT if a device wait gave up, ETRUNC when more tiles passed the
 * threshold than an explicit FITRIG_OPT_MAX_SELECTED allows (then *ncand = the
 * capacity that selection needed; results are incomplete).
 */
FITRIG_API int fitrig_detect(fitrig_plan_t plan, int32_t* ncand);

/* fitrig_candidates -- copy the candidates of the last detect, sorted by
 * (snapshot, y, x), into `out` (host, `cap` entries).  ETRUNC with *n = the
 * full count when cap is too small (the first cap entries are written).
 * Pinned host memory, reused across detects, is the fastest `out`. */
FITRIG_API int fitrig_candidates(fitrig_plan_t plan, fitrig_candidate* out, int32_t cap,
                                 int32_t* n);

/* fitrig_unit_normaliser -- the M that divides unit s in the last detect:
 * the global M (as fitrig_global_max) or, with FITRIG_MMODE_RUNNING, M_s. */
FITRIG_API int fitrig_unit_normaliser(fitrig_plan_t plan, int32_t unit, double* M);

/* fitrig_tlisi -- tLISI matrix of one unit of the last detect (Ty*Tx floats,
 * row-major, host), tLISI = 1 - v/M^2 evaluated in FP64 (Eq. tLISI), M the
 * unit's normaliser (see FITRIG_OPT_MMODE). */
FITRIG_API int fitrig_tlisi(fitrig_plan_t plan, int32_t unit, float* out_host, int32_t cap);

/* fitrig_unit_values -- the M-free tile statistic v_t = mean(Delta) max(Delta)
 * mean(r) (the Eq. tLISI numerator, FP32, NaN for invalid tiles) of one unit,
 * Ty*Tx floats to host. */
FITRIG_API int fitrig_unit_values(fitrig_plan_t plan, int32_t unit, float* out_host,
                                  int32_t cap);

/* fitrig_noise_params -- centre and scale of the noise estimate of one unit of
 * v (mean/std or median/1.4826 MAD), or of eta when unit == -1. */
FITRIG_API int fitrig_noise_params(fitrig_plan_t plan, int32_t unit, double* centre,
                                   double* scale);

/* fitrig_spectrum -- eta_t (FP32, NaN for invalid tiles) and its DFT bin per
 * tile after a frequency-branch detect; either pointer may be NULL.  eta is
 * the largest DFT magnitude of the tile's mean-removed tLISI series times
 * M^2 (the global M; the z-scores do not depend on the scale). */
FITRIG_API int fitrig_spectrum(fitrig_plan_t plan, float* eta_host, int32_t* bin_host,
                               int32_t cap);

/* fitrig_global_max -- M = max(max over finite pixels of the stack, C). */
FITRIG_API int fitrig_global_max(fitrig_plan_t plan, double* M);

/* fitrig_tile_grid -- (Ty, Tx) of the plan. */
FITRIG_API int fitrig_tile_grid(fitrig_plan_t plan, int32_t* ty, int32_t* tx);

/* fitrig_kernel_ms -- device time (CUDA events on the plan stream) of one
 * kernel group of the last detect (FITRIG_KERNEL_*). */
FITRIG_API int fitrig_kernel_ms(fitrig_plan_t plan, int kernel, float* ms);

/* fitrig_stack_device_ptr -- device address of snapshot slot s of the stack
 * and its row pitch in elements (for zero-copy producers on the same device).
 * With FITRIG_CODING_DELTA slot 0 is the FP32 key frame (its own pitch) and
 * slots 1.. hold the half-precision differences. */
FITRIG_API int fitrig_stack_device_ptr(fitrig_plan_t plan, int32_t s, void** ptr,
                                       int64_t* row_pitch_elems);

/*
 * fitrig_spectrum_map -- the image-frequency statistic of Sec. 2.4.2 (Eq.
 * eta) alone, on a caller cube in device memory: T series of n points, point
 * q of series t at dev_cube[q * stride + t] (FP32; stride >= T).  For each
 * series, its mean is removed, the unnormalised DFT of exact length n is
 * taken, and eta[t] = h(|X_1..X_(n/2)|) with bin[t] its frequency bin: h is
 * the maximum magnitude (harmonics = 1) or the incoherent harmonic sum over
 * m = 1, 2, 4, .., harmonics (a power of two <= 32), as in a plan's
 * frequency branch; a series with a non-finite point gets eta = NaN, bin =
 * -1.  Outputs go to dev_eta[T] and dev_bin[T] (device memory).  `method`
 * picks the transform: FITRIG_SPECTRUM_AUTO (what a plan uses for this n),
 * FITRIG_SPECTRUM_DIRECT (a direct O(n^2) sum) or FITRIG_SPECTRUM_RADIX (the radix
 * FFT; n a power of two from 128 to 4096, EUNSUPPORTED otherwise).  2 <= n
 * <= 4096.  Allocates and frees a twiddle table; work is enqueued on `stream`
 * (a cudaStream_t, 0 = legacy default) and the call synchronises it.
 * Optional `ms` receives the transform's device time (CUDA events).  EINVAL
 * on bad arguments.
 */
enum { FITRIG_SPECTRUM_AUTO = 0, FITRIG_SPECTRUM_DIRECT = 1, FITRIG_SPECTRUM_RADIX = 2 };
FITRIG_API int fitrig_spectrum_map(const float* dev_cube, int32_t n, int64_t T, int64_t stride,
                                   int32_t harmonics, float* dev_eta, int32_t* dev_bin,
                                   int32_t method, int64_t stream, float* ms);

/*
 * fitrig_threshold_map -- the noise + threshold stage alone (Sec. 2.4.1) on a
 * caller map of n finite-or-NaN FP32 values in device memory: centre/scale by
 * `noise_mode`, and the number of entries with z > nsigma.  `stream` is a
 * cudaStream_t (0 = legacy default).  Synchronises the stream.
 */
FITRIG_API int fitrig_threshold_map(const float* dev_map, int64_t n, double nsigma,
                                    int noise_mode, int64_t stream, int64_t* nexceed,
                                    double* centre, double* scale);

/*
 * fitrig_noise_static -- the same per-group noise estimate as the trigger uses
 * (centre and scale of each of `groups` maps of `n` FP32 values, laid out one
 * after another in device memory; NaN entries are skipped): mean and
 * population standard deviation (FITRIG_NOISE_MEANSTD) or lower median and
 * 1.482602218505602 x MAD (FITRIG_NOISE_MEDMAD).  Results go to
 * dev_centre_scale[2g], [2g+1] (device memory, 2*groups doubles); work is
 * enqueued on `stream` (a cudaStream_t; 0 = legacy default) and the call does
 * not wait for it.  The paper has no counterpart of this entry point.
 *
 * It allocates nothing.  It is for callers that cannot call cudaMalloc, such
 * as a real-time trigger loop where an allocation may block or synchronise the
 * device, or a program whose device memory belongs to another allocator that
 * forbids raw allocations.  Its working memory is one fixed device array
 * inside the library (about 0.53 MB, held on every GPU that loads the library
 * until the process exits), which limits `groups` to
 * FITRIG_NOISE_STATIC_MAX_GROUPS (EINVAL beyond it) and n to INT32_MAX.
 * Every call shares that array: calls that overlap on the GPU (for example on
 * two streams at once) race and must not be issued.  The first call on a
 * device looks up the array's device address, and so does the first call
 * after the device's context was destroyed and created again (a device
 * reset); make such a call before any stream capture.  Each map is read by
 * 608 / groups blocks (at least one): with many groups, large maps are read
 * by few blocks, which is correct but slow.
 */
#define FITRIG_NOISE_STATIC_MAX_GROUPS 64
FITRIG_API int fitrig_noise_static(const float* dev_values, int32_t groups, int64_t n,
                                   int noise_mode, double* dev_centre_scale, int64_t stream);

/*
 * Batches: many fields of uneven size and snapshot count in one go.
 *
 * fitrig_batch_create -- group `nplans` plans whose snapshots are all pushed
 * (the plans stay owned by the caller and must outlive the batch, keep their
 * shapes and push counts, and share one device).  When every plan uses the
 * thread-per-tile march (tile mode, window 3..6) with the same window, storage,
 * r reading and CTA shape, all their stack marches run as ONE persistent launch
 * that takes (field, box) work items largest field first (Sec. 2.3 tiles are
 * independent); otherwise each plan's march is launched in turn.  The work is
 * issued on the first plan's stream.
 *
 * fitrig_batch_detect -- run the trigger of every plan: the first call runs it
 * once and then captures the whole sequence (marches, every plan's noise,
 * selection and candidates, counter read-backs) into a CUDA graph; later calls
 * replay the graph.  Writes each plan's candidate count to ncand[i] (in the
 * order given at creation); results are read per plan with fitrig_candidates.
 * Returns the most severe status of the plans.
 *
 * fitrig_batch_ms -- device time of the last replay (CUDA events).
 */
FITRIG_API int fitrig_batch_create(const fitrig_plan_t* plans, int32_t nplans,
                                   fitrig_batch_t* out);
FITRIG_API int fitrig_batch_detect(fitrig_batch_t batch, int32_t* ncand);
FITRIG_API int fitrig_batch_ms(fitrig_batch_t batch, float* ms);
FITRIG_API int fitrig_batch_destroy(fitrig_batch_t batch);

/*
 * Serving: fields that stream snapshots (the real-time trigger of Sec. 3.2's
 * timeline: the input transfer of snapshot s+3 overlaps the trigger kernel).
 *
 * fitrig_server_create -- a server that admits fields against
 *   `hbm_budget_bytes` of device memory and at most `max_fields` active ones.
 * fitrig_server_admit -- a field of ny x nx pixels, window, nsigma, storage
 *   type and noise mode (image-domain branch; each unit's z-scores use that
 *   unit's tiles, Sec. 2.4.1).  Reserves the field's device memory: the last
 *   three snapshots (a ring), the unit's tile statistics and selection lists.
 *   Returns OK (active) or EBUSY when it does not fit yet: the field is then
 *   queued and activated in FIFO order as retirements free memory.
 * fitrig_server_push -- the field's next snapshot (host or device memory;
 *   any of the three dtypes, converted on the device).  From the third
 *   snapshot on, every push completes one unit, whose trigger is enqueued on
 *   the field's own stream at once, overlapping other fields' work.  Returns
 *   when `data` may be reused (its copy is done); EBUSY while queued.
 *   t_arrival_ns is carried into the result (CLOCK_MONOTONIC ns).
 * fitrig_server_poll -- moves finished results (in completion order, up to
 *   `cap`) and their candidates (up to `cand_cap`, sorted by (y, x) per
 *   result) to the caller; never blocks.
 * fitrig_server_drain -- waits until every pushed unit has finished.
 * fitrig_server_retire -- finishes the field's work, frees its memory and
 *   activates waiting fields that now fit.
 * fitrig_server_field_state -- 0 queued, 1 active, 2 retired.
 * fitrig_server_usage -- reserved bytes, active and waiting field counts.
 * The server is internally synchronised: calls may come from several threads.
 */
FITRIG_API int fitrig_server_create(int64_t hbm_budget_bytes, int max_fields, fitrig_server_t* out);
FITRIG_API int fitrig_server_admit(fitrig_server_t server, int nx, int ny, int window,
                                   double nsigma, int storage, int noise, int32_t* field_id);
/* fitrig_server_admit_freq -- as fitrig_server_admit, and the field also runs
 * the image-frequency branch (Sec. 2.4.2) in real time over its last
 * `freq_units` units (2..256): the tile statistic of each completed unit is
 * kept in a ring on the device with the weight 1 / M_s^2, M_s the maximum
 * over every snapshot seen so far (the real-time reading of M, Sec. 2.2.4),
 * and from the unit that fills the ring on, every unit's result also holds
 * the frequency candidates (branch FITRIG_BRANCH_FREQ, snapshot = the unit) of
 * the unnormalised DFT of exact length freq_units over the window ending at
 * that unit: eta = the largest spectral magnitude, its z-score over the
 * field's tiles, components, tile centre + parabolic refine.  A result lists
 * its frequency candidates first, then the image candidates, each sorted by
 * (y, x).  Reserves freq_units tile maps more than fitrig_server_admit.
 * EINVAL for freq_units < 2, EUNSUPPORTED above 256. */
FITRIG_API int fitrig_server_admit_freq(fitrig_server_t server, int nx, int ny, int window,
                                        double nsigma, int storage, int noise, int freq_units,
                                        int32_t* field_id);
FITRIG_API int fitrig_server_push(fitrig_server_t server, int32_t field, const void* data,
                                  int dtype, int64_t t_arrival_ns);
FITRIG_API int fitrig_server_poll(fitrig_server_t server, fitrig_result* out, int32_t cap,
                                  fitrig_candidate* cands, int32_t cand_cap, int32_t* n,
                                  int32_t* ncands);
FITRIG_API int fitrig_server_drain(fitrig_server_t server);
FITRIG_API int fitrig_server_retire(fitrig_server_t server, int32_t field);
FITRIG_API int fitrig_server_field_state(fitrig_server_t server, int32_t field, int32_t* state);
/* fitrig_server_field_export -- checkpoint of an active field (no counterpart
 * in the paper; the real-time trigger of Sec. 3.2 keeps this state on the
 * device): its configuration, the last two snapshots as stored, the running
 * maximum M, the frequency ring with its weights and the counters, written
 * to `out` (host memory, `cap` bytes) after the field's pushed units have
 * finished.  *size = the bytes needed; ETRUNC (nothing written) when cap is
 * smaller or out is NULL; ESTATE unless the field is active.
 * fitrig_server_field_import -- a new active field from such an image, on
 * this or another server: its later pushes give exactly the results the
 * exported field would have given (unit numbers continue).  EBUSY when it
 * does not fit now (nothing is queued), EINVAL for a malformed image. */
FITRIG_API int fitrig_server_field_export(fitrig_server_t server, int32_t field, void* out,
                                          int64_t cap, int64_t* size);
FITRIG_API int fitrig_server_field_import(fitrig_server_t server, const void* image, int64_t size,
                                          int32_t* field_id);
FITRIG_API int fitrig_server_usage(fitrig_server_t server, int64_t* used_bytes, int32_t* active,
                                   int32_t* waiting);
FITRIG_API int fitrig_server_destroy(fitrig_server_t server);

/*
 * fitrig_autotune -- pick the stack-march CTA shape for a window and storage
 * type by timing each candidate (tile rows per CTA x ring depth) on a probe
 * stack of 16 snapshots of 2048 x 2048 on the current device; the winner is
 * cached for the process and used by plans with FITRIG_OPT_AUTOTUNE = 1.
 * Writes the chosen tile rows per CTA, ring depth and its time (ms per probe
 * launch).  EUNSUPPORTED for windows outside 3..6 (a single fixed shape).
 * Allocates and frees its probe memory; synchronises the device.
 */
FITRIG_API int fitrig_autotune(int window, int storage, int32_t* tile_rows, int32_t* stages,
                               float* best_ms);

/* fitrig_wait_probe -- failure detection without a fault (no counterpart in
 * the paper): one device wait on an mbarrier that nothing completes, bounded
 * by timeout_ns through the same helper as every wait of the trigger's
 * kernels (which spin on mbarrier.try_wait and give up once %globaltimer
 * passes their deadline).  Returns FITRIG_ETIMEOUT when the wait gave up --
 * the expected result -- after which the context stays usable.  timeout_ns
 * in (0, 10^10]; stream as in FITRIG_OPT_STREAM (0: legacy stream).
 * Synchronises the stream. */
FITRIG_API int fitrig_wait_probe(int64_t timeout_ns, int64_t stream);

/* fitrig_launch_count -- number of CUDA kernels this library has launched in
 * the process so far (all plans); for accounting in benchmarks. */
FITRIG_API int fitrig_launch_count(int64_t* count);

FITRIG_API int fitrig_plan_destroy(fitrig_plan_t plan);

/* Human-readable name of a status code (static storage). */
FITRIG_API const char* fitrig_status_string(int status);

/* Library version, e.g. "0.1.0". */
FITRIG_API const char* fitrig_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FITRIG_H_ */
