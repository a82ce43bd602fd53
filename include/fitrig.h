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
 *     calls that return host-visible results synchronise that stream.
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
  FITRIG_OPT_EDGE = 5,       /* FITRIG_EDGE_PARTIAL (default) | FITRIG_EDGE_DROP      */
  FITRIG_OPT_STRIDE = 6,     /* FITRIG_STRIDE_TILE (default) | FITRIG_STRIDE_SLIDING  */
  FITRIG_OPT_STREAM = 8,     /* cudaStream_t cast to int64; 0 = the plan's own stream */
  FITRIG_OPT_TIMEOUT_NS = 9  /* bound of every device-side wait (default 2e9 ns)      */
};
enum { FITRIG_NOISE_MEANSTD = 0, FITRIG_NOISE_MEDMAD = 1 };
enum { FITRIG_RMODE_ABS = 0, FITRIG_RMODE_SIGNED = 1 };
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
 * window above 128.
 */
FITRIG_API int fitrig_plan_create(int nx, int ny, int nsnap, int window, double nsigma,
                                  int branch, fitrig_plan_t* out);

/* fitrig_plan_set -- set an option (see the enum).  STORAGE, NOISE, RMODE and
 * EDGE are accepted only before the first push (ESTATE after); STREAM and
 * TIMEOUT_NS at any time.  EINVAL for an unknown option or value. */
FITRIG_API int fitrig_plan_set(fitrig_plan_t plan, int option, int64_t value);

/*
 * fitrig_push_snapshot -- copy the next snapshot (slot = number pushed so far)
 * into the plan's device stack.  `data` holds ny rows of `row_pitch_elems`
 * elements (0 means nx) of type `dtype`; it is a device pointer when
 * `on_device` is non-zero, else host memory.  A dtype different from the
 * storage type is converted on the device (round to nearest even).  The
 * buffer is borrowed: a host buffer may be reused when the call returns; a
 * device buffer once the plan's stream has passed this point.  ESTATE when
 * nsnap snapshots were already pushed.
 */
FITRIG_API int fitrig_push_snapshot(fitrig_plan_t plan, const void* data, int dtype,
                                    int on_device, int64_t row_pitch_elems);

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
 * ETIMEOUT if a device wait gave up.
 */
FITRIG_API int fitrig_detect(fitrig_plan_t plan, int32_t* ncand);

/* fitrig_candidates -- copy the candidates of the last detect, sorted by
 * (snapshot, y, x), into `out` (host, `cap` entries).  ETRUNC with *n = the
 * full count when cap is too small (the first cap entries are written). */
FITRIG_API int fitrig_candidates(fitrig_plan_t plan, fitrig_candidate* out, int32_t cap,
                                 int32_t* n);

/* fitrig_tlisi -- tLISI matrix of one unit of the last detect (Ty*Tx floats,
 * row-major, host), tLISI = 1 - v/M^2 evaluated in FP64 (Eq. tLISI). */
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
 * tile after a frequency-branch detect; either pointer may be NULL. */
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
 * and its row pitch in elements (for zero-copy producers on the same device). */
FITRIG_API int fitrig_stack_device_ptr(fitrig_plan_t plan, int32_t s, void** ptr,
                                       int64_t* row_pitch_elems);

/*
 * fitrig_threshold_map -- the noise + threshold stage alone (Sec. 2.4.1) on a
 * caller map of n finite-or-NaN FP32 values in device memory: centre/scale by
 * `noise_mode`, and the number of entries with z > nsigma.  `stream` is a
 * cudaStream_t (0 = legacy default).  Synchronises the stream.
 */
FITRIG_API int fitrig_threshold_map(const float* dev_map, int64_t n, double nsigma,
                                    int noise_mode, int64_t stream, int64_t* nexceed,
                                    double* centre, double* scale);

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
