// Internal declarations shared by the translation units of libfitrig.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fitrig.h"

namespace fitrig {

constexpr float kGuardC = 1e-6f;           // Eq. 5 guard constant C
constexpr double kMadToSigma = 1.482602218505602;  // 1 / Phi^-1(3/4)

// Device error flags (bit mask in Plan::d_status[0]).
enum : unsigned {
  kErrTimeout = 1u,      // an mbarrier wait gave up
  kErrCcLimit = 2u,      // union-find retry bound reached
  kErrCapacity = 4u,     // a list exceeded its capacity
};

// ---------------------------------------------------------------- keys
// Order-preserving map float -> uint32 (NaN must be filtered by the caller).
__host__ __device__ inline uint32_t f32_key(float f) {
#ifdef __CUDA_ARCH__
  uint32_t b = __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
#endif
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ inline float f32_from_key(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
__device__ inline unsigned long long f64_key(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// ---------------------------------------------------------------- storage types
struct bf16_t { uint16_t v; };
struct f16_t { uint16_t v; };

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(bf16_t x) { return __uint_as_float(((uint32_t)x.v) << 16); }
__device__ __forceinline__ float to_f32(f16_t x) {
  float f;
  asm("{ .reg .f16 h; mov.b16 h, %1; cvt.f32.f16 %0, h; }" : "=f"(f) : "h"(x.v));
  return f;
}

// One warp's maximum of v into *key (order-preserving key; -inf is skipped).
// Every lane of the warp must call it.
__device__ __forceinline__ void warp_max_to(float v, unsigned* key) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > -INFINITY) atomicMax(key, f32_key(v));
}

// Three-input maximum (one instruction on sm_100 and later; NaN inputs are
// ignored unless all are NaN, as with fmaxf).
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// ---------------------------------------------------------------- PTX: time, mbarrier, TMA
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: spins on try_wait until the phase completes or `deadline`
// (globaltimer ns) passes; returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t deadline) {
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && globaltimer_ns() > deadline) return false;
  }
}
// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Programmatic dependent launch.  A kernel launched by launch_pdl may be set
// up while the kernel ahead of it in the stream is finishing, so that a chain
// of short kernels does not pay a full launch gap at every step.  Every
// kernel that may be launched that way begins with pdl_begin(), which waits
// (in hardware, not a spin) until the grids this one depends on have
// completed and their writes are visible; launched normally, it is a no-op.
// No kernel signals its dependents early: CTAs parked in that wait would hold
// SM resources that the other stream's kernels of a detect use.
__device__ __forceinline__ void pdl_begin() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------- host-side launchers
// Adds n to the process-wide count of kernel launches (fitrig_launch_count).
void count_launches(int n);
// Launches kernel k with programmatic stream serialisation allowed (the kernel
// must start with pdl_begin()).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Stack-march geometry chosen on the host (see k_stack.cu).
struct StackGeom {
  int w;              // tile size
  int R;              // rows per thread segment (template parameter)
  int nseg;           // row segments per tile band
  int TBX, TBY;       // tiles per CTA in x / y
  int BW;             // pixel columns per CTA (TBX * w)
  int BH;             // pixel rows per CTA (TBY * w)
  int boxW;           // TMA box width (BW, or widened for unaligned origins)
  bool aligned;       // CTA column origin always a multiple of 8 elements
  int stages;         // TMA ring depth
  int threads;        // BW * TBY * nseg
  size_t stage_bytes; // boxW * BH * elem, rounded to 128
  size_t smem_bytes;
  int gridX, gridY;
};

struct StackArgs {
  int nx, ny;          // analysed image size (cropped in EDGE_DROP)
  int nsnap;           // snapshots to march over (>= 3)
  int Tx, Ty;
  int64_t T;           // Tx * Ty
  int64_t vstride;     // floats between units in vp (T rounded up to 4)
  float* vp;           // [nsnap-2][vstride] tile statistic (NaN padding)
  uint8_t* arg = nullptr;     // [nsnap-2][vstride] in-tile arg-max of Delta (small path), or null
  int zrot;            // snapshot j of the march is stack slot (zrot + j) % nsnap (ring use)
  unsigned* gmax;      // ordered key of the running maximum
  unsigned* smax = nullptr;   // [nsnap] ordered key of each snapshot's maximum, or null
  unsigned* status;    // error flags
  uint64_t timeout_ns;
  StackGeom g;
  const float* key = nullptr;   // difference-coded stack: FP32 snapshot 0 ([ny][kpitch]),
  int64_t kpitch = 0;           // the stack slots 1.. then hold half differences
};

// One field of a batched (persistent, multi-field) stack march.  The TMA
// descriptor must stay 64-byte aligned in device memory.
struct alignas(128) FieldDesc {
  CUtensorMap tmap;
  int zrot;            // as StackArgs::zrot
  float* vp;
  uint8_t* arg;
  unsigned* gmax;
  unsigned* smax = nullptr;   // as StackArgs::smax
  unsigned* status;
  int nx, ny, L, Tx, Ty, gridX;
  int64_t vstride;
  int64_t item0;       // first work item (box) of this field
};
cudaError_t launch_stack_multi(const FieldDesc* fields, int nfields, int64_t nitems,
                               unsigned long long* counter, const StackGeom& g, int grid,
                               int storage, int rmode, uint64_t timeout_ns, cudaStream_t st);
int multi_blocks_per_sm(const StackGeom& g, int storage, int rmode);

bool stack_geometry(int w, int elem_bytes, StackGeom* g);
// Thread-per-tile geometry for 3 <= w <= 6 with TBY tile rows per CTA and a
// ring of `stages` buffers (the autotuner's search space).
bool small_geometry(int w, int elem_bytes, int tby, int stages, StackGeom* g);
cudaError_t launch_stack(const CUtensorMap* tmap, const StackArgs& a, int storage, int rmode,
                         cudaStream_t st);
cudaError_t launch_finite_max(const void* stack, int storage, int L, int ny, int nx,
                              int64_t pitch, unsigned* gmax, cudaStream_t st);
// The same for a difference-coded stack (decoded in snapshot order): the
// finite maximum over every snapshot into *gmax (if set), and with smax (2L
// words, as launch_running_norm's) the finite maximum of each snapshot whose
// fused maximum smax[k] was +inf into smax[L + k].  L <= kDeltaMaxSnaps when
// smax is set.
constexpr int kDeltaMaxSnaps = 8192;
cudaError_t launch_delta_finite_max(const float* key, int64_t kpitch, const void* stack,
                                    int storage, int L, int ny, int nx, int64_t pitch,
                                    unsigned* gmax, unsigned* smax, cudaStream_t st);
// One device wait, bounded like the march's, on a barrier nothing completes.
cudaError_t launch_wait_probe(uint64_t timeout_ns, unsigned* gave_up, cudaStream_t st);

// Sliding-window mode geometry (see k_slide.cu).
struct SlideGeom {
  int w, h;            // window and half-width
  int OW, OH;          // output pixels per CTA
  int EW, EH;          // extended block with halo
  int nseg;            // row segments of kSlideR rows
  int boxW;            // TMA box width (x origin rounded down to 8 elements)
  int threads, stages;
  size_t stage_bytes, smem_bytes;
  int gridX, gridY;
};
struct SlideArgs {
  int nx, ny, nsnap;
  int zrot;            // snapshot j is stack slot (zrot + j) % nsnap
  int64_t vstride;     // floats between units in vp (nx*ny rounded up to 4)
  float* vp;           // [nsnap-2][vstride]
  unsigned* gmax;
  unsigned* smax = nullptr;   // [nsnap] per-snapshot maximum keys, or null
  unsigned* status;
  uint64_t timeout_ns;
  SlideGeom g;
};
bool slide_geometry(int w, int elem_bytes, SlideGeom* g);
cudaError_t launch_slide(const CUtensorMap* tmap, const SlideArgs& a, int storage, int rmode,
                         cudaStream_t st);

// Noise: per-group centre/scale of `vals` ([groups][n], NaN = excluded).
struct NoiseScratch {
  double* part;        // [groups][nblk] partial sums
  int* cnt;            // [groups][nblk] partial counts
  unsigned* hist;      // [groups][2048] radix histogram
  unsigned* rsel;      // [groups][4] radix-select state
  float* shift;        // [groups] FP32 mean used by the second MEANSTD pass
  unsigned long long* invalid;  // device counter of non-finite values seen (may be null)
  int nblk;
  bool allow_cluster = true;    // median/MAD may use the one-launch cluster form
  // median/MAD of groups up to 2 Mi values: per-group state and key copies of
  // the split form (noise_split_bytes); null: the bracketed cluster form
  void* split = nullptr;
  int64_t split_cap = 0;        // copied keys per group
};
size_t noise_scratch_bytes(int groups, int nblk);
void noise_scratch_carve(void* base, int groups, int nblk, NoiseScratch* s);
// Scratch of the split median/MAD form for `groups` maps of `stride` values
// (0 when maps that large take another form).
size_t noise_split_bytes(int groups, int64_t stride);
void noise_split_carve(void* base, int groups, int64_t stride, NoiseScratch* s);
// Group g's values are vals[g*stride .. g*stride + stride); entries that are
// not finite (including padding) are skipped; n = real entries per group
// (for the count of invalid ones).
cudaError_t launch_noise(const float* vals, int groups, int64_t stride, int64_t n, int mode,
                         const NoiseScratch& s, double* centre_scale, cudaStream_t st);
// thr32[g] = largest float <= centre + tau*scale (+inf if degenerate), and
// inv_scale[g] = 1/scale (0 if degenerate)
cudaError_t launch_thresholds(const double* centre_scale, int groups, double tau, float* thr,
                              double* inv_scale, cudaStream_t st);

// Selection / components / candidates.
// One selected tile: its group (unit, or 0 for eta), tile index and value.
// Within a group z = (v - centre) / scale is strictly increasing in v, so the
// value orders the tiles of a component exactly; the FP64 significance is
// computed for the candidates only.
struct SelItem {
  int32_t group;
  int32_t t;
  float v;
};
struct SelectScratch {
  int nblk;            // fixed grid of the ordered compaction
  int* blkcnt;         // [nblk]
  int* blkoff;         // [nblk + 1]
  SelItem* items;      // capacity entries
  int* nsel;           // device count
  int* parent;         // capacity
  unsigned* compmax;   // capacity: largest value key of each component
  int* peak;           // capacity
  uint32_t* bits;      // [nwords] selection bitmap over the element space groups * stride
  int* wbase;          // [nwords] list index of the first selected element of each word
  int* plist;          // capacity: list indices of component peaks, in list order
  int* npeak;          // device count of plist
  int64_t capacity;
  unsigned* want;      // max over overflowing selections of the entries needed
};
// Element space [0, groups*stride); selected entries get SelItem{g, t, z} in
// order and map[g*stride + t] = list index + 1.  blkcnt/blkoff need nblk*8
// entries (one per warp).
cudaError_t launch_select(const float* vals, int groups, int64_t stride, const float* thr,
                          const SelectScratch& s, unsigned* status, cudaStream_t st);
cudaError_t launch_count_selected(const float* vals, int groups, int64_t stride, const float* thr,
                                  int nblk, int* wcnt, long long* total, cudaStream_t st);
cudaError_t launch_clamp_count(int* n, int cap, unsigned* status, cudaStream_t st);
cudaError_t launch_components(int Tx, int Ty, int64_t T, const SelectScratch& s,
                              unsigned* status, cudaStream_t st);

// Block-tiled selection and components: each CTA takes a kBlkY x kBlkX block
// of one group's tile map.  Components that touch a block edge are merged
// through a global union-find over "boundary components"; every peak ends up
// as a bit in a dense per-group bitmap, compacted in (group, t) order.
constexpr int kBlkY = 64, kBlkX = 64;
struct BlockScratch {
  int* glab;                  // [groups * stride] boundary-component id of edge tiles (never cleared)
  int* bpar;                  // [cap] union-find parents of boundary components (block slots)
  int* bgrp;                  // [cap] group of each boundary component
  unsigned long long* bkey;   // [cap] block-local peak key (value key << 32 | ~t)
  unsigned long long* rkey;   // [cap] merged peak key (roots)
  uint32_t* pbits;            // [groups][Ty][words] peak bitmap
  uint32_t* sbits;            // [groups][Ty][words] selected-tile bitmap (v > thr)
  unsigned long long* pairs;  // [blocks][pairs per block] selected neighbours across block edges
  int64_t pcap;
  int4* bstat;                // [blocks] boundary components, pairs, selected tiles of each block
  int* counters;              // [2] peaks
  int64_t cap;                // boundary-component slots (blocks x slots per block)
  int words;                  // bitmap words per tile row
  int nblk;                   // CTAs of the ordered compaction (kRowsPerCta tile rows each)
  int* blkcnt;                // [nblk] peaks of each CTA's rows
  int* blkoff;                // [nblk + 1] their exclusive scan
  int* rowcnt;                // [groups * Ty] peaks of each tile row
};
// Bytes of BlockScratch for `groups` maps of Ty x Tx tiles at group stride
// `stride` (carved by block_scratch_carve in the same order).
size_t block_scratch_bytes(int groups, int Tx, int Ty, int64_t stride);
void block_scratch_carve(void* base, int groups, int Tx, int Ty, int64_t stride, BlockScratch* b);
// Threshold (v > thr[g]), 8-connected components and their peaks over groups
// x Ty x Tx tiles at vals[g * stride + ty * Tx + tx]; writes the peaks, in
// (group, t) order, as SelItem{g, t, v} to peaks[0..min(n, cap)) with n in
// b.counters[2] (with peaks == nullptr the list is left to launch_emit_rows:
// the peak bitmap and the rows' offsets stay in b); flags kErrCapacity (and
// *want = selected count) when more than `cap` tiles are selected.
cudaError_t launch_block_select(const float* vals, int groups, int64_t stride, int Tx, int Ty,
                                const float* thr, const BlockScratch& b, SelItem* peaks,
                                int64_t cap, unsigned* status, unsigned* want, cudaStream_t st);

struct CandArgs {
  int nx, ny, w, Tx, Ty;
  int64_t T;
  int64_t stride;      // group stride of the selection element space
  const uint8_t* arg;  // fused in-tile arg-max [units][stride], or null (recompute)
  int branch;          // 1 image, 2 freq
  // image branch: stack access for the in-tile arg-max of Delta
  const void* stack;
  int storage;
  int64_t pitch;       // elements per row
  int64_t slice;       // elements per snapshot
  int zrot, zmod;      // snapshot j of unit 0 is slot (zrot + j) % zmod (zmod 0: slot = unit + j)
  const float* key = nullptr;   // difference-coded stack: FP32 snapshot 0 (slots 1.. hold
  int64_t kpitch = 0;           // half differences, decoded in snapshot order)
  // freq branch
  const float* eta;
  const int* bin;
  int refine;          // FITRIG_REFINE_PARABOLIC or FITRIG_REFINE_CUBIC
  // significance z = (v - cs[2g]) * inv[g] in FP64 (per group g)
  const double* cs;
  const double* inv;
  fitrig_candidate* out;
  int* nout;
  int64_t cap;
};
// Appends the branch's candidates in (snapshot, y, x) order: frequency
// candidates at positions [0, n_peaks), image candidates after *base.  Adds
// the number of peaks to *a.nout and clears the selection map.
cudaError_t launch_emit_candidates(const CandArgs& a, const SelectScratch& s, int* base,
                                   fitrig_candidate* tmp, unsigned* status, cudaStream_t st);

// The candidates of an ordered peak list (launch_block_select), as
// launch_emit_candidates does from its own list.
cudaError_t launch_emit_peaks(const CandArgs& a, const SelItem* peaks, const int* npeak,
                              int* base, fitrig_candidate* tmp, cudaStream_t st);
// The image candidates of a launch_block_select run without a peak list
// (peaks == nullptr), from its peak bitmap: needs a.arg, a.w <= 8 and
// Tx <= 1024 (one bitmap word per lane of a row's warp); the
// same candidates, in the same places, as launch_emit_peaks on the list.
// Adds the peak count to *a.nout.
cudaError_t launch_emit_rows(const CandArgs& a, const float* vals, int groups, const BlockScratch& b,
                             int64_t cap, int* base, cudaStream_t st);
cudaError_t launch_export_candidates(const fitrig_candidate* src, const int* n,
                                     fitrig_candidate* dst, int cap, cudaStream_t st);

// Frequency branch.
cudaError_t launch_spectrum(const float* vp, int n, int64_t T, int64_t vs,
                            const float2* twiddle, const float* wts, int hmax, float* eta,
                            int* bin, cudaStream_t st);
int spectrum_max_n();   // longest series launch_spectrum takes
// The twiddle table launch_spectrum expects for series of n points (host
// side, FP64 angles rounded once): the full circle (cos, sin)(2 pi a / n) for
// the radix kernel's lengths (powers of two from 128), else the direct
// kernels' rows.
std::vector<float2> spectrum_twiddles(int n);
// launch_spectrum with the transform chosen: automatic (what a plan uses),
// the direct O(n^2) warp kernel, or the radix FFT (powers of two 128..4096,
// cudaErrorInvalidValue otherwise).
enum { kSpectrumAuto = 0, kSpectrumDirect = 1, kSpectrumRadix = 2 };
cudaError_t launch_spectrum_method(const float* vp, int n, int64_t T, int64_t vs,
                                   const float2* twiddle, const float* wts, int hmax, float* eta,
                                   int* bin, int method, cudaStream_t st);

// Ingest conversion (fp32 <-> bf16/fp16).
cudaError_t launch_convert(const void* src, int src_type, int64_t src_pitch, void* dst,
                           int dst_type, int64_t dst_pitch, int ny, int nx, cudaStream_t st);
// Difference coding of one pushed snapshot (FITRIG_CODING_DELTA): with
// `first` the snapshot goes to the FP32 key frame (pitch key_pitch) and to the
// coder's running decoded snapshot `state` (ny x nx dense); otherwise
// q = half(fl32(x - state)) goes to dst (dst_type, dst_pitch) and state
// becomes fl32(state + q).
cudaError_t launch_delta_encode(const void* src, int src_type, int64_t src_pitch, float* state,
                                float* key, int64_t key_pitch, void* dst, int dst_type,
                                int64_t dst_pitch, bool first, int ny, int nx, cudaStream_t st);
// w = 1 / M^2 (M from the running-maximum key, floored at C): the weight of a
// serving unit in the real-time frequency series.
cudaError_t launch_unit_weight(const unsigned* gmax_key, float* w, cudaStream_t st);
// Snapshot accumulation: acc (FP32, ny x nx dense) = src (first) or acc + src;
// with `last` the sum goes to dst (storage type, pitch dst_pitch) instead.
cudaError_t launch_accumulate(const void* src, int src_type, int64_t src_pitch, float* acc,
                              bool first, bool last, void* dst, int dst_type, int64_t dst_pitch,
                              int ny, int nx, cudaStream_t st);

// Small helpers.
// The GPU's global nanosecond timer into *dst when the stream reaches it.
cudaError_t launch_stamp(long long* dst, cudaStream_t st);
cudaError_t launch_fill_probe(void* dst, int type, int64_t n, uint32_t seed, cudaStream_t st);
cudaError_t launch_tlisi_from_values(const float* vp, int64_t n, const unsigned* gmax,
                                     const double* m_unit, float* out, cudaStream_t st);
// Running normalisers (real-time M): smax holds 2 * nsnap keys (the march's
// per-snapshot maxima, then finite maxima where those were +inf).  A null
// stack skips the finite maxima (a difference-coded stack: the caller runs
// launch_delta_finite_max first).
cudaError_t launch_running_norm(const void* stack, int storage, int L, int ny, int nx,
                                int64_t pitch, unsigned* smax, double* m_unit, float* wts,
                                cudaStream_t st);

}  // namespace fitrig
