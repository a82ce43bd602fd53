// Plan runtime and the C ABI declared in include/fitrig.h.
//
// A plan owns one field's device memory: the snapshot stack (L x ny x pitch,
// rows padded to 128 bytes so every row start is TMA-aligned), the tile
// statistic cube [L-2][T], per-unit noise parameters and thresholds, the
// selection / component lists and the candidate buffers.  fitrig_detect
// enqueues the whole trigger on the plan stream and synchronises once, when
// the candidate count is read back.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <deque>
#include <map>
#include <mutex>
#include <time.h>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

using namespace fitrig;

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int elem_bytes(int t) { return t == FITRIG_F32 ? 4 : 2; }

std::atomic<long long> g_launches{0};

}  // namespace

void fitrig::count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct fitrig_plan_s {
  // configuration
  int nx = 0, ny = 0, L = 0, w = 0, branch = 0;
  double tau = 0.0;
  int storage = FITRIG_F32, noise = FITRIG_NOISE_MEANSTD, rmode = FITRIG_RMODE_ABS;
  int edge = FITRIG_EDGE_PARTIAL;
  int stride = FITRIG_STRIDE_TILE;
  int mmode = FITRIG_MMODE_GLOBAL;
  int autotune = 0;
  // real-time frequency branch of a serving field: a ring of the last hist_n
  // units' tile statistics, with each unit's weight 1 / M_s^2 (running M)
  int hist_n = 0;
  int64_t hist_units = 0;    // units written into the ring so far
  bool freq_ready = false;   // the ring holds hist_n units
  float* d_hist = nullptr;   // [hist_n][vstride]
  float* d_hwts = nullptr;   // [hist_n]
  float2* d_htw = nullptr;   // twiddles of length hist_n
  int accumulate = 1;        // raw snapshots summed into one stack snapshot
  // difference-coded half storage: FP32 key frame (snapshot 0) and the
  // device coder's running decoded snapshot
  int coding = FITRIG_CODING_VALUE;
  float* d_key = nullptr;    // [ny][kpitch]
  float* d_dstate = nullptr; // [ny][nx]
  int64_t kpitch = 0;
  bool dstate_stale = false; // already-encoded differences were pushed
  int hmax = 1;              // harmonics of the frequency branch's h (1: max magnitude)
  int refine = FITRIG_REFINE_PARABOLIC;   // frequency candidates' position refine
  int raw_pushed = 0;        // raw snapshots of the block being summed
  float* d_accum = nullptr;  // [ny][nx] FP32 running sum (accumulate > 1)
  int64_t max_selected = 0;  // 0: automatic selection capacity
  int64_t auto_selected = 0; // the automatic capacity after growing (0: default)
  int64_t sel_bytes = 0;     // device bytes of the selection lists
  bool ring = false;       // serving field: the stack is a ring of L slots
  int64_t bytes = 0;       // device bytes allocated by the plan
  int zrot = 0;            // slot of the current unit's first snapshot
  uint64_t timeout_ns = 2000000000ull;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  // derived
  int Tx = 0, Ty = 0, nxu = 0, nyu = 0, units = 0;
  int64_t T = 0;
  int64_t vstride = 0;     // floats between units of the statistic cube
  int64_t pitch = 0;       // elements per row
  size_t slice_bytes = 0;  // bytes per snapshot
  StackGeom geom{};
  SlideGeom sgeom{};
  int pushed = 0;
  bool allocated = false;
  bool detected = false;
  int last_ncand = 0;
  int detected_branch = 0;
  int detected_units = 0;
  // device memory
  char* d_stack = nullptr;
  float* d_vp = nullptr;
  uint8_t* d_arg = nullptr;      // fused in-tile arg-max (thread-per-tile path)
  double* d_inv = nullptr;       // units + 1 reciprocal scales
  unsigned* d_small = nullptr;   // [0] gmax key, [1] status flags, [2] ncand
  unsigned long long* d_invalid = nullptr;
  double* d_cs = nullptr;        // (units + 1) x (centre, scale)
  float* d_thr = nullptr;        // units + 1
  void* d_noise = nullptr;
  void* d_split = nullptr;       // split median/MAD scratch (NoiseScratch::split)
  void* d_blk = nullptr;         // block-tiled components (BlockScratch) of the image branch
  BlockScratch blk{};
  // the frequency branch runs beside the image branch (its own stream), so
  // it has its own noise, split, components and peak buffers
  void* d_noise_f = nullptr;
  void* d_split_f = nullptr;
  void* d_blk_f = nullptr;
  BlockScratch blk_f{};
  SelItem* d_fpeaks = nullptr;   // [T] eta's component peaks
  cudaStream_t side_st = nullptr;   // the image branch's post-march work
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  NoiseScratch ns_img{}, ns_freq{};
  void* d_sel = nullptr;
  SelectScratch sel{};
  fitrig_candidate* d_cand = nullptr;
  fitrig_candidate* d_cand_tmp = nullptr;
  int64_t cand_cap = 0;
  float* d_eta = nullptr;        // slot U of d_vp (frequency branch)
  int* d_bin = nullptr;
  float2* d_tw = nullptr;
  void* d_staging = nullptr;
  float* d_report = nullptr;
  unsigned* d_smax = nullptr;    // running M: [2L] per-snapshot maximum keys
  double* d_mrun = nullptr;      // running M: [units] normaliser of each unit
  float* d_wts = nullptr;        // running M: [units] frequency-series weights
  unsigned* h_pinned = nullptr;   // [0..3] readback words
  CUtensorMap tmap;
  cudaEvent_t ev[2 * FITRIG_KERNEL_COUNT] = {};
  float ms[FITRIG_KERNEL_COUNT] = {};
  // host-to-device pushes are split over these streams (several copy engines)
  cudaStream_t copy_st[4] = {};
  cudaEvent_t copy_ev[5] = {};
  // a detect repeated on the same state replays a captured graph of its
  // stream work (see fitrig_detect); the state is (pushed, zrot, generation
  // of the selection lists)
  int64_t sel_gen = 0;
  int64_t last_key[3] = {-1, -1, -1};
  int64_t graph_key[3] = {-1, -1, -1};
  cudaGraphExec_t graph = nullptr;
  long long graph_launches = 0;
  bool no_graph = false;
  bool capturing = false;
};

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) {                       \
      (void)cudaGetLastError();                    \
      return e_ == cudaErrorMemoryAllocation ? FITRIG_ENOMEM : FITRIG_ECUDA; \
    }                                              \
  } while (0)

static cudaStream_t plan_stream(fitrig_plan_t p) { return p->stream ? p->stream : p->own_stream; }

// Selected tiles one detect can hold (also the candidate capacity).  The
// automatic capacity starts at 1/12 of all tiles of all units plus 4 Mi and
// grows when a detect needs more (the median/MAD trigger on dirty-image stacks
// selects 5-11% of tiles at 6 sigma: the statistic's right tail is heavy); an
// explicit MAX_SELECTED is a hard limit (ETRUNC beyond it).  Capped by the tile
// count and by the int32 list indices.
static int select_capacity(fitrig_plan_t p) {
  const int64_t all = (int64_t)p->units * p->T;
  int64_t cap = p->max_selected > 0    ? p->max_selected
                : p->auto_selected > 0 ? p->auto_selected
                                       : (int64_t)(4 << 20) + all / 12;
  cap = std::min<int64_t>(std::min<int64_t>(cap, all), (int64_t)INT32_MAX - 1);
  return (int)std::max<int64_t>(cap, 1);
}

static void drop_graph(fitrig_plan_t p);

static void free_all(fitrig_plan_t p) {
  drop_graph(p);
  void* ptrs[] = {p->d_stack, p->d_vp,  p->d_small, p->d_invalid,  p->d_cs, p->d_arg, p->d_inv,
                  p->d_thr,   p->d_noise, p->d_split, p->d_blk, p->d_noise_f, p->d_split_f,
                  p->d_blk_f, p->d_fpeaks, p->d_sel, p->d_cand, p->d_cand_tmp,
                  p->d_bin,   p->d_tw,  p->d_staging, p->d_report, p->d_accum,
                  p->d_hist,  p->d_hwts, p->d_htw,
                  p->d_smax,  p->d_mrun, p->d_wts, p->d_key, p->d_dstate};   // d_eta lives inside d_vp
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->h_pinned) cudaFreeHost(p->h_pinned);
  p->h_pinned = nullptr;
  p->allocated = false;
}

// ---------------------------------------------------------------- autotuner
// Times every thread-per-tile shape (tile rows per CTA x ring depth) of the
// stack march on a probe stack and keeps the fastest per (window, storage).
namespace {
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, std::pair<std::pair<int, int>, float>> g_tuned;
}  // namespace

static int run_autotune(int w, int storage, int* tby_out, int* ns_out, float* ms_out) {
  const int eb = elem_bytes(storage);
  const int L = 16, ny = 2048, nx = 2048;
  const int64_t pitch = ((int64_t)nx * eb + 127) / 128 * 128 / eb;
  const size_t slice = (size_t)pitch * ny * eb;
  const int Tx = (nx + w - 1) / w, Ty = (ny + w - 1) / w;
  const int64_t T = (int64_t)Tx * Ty, vs = (T + 3) / 4 * 4;
  void* stack = nullptr;
  float* vp = nullptr;
  unsigned* small = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FITRIG_OK;
  float best = 1e30f;
  int btby = 4, bns = 4;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return FITRIG_ECUDA;
  if (cudaMalloc(&stack, slice * L) != cudaSuccess || cudaMalloc(&vp, sizeof(float) * (L - 2) * vs) != cudaSuccess ||
      cudaMalloc(&small, 64) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = FITRIG_ENOMEM;
  }
  if (rc == FITRIG_OK && launch_fill_probe(stack, storage, (int64_t)(slice / eb) * L, 12345u, st) != cudaSuccess)
    rc = FITRIG_ECUDA;
  const CUtensorMapDataType dt = storage == FITRIG_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : storage == FITRIG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const int tbys[3] = {2, 4, 8}, nss[4] = {2, 3, 4, 6};
  for (int a = 0; a < 3 && rc == FITRIG_OK; ++a) {
    for (int b = 0; b < 4 && rc == FITRIG_OK; ++b) {
      StackGeom g;
      if (!small_geometry(w, eb, tbys[a], nss[b], &g)) continue;
      g.gridX = (Tx + g.TBX - 1) / g.TBX;
      g.gridY = (Ty + g.TBY - 1) / g.TBY;
      CUtensorMap tmap;
      const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)L};
      const cuuint64_t strides[2] = {(cuuint64_t)pitch * eb, (cuuint64_t)slice};
      const cuuint32_t box[3] = {(cuuint32_t)g.boxW, (cuuint32_t)g.BH, 1};
      const cuuint32_t es[3] = {1, 1, 1};
      if (enc(&tmap, dt, 3, stack, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        rc = FITRIG_ECUDA;
        break;
      }
      StackArgs sa{};   // every field starts zeroed (null pointers)
      sa.nx = nx;
      sa.ny = ny;
      sa.nsnap = L;
      sa.Tx = Tx;
      sa.Ty = Ty;
      sa.T = T;
      sa.vstride = vs;
      sa.vp = vp;
      sa.arg = nullptr;
      sa.zrot = 0;
      sa.gmax = small;
      sa.status = small + 1;
      sa.timeout_ns = 2000000000ull;
      sa.g = g;
      float total = 0.f;
      for (int it = 0; it < 4 && rc == FITRIG_OK; ++it) {
        if (cudaEventRecord(e0, st) != cudaSuccess || launch_stack(&tmap, sa, storage, FITRIG_RMODE_ABS, st) != cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          rc = FITRIG_ECUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (it > 0) total += ms;   // the first launch warms up
      }
      const float ms = total / 3.f;
      if (rc == FITRIG_OK && ms < best) {
        best = ms;
        btby = tbys[a];
        bns = nss[b];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (stack) cudaFree(stack);
  if (vp) cudaFree(vp);
  if (small) cudaFree(small);
  if (rc != FITRIG_OK) {
    (void)cudaGetLastError();
    return rc;
  }
  *tby_out = btby;
  *ns_out = bns;
  *ms_out = best;
  return FITRIG_OK;
}

static int tuned_shape(int w, int storage, int* tby, int* ns) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tuned.find({w, storage});
  if (it == g_tuned.end()) {
    float ms = 0.f;
    const int rc = run_autotune(w, storage, tby, ns, &ms);
    if (rc != FITRIG_OK) return rc;
    g_tuned[{w, storage}] = {{*tby, *ns}, ms};
    return FITRIG_OK;
  }
  *tby = it->second.first.first;
  *ns = it->second.first.second;
  return FITRIG_OK;
}

// cudaMalloc that also counts the plan's device bytes (serving admission).
template <typename Ptr>
static cudaError_t dmalloc(fitrig_plan_t p, Ptr** ptr, size_t bytes) {
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
  if (e == cudaSuccess) p->bytes += (int64_t)bytes;
  return e;
}

// Selection lists, the dense map of list indices and the candidate buffers,
// sized by select_capacity(); replaces any earlier ones.
static void drop_graph(fitrig_plan_t p) {
  if (p->graph) cudaGraphExecDestroy(p->graph);
  p->graph = nullptr;
  p->graph_key[0] = p->graph_key[1] = p->graph_key[2] = -1;
}

static int alloc_select(fitrig_plan_t p) {
  ++p->sel_gen;   // the lists move: a captured detect would use the old ones
  drop_graph(p);
  void* old[] = {p->d_sel, p->d_cand, p->d_cand_tmp};
  for (void* q : old)
    if (q) cudaFree(q);
  p->bytes -= p->sel_bytes;
  p->sel_bytes = 0;
  p->d_sel = nullptr;
  p->d_cand = nullptr;
  p->d_cand_tmp = nullptr;
  const int64_t b0 = p->bytes;
  const int U = p->units;
  SelectScratch& s = p->sel;
  s.nblk = 152 * 8;
  s.capacity = select_capacity(p);
  const size_t cap = (size_t)s.capacity;
  size_t bytes = 0;
  auto carve = [&](size_t n) {
    const size_t off = bytes;
    bytes += (n + 255) / 256 * 256;
    return off;
  };
  const size_t o_cnt = carve(sizeof(int) * s.nblk * 8), o_off = carve(sizeof(int) * (s.nblk * 8 + 1));
  const size_t o_items = carve(sizeof(SelItem) * cap), o_nsel = carve(sizeof(int));
  const size_t o_par = carve(sizeof(int) * cap), o_cm = carve(sizeof(unsigned) * cap);
  const size_t o_pk = carve(sizeof(int) * cap);
  const size_t o_pl = carve(sizeof(int) * cap), o_np = carve(sizeof(int));
  // bitmap words over the element space units * vstride (whole 128-element
  // blocks, as the compaction writes them)
  const size_t nwords = ((size_t)std::max<int64_t>(1, (int64_t)U * p->vstride) + 127) / 128 * 4;
  const size_t o_bits = carve(sizeof(uint32_t) * nwords), o_wb = carve(sizeof(int) * nwords);
  CK(dmalloc(p, &p->d_sel, bytes));
  CK(cudaMemset(p->d_sel, 0, bytes));
  char* b = static_cast<char*>(p->d_sel);
  s.blkcnt = reinterpret_cast<int*>(b + o_cnt);
  s.blkoff = reinterpret_cast<int*>(b + o_off);
  s.items = reinterpret_cast<SelItem*>(b + o_items);
  s.nsel = reinterpret_cast<int*>(b + o_nsel);
  s.parent = reinterpret_cast<int*>(b + o_par);
  s.compmax = reinterpret_cast<unsigned*>(b + o_cm);
  s.peak = reinterpret_cast<int*>(b + o_pk);
  s.plist = reinterpret_cast<int*>(b + o_pl);
  s.npeak = reinterpret_cast<int*>(b + o_np);
  s.want = p->d_small + 3;
  s.bits = reinterpret_cast<uint32_t*>(b + o_bits);
  s.wbase = reinterpret_cast<int*>(b + o_wb);
  p->cand_cap = s.capacity;
  CK(dmalloc(p, &p->d_cand, sizeof(fitrig_candidate) * cap));
  CK(dmalloc(p, &p->d_cand_tmp, sizeof(fitrig_candidate) * cap));
  p->sel_bytes = p->bytes - b0;
  return FITRIG_OK;
}

// Twiddle table of the length-n transform (layout chosen by the spectrum
// kernels: spectrum_twiddles), computed in FP64 on the host.
static int make_twiddles(fitrig_plan_t p, int n, float2** out) {
  const std::vector<float2> tw = spectrum_twiddles(n);
  CK(dmalloc(p, out, sizeof(float2) * tw.size()));
  CK(cudaMemcpy(*out, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice));
  return FITRIG_OK;
}

static int allocate(fitrig_plan_t p) {
  if (p->allocated) return FITRIG_OK;
  const int eb = elem_bytes(p->storage);
  const bool delta = p->coding == FITRIG_CODING_DELTA;
  if (delta && (p->storage == FITRIG_F32 || p->stride != FITRIG_STRIDE_TILE || p->accumulate != 1 ||
                p->ring))
    return FITRIG_EUNSUPPORTED;
  p->pitch = ((int64_t)p->nx * eb + 127) / 128 * 128 / eb;
  p->slice_bytes = (size_t)p->pitch * p->ny * eb;
  int boxW, boxH;
  if (p->stride == FITRIG_STRIDE_SLIDING) {
    if (!slide_geometry(p->w, eb, &p->sgeom)) return FITRIG_EUNSUPPORTED;
    p->sgeom.gridX = (p->nx + p->sgeom.OW - 1) / p->sgeom.OW;
    p->sgeom.gridY = (p->ny + p->sgeom.OH - 1) / p->sgeom.OH;
    if (p->sgeom.gridY > 65535) return FITRIG_EUNSUPPORTED;
    boxW = p->sgeom.boxW;
    boxH = p->sgeom.EH;
  } else {
    int tby = 0, ns = 0;
    if (p->autotune && p->w >= 3 && p->w <= 6 &&
        tuned_shape(p->w, p->storage, &tby, &ns) == FITRIG_OK &&
        small_geometry(p->w, eb, tby, ns, &p->geom)) {
      // tuned thread-per-tile shape
    } else if (!stack_geometry(p->w, eb, &p->geom)) {
      return FITRIG_EUNSUPPORTED;
    }
    // the difference-coded march exists for the thread-per-tile and sub-tile
    // paths (windows 3..6, 8, 16, 32, 64)
    if (delta && p->geom.R > 0) return FITRIG_EUNSUPPORTED;
    p->geom.gridX = (p->Tx + p->geom.TBX - 1) / p->geom.TBX;
    p->geom.gridY = (p->Ty + p->geom.TBY - 1) / p->geom.TBY;
    if (p->geom.gridY > 65535) return FITRIG_EUNSUPPORTED;
    boxW = p->geom.boxW;
    boxH = p->geom.BH;
  }
  const int U = p->units;
  p->vstride = (p->T + 3) / 4 * 4;
  CK(dmalloc(p, &p->d_stack, p->slice_bytes * p->L));
  if (delta) {
    p->kpitch = ((int64_t)p->nx + 31) / 32 * 32;
    CK(dmalloc(p, &p->d_key, sizeof(float) * (size_t)p->kpitch * p->ny));
    CK(dmalloc(p, &p->d_dstate, sizeof(float) * (size_t)p->nx * p->ny));
  }
  // with the frequency branch, eta is one more slot after the U units, so that
  // both branches' noise estimates run as one launch over U + 1 groups
  const int vslots = (p->branch & FITRIG_BRANCH_FREQ) ? U + 1 : U;
  CK(dmalloc(p, &p->d_vp, sizeof(float) * (size_t)vslots * p->vstride));
  CK(cudaMemset(p->d_vp, 0xff, sizeof(float) * (size_t)vslots * p->vstride));   // NaN padding
  if (p->branch & FITRIG_BRANCH_FREQ) p->d_eta = p->d_vp + (size_t)U * p->vstride;
  if (p->stride == FITRIG_STRIDE_TILE && p->geom.R == 0)
    CK(dmalloc(p, &p->d_arg, (size_t)U * p->vstride));
  CK(dmalloc(p, &p->d_inv, sizeof(double) * (U + 1)));
  CK(dmalloc(p, &p->d_small, 64));
  CK(dmalloc(p, &p->d_invalid, sizeof(unsigned long long)));
  CK(dmalloc(p, &p->d_cs, sizeof(double) * 2 * (U + 1)));
  CK(dmalloc(p, &p->d_thr, sizeof(float) * (U + 1)));
  const int nblk_img = std::max(1, std::min(1024, (152 * 4 + U - 1) / U));
  const int nblk_freq = 152 * 4;
  // the image branch's estimates (U maps) and eta's (one map) run on two
  // streams at once, so each has its own scratch
  CK(dmalloc(p, &p->d_noise, noise_scratch_bytes(U, nblk_img)));
  noise_scratch_carve(p->d_noise, U, nblk_img, &p->ns_img);
  p->ns_img.invalid = p->d_invalid;
  if (p->noise == FITRIG_NOISE_MEDMAD) {
    const size_t sb = noise_split_bytes(U, p->vstride);
    if (sb > 0) {
      CK(dmalloc(p, &p->d_split, sb));
      noise_split_carve(p->d_split, U, p->vstride, &p->ns_img);
    }
  }
  if (p->branch & FITRIG_BRANCH_FREQ) {
    CK(dmalloc(p, &p->d_noise_f, noise_scratch_bytes(1, nblk_freq)));
    noise_scratch_carve(p->d_noise_f, 1, nblk_freq, &p->ns_freq);
    p->ns_freq.invalid = p->d_invalid;
    if (p->noise == FITRIG_NOISE_MEDMAD) {
      const size_t sb = noise_split_bytes(1, p->vstride);
      if (sb > 0) {
        CK(dmalloc(p, &p->d_split_f, sb));
        noise_split_carve(p->d_split_f, 1, p->vstride, &p->ns_freq);
      }
    }
    CK(dmalloc(p, &p->d_blk_f, block_scratch_bytes(1, p->Tx, p->Ty, p->vstride)));
    block_scratch_carve(p->d_blk_f, 1, p->Tx, p->Ty, p->vstride, &p->blk_f);
    CK(dmalloc(p, &p->d_fpeaks, sizeof(SelItem) * (size_t)std::max<int64_t>(1, p->T)));
  }
  if (p->branch & FITRIG_BRANCH_IMAGE) {
    CK(dmalloc(p, &p->d_blk, block_scratch_bytes(std::max(U, 1), p->Tx, p->Ty, p->vstride)));
    block_scratch_carve(p->d_blk, std::max(U, 1), p->Tx, p->Ty, p->vstride, &p->blk);
  }
  if (!p->side_st) {
    CK(cudaStreamCreateWithFlags(&p->side_st, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming));
  }
  {
    const int rc = alloc_select(p);
    if (rc != FITRIG_OK) return rc;
  }
  if (p->branch & FITRIG_BRANCH_FREQ) {
    CK(dmalloc(p, &p->d_bin, sizeof(int) * p->T));
    const int rc = make_twiddles(p, U, &p->d_tw);
    if (rc != FITRIG_OK) return rc;
  }
  if (p->mmode == FITRIG_MMODE_RUNNING) {
    CK(dmalloc(p, &p->d_smax, sizeof(unsigned) * 2 * p->L));
    CK(dmalloc(p, &p->d_mrun, sizeof(double) * U));
    CK(dmalloc(p, &p->d_wts, sizeof(float) * U));
  }
  CK(cudaMallocHost(&p->h_pinned, 64));
  for (int i = 0; i < 2 * FITRIG_KERNEL_COUNT; ++i)
    if (!p->ev[i]) CK(cudaEventCreate(&p->ev[i]));
  // TMA descriptor over the analysed region of the stack (zero fill outside)
  EncodeTiledFn enc = encode_fn();
  if (!enc) return FITRIG_ECUDA;
  const CUtensorMapDataType dt = p->storage == FITRIG_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : p->storage == FITRIG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                             : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const cuuint64_t dims[3] = {(cuuint64_t)p->nxu, (cuuint64_t)p->nyu, (cuuint64_t)p->L};
  const cuuint64_t strides[2] = {(cuuint64_t)p->pitch * eb, (cuuint64_t)p->slice_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)boxW, (cuuint32_t)boxH, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  if (enc(&p->tmap, dt, 3, p->d_stack, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return FITRIG_ECUDA;
  p->allocated = true;
  return FITRIG_OK;
}

static int ensure_allocated(fitrig_plan_t p) {
  if (p->allocated) return FITRIG_OK;
  const int rc = allocate(p);
  if (rc != FITRIG_OK) free_all(p);
  return rc;
}

extern "C" {

FITRIG_API const char* fitrig_version(void) { return "0.1.0"; }

FITRIG_API const char* fitrig_status_string(int s) {
  switch (s) {
    case FITRIG_OK: return "ok";
    case FITRIG_EINVAL: return "invalid argument";
    case FITRIG_ENOMEM: return "out of memory";
    case FITRIG_ESTATE: return "invalid state";
    case FITRIG_ECUDA: return "CUDA error";
    case FITRIG_ETIMEOUT: return "device wait timed out";
    case FITRIG_ETRUNC: return "output truncated";
    case FITRIG_ENONFINITE: return "non-finite pixels invalidated tiles";
    case FITRIG_EBUSY: return "busy";
    case FITRIG_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

FITRIG_API int fitrig_plan_create(int nx, int ny, int nsnap, int window, double nsigma,
                                  int branch, fitrig_plan_t* out) {
  if (!out) return FITRIG_EINVAL;
  *out = nullptr;
  if (nx < 1 || ny < 1 || window < 1 || window > std::min(nx, ny)) return FITRIG_EINVAL;
  if (branch < FITRIG_BRANCH_IMAGE || branch > FITRIG_BRANCH_BOTH) return FITRIG_EINVAL;
  if (nsnap < 3 || ((branch & FITRIG_BRANCH_FREQ) && nsnap < 4)) return FITRIG_EINVAL;
  if (!(nsigma > 0.0) || !std::isfinite(nsigma)) return FITRIG_EINVAL;
  if (window > 128) return FITRIG_EUNSUPPORTED;
  if ((branch & FITRIG_BRANCH_FREQ) && nsnap - 2 > spectrum_max_n()) return FITRIG_EUNSUPPORTED;
  fitrig_plan_t p = new (std::nothrow) fitrig_plan_s();
  if (!p) return FITRIG_ENOMEM;
  p->nx = nx;
  p->ny = ny;
  p->L = nsnap;
  p->w = window;
  p->tau = nsigma;
  p->branch = branch;
  p->units = nsnap - 2;
  cudaGetDevice(&p->device);
  // a blocking stream: ordered with the legacy default stream, so device
  // snapshots produced there are complete before a push reads them
  if (cudaStreamCreateWithFlags(&p->own_stream, cudaStreamDefault) != cudaSuccess) {
    delete p;
    return FITRIG_ECUDA;
  }
  p->nxu = nx;
  p->nyu = ny;
  p->Tx = (nx + window - 1) / window;
  p->Ty = (ny + window - 1) / window;
  p->T = (int64_t)p->Tx * p->Ty;
  *out = p;
  return FITRIG_OK;
}

FITRIG_API int fitrig_plan_set(fitrig_plan_t p, int option, int64_t value) {
  if (!p) return FITRIG_EINVAL;
  switch (option) {
    case FITRIG_OPT_STREAM:
      p->stream = reinterpret_cast<cudaStream_t>(value);
      return FITRIG_OK;
    case FITRIG_OPT_AUTOTUNE:
      if (p->allocated) return FITRIG_ESTATE;
      p->autotune = value != 0;
      return FITRIG_OK;
    case FITRIG_OPT_MAX_SELECTED: {
      if (value < 0 || value >= INT32_MAX) return FITRIG_EINVAL;
      p->max_selected = value;
      if (!p->allocated) return FITRIG_OK;
      // resize the selection lists now; the pushed stack stays
      CK(cudaSetDevice(p->device));
      CK(cudaStreamSynchronize(plan_stream(p)));
      p->detected = false;
      return alloc_select(p);
    }
    case FITRIG_OPT_TIMEOUT_NS:
      if (value <= 0) return FITRIG_EINVAL;
      p->timeout_ns = (uint64_t)value;
      drop_graph(p);   // the captured kernels carry the old bound
      return FITRIG_OK;
    case FITRIG_OPT_REFINE:
      if (value != FITRIG_REFINE_PARABOLIC && value != FITRIG_REFINE_CUBIC) return FITRIG_EINVAL;
      if (p->refine != (int)value) drop_graph(p);
      p->refine = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_HARMONICS:
      if (value < 1 || value > 32 || (value & (value - 1))) return FITRIG_EINVAL;
      if (p->hmax != (int)value) drop_graph(p);
      p->hmax = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_GRAPH:
      if (value != 0 && value != 1) return FITRIG_EINVAL;
      p->no_graph = value == 0;
      if (p->no_graph) drop_graph(p);
      return FITRIG_OK;
    default:
      break;
  }
  if (p->pushed > 0 || p->allocated) return FITRIG_ESTATE;
  switch (option) {
    case FITRIG_OPT_STORAGE:
      if (value != FITRIG_F32 && value != FITRIG_BF16 && value != FITRIG_F16) return FITRIG_EINVAL;
      p->storage = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_CODING:
      if (value != FITRIG_CODING_VALUE && value != FITRIG_CODING_DELTA) return FITRIG_EINVAL;
      if (p->ring) return FITRIG_EUNSUPPORTED;
      p->coding = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_ACCUMULATE:
      if (value < 1 || value > 1 << 20) return FITRIG_EINVAL;
      if (p->ring) return FITRIG_EUNSUPPORTED;
      p->accumulate = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_NOISE:
      if (value != FITRIG_NOISE_MEANSTD && value != FITRIG_NOISE_MEDMAD) return FITRIG_EINVAL;
      p->noise = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_RMODE:
      if (value != FITRIG_RMODE_ABS && value != FITRIG_RMODE_SIGNED) return FITRIG_EINVAL;
      p->rmode = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_MMODE:
      if (value != FITRIG_MMODE_GLOBAL && value != FITRIG_MMODE_RUNNING) return FITRIG_EINVAL;
      p->mmode = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_STRIDE:
      if (value == FITRIG_STRIDE_TILE) {
        p->stride = FITRIG_STRIDE_TILE;
        p->Tx = (p->nx + p->w - 1) / p->w;
        p->Ty = (p->ny + p->w - 1) / p->w;
      } else if (value == FITRIG_STRIDE_SLIDING) {
        if ((p->w & 1) == 0) return FITRIG_EINVAL;
        if (p->w > 31) return FITRIG_EUNSUPPORTED;
        if (p->edge != FITRIG_EDGE_PARTIAL) return FITRIG_EINVAL;
        p->stride = FITRIG_STRIDE_SLIDING;
        p->Tx = p->nx;
        p->Ty = p->ny;
      } else {
        return FITRIG_EINVAL;
      }
      p->nxu = p->nx;
      p->nyu = p->ny;
      p->T = (int64_t)p->Tx * p->Ty;
      return FITRIG_OK;
    case FITRIG_OPT_EDGE:
      if (p->stride == FITRIG_STRIDE_SLIDING) return FITRIG_EINVAL;
      if (value == FITRIG_EDGE_PARTIAL) {
        p->edge = (int)value;
        p->nxu = p->nx;
        p->nyu = p->ny;
        p->Tx = (p->nx + p->w - 1) / p->w;
        p->Ty = (p->ny + p->w - 1) / p->w;
      } else if (value == FITRIG_EDGE_DROP) {
        p->edge = (int)value;
        p->Tx = p->nx / p->w;
        p->Ty = p->ny / p->w;
        p->nxu = p->Tx * p->w;
        p->nyu = p->Ty * p->w;
      } else {
        return FITRIG_EINVAL;
      }
      p->T = (int64_t)p->Tx * p->Ty;
      return FITRIG_OK;
    default:
      return FITRIG_EINVAL;
  }
}

// Host-to-device copy of ny rows of `width` bytes, ordered on `st`.  Large
// snapshots are split into row bands copied on up to four side streams, so
// that several copy engines move them at once; the bands start after the work
// already on `st` and `st` waits for all of them.  A copy whose rows are
// contiguous on both sides goes as one linear copy per band.
static cudaError_t copy_rows_h2d(fitrig_plan_t p, void* dst, size_t dpitch, const void* src,
                                 size_t spitch, size_t width, int64_t ny, cudaStream_t st) {
  const size_t bytes = width * (size_t)ny;
  const bool linear = dpitch == width && spitch == width;
  int nb = bytes >= ((size_t)32 << 20) ? 4 : 1;
  if (nb > 1 && !p->copy_st[0]) {
    for (int i = 0; i < 4; ++i) {
      cudaError_t e = cudaStreamCreateWithFlags(&p->copy_st[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < 5; ++i) {
      cudaError_t e = cudaEventCreateWithFlags(&p->copy_ev[i], cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
  }
  if (nb == 1) {
    if (linear)
      return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, ny, cudaMemcpyHostToDevice, st);
  }
  cudaError_t e = cudaEventRecord(p->copy_ev[4], st);
  const int64_t band = (ny + nb - 1) / nb;
  for (int i = 0; i < nb && e == cudaSuccess; ++i) {
    const int64_t r0 = i * band, r1 = std::min(ny, r0 + band);
    if (r0 >= r1) break;
    cudaStream_t cs = p->copy_st[i];
    e = cudaStreamWaitEvent(cs, p->copy_ev[4], 0);
    char* d = static_cast<char*>(dst) + (size_t)r0 * dpitch;
    const char* s = static_cast<const char*>(src) + (size_t)r0 * spitch;
    if (e == cudaSuccess)
      e = linear ? cudaMemcpyAsync(d, s, width * (size_t)(r1 - r0), cudaMemcpyHostToDevice, cs)
                 : cudaMemcpy2DAsync(d, dpitch, s, spitch, width, r1 - r0,
                                     cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(p->copy_ev[i], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->copy_ev[i], 0);
  }
  return e;
}

// One snapshot into the next slot; arguments already validated.  With `sync`
// a host push returns only after its copy finished (the caller may then reuse
// the buffer); without it the caller synchronises the plan's stream.
static int push_one(fitrig_plan_t p, const void* data, int dtype, int on_device, int64_t rp,
                    bool sync) {
  cudaStream_t st = plan_stream(p);
  const int eb = elem_bytes(p->storage), ib = elem_bytes(dtype);
  char* dst = p->d_stack + p->slice_bytes * p->pushed;
  if (p->coding == FITRIG_CODING_DELTA && (p->pushed == 0 || dtype != p->storage)) {
    // the key frame, or a snapshot the device coder encodes against its
    // running decoded snapshot (which already-encoded pushes do not advance)
    if (p->pushed > 0 && p->dstate_stale) return FITRIG_ESTATE;
    const void* src = data;
    int64_t sp = rp;
    if (!on_device) {
      if (!p->d_staging) CK(dmalloc(p, &p->d_staging, (size_t)p->nx * p->ny * 4));
      CK(copy_rows_h2d(p, p->d_staging, (size_t)p->nx * ib, data, (size_t)rp * ib,
                       (size_t)p->nx * ib, p->ny, st));
      src = p->d_staging;
      sp = p->nx;
    }
    CK(launch_delta_encode(src, dtype, sp, p->d_dstate, p->d_key, p->kpitch, dst, p->storage,
                           p->pitch, p->pushed == 0, p->ny, p->nx, st));
    if (!on_device && sync) CK(cudaStreamSynchronize(st));
    p->pushed += 1;
    p->detected = false;
    return FITRIG_OK;
  }
  if (p->coding == FITRIG_CODING_DELTA) p->dstate_stale = true;   // already-encoded differences
  if (p->accumulate > 1) {
    // Sec. 3.3.2: K raw snapshots summed (FP32, push order) into one
    const void* src = data;
    int64_t sp = rp;
    if (!on_device) {
      if (!p->d_staging) CK(dmalloc(p, &p->d_staging, (size_t)p->nx * p->ny * 4));
      CK(copy_rows_h2d(p, p->d_staging, (size_t)p->nx * ib, data, (size_t)rp * ib,
                       (size_t)p->nx * ib, p->ny, st));
      src = p->d_staging;
      sp = p->nx;
    }
    if (!p->d_accum) CK(dmalloc(p, &p->d_accum, (size_t)p->nx * p->ny * 4));
    const bool first = p->raw_pushed == 0, last = p->raw_pushed + 1 == p->accumulate;
    CK(launch_accumulate(src, dtype, sp, p->d_accum, first, last, dst, p->storage, p->pitch,
                         p->ny, p->nx, st));
    if (!on_device && sync) CK(cudaStreamSynchronize(st));
    if (!last) {
      p->raw_pushed += 1;
      return FITRIG_OK;
    }
    p->raw_pushed = 0;
    p->pushed += 1;
    p->detected = false;
    return FITRIG_OK;
  }
  if (dtype == p->storage) {
    if (on_device)
      CK(cudaMemcpy2DAsync(dst, p->pitch * eb, data, rp * ib, (size_t)p->nx * ib, p->ny,
                           cudaMemcpyDeviceToDevice, st));
    else
      CK(copy_rows_h2d(p, dst, (size_t)p->pitch * eb, data, (size_t)rp * ib, (size_t)p->nx * ib,
                       p->ny, st));
  } else {
    const void* src = data;
    int64_t sp = rp;
    if (!on_device) {
      if (!p->d_staging) CK(dmalloc(p, &p->d_staging, (size_t)p->nx * p->ny * 4));
      CK(copy_rows_h2d(p, p->d_staging, (size_t)p->nx * ib, data, (size_t)rp * ib,
                       (size_t)p->nx * ib, p->ny, st));
      src = p->d_staging;
      sp = p->nx;
    }
    CK(launch_convert(src, dtype, sp, dst, p->storage, p->pitch, p->ny, p->nx, st));
  }
  if (!on_device && sync) CK(cudaStreamSynchronize(st));
  p->pushed += 1;
  p->detected = false;
  return FITRIG_OK;
}

static int push_args(fitrig_plan_t p, const void* data, int dtype, int64_t row_pitch_elems,
                     int64_t* rp) {
  if (!p || !data) return FITRIG_EINVAL;
  if (dtype != FITRIG_F32 && dtype != FITRIG_BF16 && dtype != FITRIG_F16) return FITRIG_EINVAL;
  *rp = row_pitch_elems ? row_pitch_elems : p->nx;
  if (*rp < p->nx) return FITRIG_EINVAL;
  return FITRIG_OK;
}

FITRIG_API int fitrig_push_snapshot(fitrig_plan_t p, const void* data, int dtype, int on_device,
                                    int64_t row_pitch_elems) {
  int64_t rp = 0;
  int rc = push_args(p, data, dtype, row_pitch_elems, &rp);
  if (rc != FITRIG_OK) return rc;
  if (p->pushed >= p->L) return FITRIG_ESTATE;
  CK(cudaSetDevice(p->device));
  rc = ensure_allocated(p);
  if (rc != FITRIG_OK) return rc;
  return push_one(p, data, dtype, on_device, rp, true);
}

FITRIG_API int fitrig_push_snapshots(fitrig_plan_t p, const void* data, int32_t count, int dtype,
                                     int on_device, int64_t row_pitch_elems,
                                     int64_t snap_stride_elems) {
  int64_t rp = 0;
  int rc = push_args(p, data, dtype, row_pitch_elems, &rp);
  if (rc != FITRIG_OK) return rc;
  if (count < 0) return FITRIG_EINVAL;
  const int64_t ss = snap_stride_elems ? snap_stride_elems : rp * p->ny;
  if (ss < rp * p->ny) return FITRIG_EINVAL;
  // with accumulation every K raw snapshots fill one slot
  const int64_t k = p->accumulate > 1 ? p->accumulate : 1;
  if (p->pushed + (p->raw_pushed + (int64_t)count + k - 1) / k > p->L) return FITRIG_ESTATE;
  if (count == 0) return FITRIG_OK;
  CK(cudaSetDevice(p->device));
  rc = ensure_allocated(p);
  if (rc != FITRIG_OK) return rc;
  cudaStream_t st = plan_stream(p);
  const int eb = elem_bytes(p->storage);
  // (a difference-coded plan takes its first snapshot as the key frame)
  const bool contiguous = !on_device && k == 1 && dtype == p->storage && rp == p->nx &&
                          p->pitch == p->nx && ss == rp * p->ny &&
                          !(p->coding == FITRIG_CODING_DELTA && p->pushed == 0);
  if (contiguous) {
    // host rows and device slots line up: one transfer of count * ny rows
    char* dst = p->d_stack + p->slice_bytes * p->pushed;
    const size_t row = (size_t)p->nx * eb;
    CK(copy_rows_h2d(p, dst, row, data, row, row, (int64_t)count * p->ny, st));
    p->pushed += count;
    p->detected = false;
    if (p->coding == FITRIG_CODING_DELTA) p->dstate_stale = true;
  } else {
    const size_t ib = (size_t)elem_bytes(dtype);
    for (int32_t i = 0; i < count; ++i) {
      rc = push_one(p, static_cast<const char*>(data) + (size_t)ss * ib * i, dtype, on_device,
                    rp, false);
      if (rc != FITRIG_OK) return rc;
    }
  }
  if (!on_device) CK(cudaStreamSynchronize(st));
  return FITRIG_OK;
}

FITRIG_API int fitrig_plan_reset(fitrig_plan_t p) {
  if (!p) return FITRIG_EINVAL;
  p->pushed = 0;
  p->raw_pushed = 0;
  p->dstate_stale = false;
  p->detected = false;
  return FITRIG_OK;
}

// (while a detect is captured into a graph the records are external, so that
// they stay timestamps the host reads)
static void rec(fitrig_plan_t p, int k, int end, cudaStream_t st) {
  if (p->capturing) cudaEventRecordWithFlags(p->ev[2 * k + end], st, cudaEventRecordExternal);
  else cudaEventRecord(p->ev[2 * k + end], st);
}

// The trigger as stream work, in three pieces so that a batch can put the
// stack marches of many plans into one launch and capture everything in one
// CUDA graph: clear (counters), march (a2, or a4 in sliding mode), post
// (a5-a9 and the read-back of the counters).  `timed` records the per-kernel
// events (not used inside graphs).
static cudaError_t enqueue_clear(fitrig_plan_t p, cudaStream_t st) {
  // a serving ring keeps word 0, the running maximum M over every snapshot seen
  cudaError_t e = p->ring ? cudaMemsetAsync(p->d_small + 1, 0, 12, st)
                          : cudaMemsetAsync(p->d_small, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_invalid, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess && p->d_smax)
    e = cudaMemsetAsync(p->d_smax, 0, sizeof(unsigned) * 2 * p->L, st);
  return e;
}

static cudaError_t enqueue_march(fitrig_plan_t p, cudaStream_t st) {
  StackArgs a{};
  a.nx = p->nxu;
  a.ny = p->nyu;
  a.nsnap = p->pushed;
  a.Tx = p->Tx;
  a.Ty = p->Ty;
  a.T = p->T;
  a.vstride = p->vstride;
  a.vp = p->d_vp;
  a.arg = p->d_arg;
  a.zrot = p->zrot;
  a.gmax = p->d_small;
  a.smax = p->d_smax;
  a.status = p->d_small + 1;
  a.timeout_ns = p->timeout_ns;
  a.g = p->geom;
  if (p->coding == FITRIG_CODING_DELTA) {
    a.key = p->d_key;
    a.kpitch = p->kpitch;
  }
  if (p->stride == FITRIG_STRIDE_SLIDING) {
    SlideArgs sa{};
    sa.zrot = p->zrot;
    sa.nx = p->nx;
    sa.ny = p->ny;
    sa.nsnap = p->pushed;
    sa.vstride = p->vstride;
    sa.vp = p->d_vp;
    sa.gmax = p->d_small;
    sa.smax = p->d_smax;
    sa.status = p->d_small + 1;
    sa.timeout_ns = p->timeout_ns;
    sa.g = p->sgeom;
    return launch_slide(&p->tmap, sa, p->storage, p->rmode, st);
  }
  return launch_stack(&p->tmap, a, p->storage, p->rmode, st);
}

#define CKE(expr)                          \
  do {                                     \
    const cudaError_t e_ = (expr);         \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

static cudaError_t enqueue_post(fitrig_plan_t p, cudaStream_t st, bool timed) {
  const int U = p->pushed - 2;
  unsigned* status = p->d_small + 1;
  int* nout = reinterpret_cast<int*>(p->d_small + 2);
  auto mark = [&](int k, int end) {
    if (timed) rec(p, k, end, st);
  };
  CandArgs ca{};
  ca.nx = p->nxu;
  ca.ny = p->nyu;
  ca.w = p->stride == FITRIG_STRIDE_SLIDING ? 1 : p->w;   // pixels are 1 x 1 tiles
  ca.Tx = p->Tx;
  ca.Ty = p->Ty;
  ca.T = p->T;
  ca.stride = p->vstride;
  ca.arg = nullptr;
  ca.stack = p->d_stack;
  ca.storage = p->storage;
  ca.pitch = p->pitch;
  ca.slice = (int64_t)p->pitch * p->ny;
  ca.zrot = p->zrot;
  ca.zmod = p->ring ? p->L : 0;
  if (p->coding == FITRIG_CODING_DELTA) {
    ca.key = p->d_key;
    ca.kpitch = p->kpitch;
  }
  ca.eta = p->d_eta;
  ca.bin = p->d_bin;
  ca.refine = p->refine;
  ca.out = p->d_cand;
  ca.nout = nout;
  ca.cap = p->cand_cap;
  // a serving field's frequency branch runs once its ring of units is full
  const bool freq = (p->branch & FITRIG_BRANCH_FREQ) && (p->hist_n == 0 || p->freq_ready);
  const bool image = (p->branch & FITRIG_BRANCH_IMAGE) != 0;
  // The image branch's noise, thresholds and components need only the tile
  // statistics, so they run on the side stream beside the spectrum and the
  // frequency branch; the two join before the image candidates are written
  // (frequency candidates, snapshot -1, lead the sorted list).
  // with the march's in-tile arg-max, a small window and tile rows of at most
  // 1024 tiles the image candidates come straight from the peak bitmap,
  // already in (snapshot, y, x) order
  const bool rows_emit = image && p->d_arg && ca.w <= 8 && p->Tx <= 1024;
  cudaStream_t is = st;
  if (image && freq) {
    CKE(cudaEventRecord(p->fork_ev, st));
    CKE(cudaStreamWaitEvent(p->side_st, p->fork_ev, 0));
    is = p->side_st;
  }
  if (image) {
    if (timed) rec(p, FITRIG_KERNEL_NOISE, 0, is);
    CKE(launch_noise(p->d_vp, U, p->vstride, p->T, p->noise, p->ns_img, p->d_cs, is));
    CKE(launch_thresholds(p->d_cs, U, p->tau, p->d_thr, p->d_inv, is));
    if (timed) rec(p, FITRIG_KERNEL_NOISE, 1, is);
    if (timed) rec(p, FITRIG_KERNEL_SELECT, 0, is);
    CKE(launch_block_select(p->d_vp, U, p->vstride, p->Tx, p->Ty, p->d_thr, p->blk,
                            rows_emit ? nullptr : p->sel.items, p->sel.capacity, status,
                            p->sel.want, is));
    if (is != st) CKE(cudaEventRecord(p->join_ev, is));
  }
  if (p->d_smax && p->coding == FITRIG_CODING_DELTA) {
    CKE(launch_delta_finite_max(p->d_key, p->kpitch, p->d_stack, p->storage, p->pushed, p->nyu,
                                p->nxu, p->pitch, nullptr, p->d_smax, st));
    CKE(launch_running_norm(nullptr, p->storage, p->pushed, p->nyu, p->nxu, p->pitch, p->d_smax,
                            p->d_mrun, p->d_wts, st));
  } else if (p->d_smax) {
    CKE(launch_running_norm(p->d_stack, p->storage, p->pushed, p->nyu, p->nxu, p->pitch, p->d_smax,
                            p->d_mrun, p->d_wts, st));
  }
  if (freq) {
    mark(FITRIG_KERNEL_SPECTRUM, 0);
    if (p->hist_n > 0)   // the ring in any rotation: |X_k| ignores circular shifts
      CKE(launch_spectrum(p->d_hist, p->hist_n, p->T, p->vstride, p->d_htw, p->d_hwts, p->hmax,
                          p->d_eta, p->d_bin, st));
    else
      CKE(launch_spectrum(p->d_vp, U, p->T, p->vstride, p->d_tw, p->d_wts, p->hmax, p->d_eta,
                          p->d_bin, st));
    mark(FITRIG_KERNEL_SPECTRUM, 1);
    double* cs = p->d_cs + 2 * U;
    CKE(launch_noise(p->d_eta, 1, p->vstride, p->T, p->noise, p->ns_freq, cs, st));
    CKE(launch_thresholds(cs, 1, p->tau, p->d_thr + U, p->d_inv + U, st));
    CKE(launch_block_select(p->d_eta, 1, p->vstride, p->Tx, p->Ty, p->d_thr + U, p->blk_f,
                            p->d_fpeaks, p->T, status, p->sel.want, st));
    ca.branch = FITRIG_BRANCH_FREQ;
    ca.cs = cs;              // eta's estimate (group 0 of its selection)
    ca.inv = p->d_inv + U;
    CKE(launch_emit_peaks(ca, p->d_fpeaks, &p->blk_f.counters[2], nout, p->d_cand_tmp, st));
  }
  if (image) {
    if (is != st) CKE(cudaStreamWaitEvent(st, p->join_ev, 0));
    ca.branch = FITRIG_BRANCH_IMAGE;
    ca.arg = p->d_arg;
    ca.cs = p->d_cs;
    ca.inv = p->d_inv;
    if (rows_emit)
      CKE(launch_emit_rows(ca, p->d_vp, U, p->blk, p->sel.capacity, nout, st));
    else
      CKE(launch_emit_peaks(ca, p->sel.items, &p->blk.counters[2], nout, p->d_cand_tmp, st));
    mark(FITRIG_KERNEL_SELECT, 1);
  }
  CKE(launch_clamp_count(nout, (int)p->cand_cap, status, st));
  CKE(cudaMemcpyAsync(p->h_pinned, p->d_small, 16, cudaMemcpyDeviceToHost, st));
  CKE(cudaMemcpyAsync(p->h_pinned + 4, p->d_invalid, 8, cudaMemcpyDeviceToHost, st));
  return cudaSuccess;
}

// After the stream has passed enqueue_post: record the results on the host.
static int finish_detect(fitrig_plan_t p, int32_t* ncand) {
  const unsigned flags = p->h_pinned[1];
  const int n = (int)p->h_pinned[2];
  unsigned long long invalid;
  memcpy(&invalid, p->h_pinned + 4, 8);
  p->last_ncand = n;
  p->detected = true;
  p->detected_branch = p->branch;
  p->detected_units = p->pushed - 2;
  if (ncand) *ncand = n;
  if (flags & kErrTimeout) return FITRIG_ETIMEOUT;
  if (flags & kErrCapacity) {
    // the selection that did not fit: the capacity it would have needed
    const unsigned want = p->h_pinned[3];
    if (ncand) *ncand = (int32_t)std::min<unsigned>(want, (unsigned)INT32_MAX);
    return FITRIG_ETRUNC;
  }
  if (flags & kErrCcLimit) return FITRIG_ETRUNC;
  if (invalid) return FITRIG_ENONFINITE;
  return FITRIG_OK;
}

// The capacity an overflowing selection of the last detect needed (0 when
// everything fitted).
static int64_t overflow_need(fitrig_plan_t p) {
  return (p->h_pinned[1] & kErrCapacity) ? (int64_t)p->h_pinned[3] : 0;
}

// With the automatic capacity (MAX_SELECTED = 0): grow the selection lists to
// what the last detect needed, with a margin.  The tile statistics of the
// march stay valid, so only the post-processing has to run again.
static int grow_select(fitrig_plan_t p) {
  const int64_t need = overflow_need(p);
  if (need <= 0 || p->max_selected != 0) return FITRIG_ETRUNC;
  const int64_t all = (int64_t)p->units * p->T;
  p->auto_selected = std::min<int64_t>(all, need + need / 4 + (1 << 20));
  return alloc_select(p);
}

// Post-processing again after grow_select (status words and invalid counts
// are cleared; M and the tile statistics are kept).
static int repost(fitrig_plan_t p, cudaStream_t st, int32_t* ncand) {
  CK(cudaMemsetAsync(p->d_small + 1, 0, 12, st));
  CK(cudaMemsetAsync(p->d_invalid, 0, sizeof(unsigned long long), st));
  CK(enqueue_post(p, st, true));
  CK(cudaStreamSynchronize(st));
  return finish_detect(p, ncand);
}

static int detect_ready(fitrig_plan_t p) {
  if (p->pushed < 3) return FITRIG_ESTATE;
  if ((p->branch & FITRIG_BRANCH_FREQ) && p->pushed != p->L) return FITRIG_ESTATE;
  return FITRIG_OK;
}

// The stream work of one detect: clear, march, post-processing and the
// read-back of the status words, with the per-stage events.
static cudaError_t enqueue_detect(fitrig_plan_t p, cudaStream_t st) {
  CKE(enqueue_clear(p, st));
  rec(p, FITRIG_KERNEL_DETECT, 0, st);
  rec(p, FITRIG_KERNEL_STACK, 0, st);
  CKE(enqueue_march(p, st));
  rec(p, FITRIG_KERNEL_STACK, 1, st);
  CKE(enqueue_post(p, st, true));
  rec(p, FITRIG_KERNEL_DETECT, 1, st);
  return cudaSuccess;
}

FITRIG_API int fitrig_detect(fitrig_plan_t p, int32_t* ncand) {
  if (!p || !ncand) return FITRIG_EINVAL;
  *ncand = 0;
  int rc = detect_ready(p);
  if (rc != FITRIG_OK) return rc;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = plan_stream(p);
  // The first detect of a state runs eagerly; the second captures the same
  // stream work into a graph, which this and later detects of that state
  // replay (the launches then cost one graph launch).  Results are the same.
  const int64_t key[3] = {p->pushed, p->zrot, p->sel_gen};
  auto same = [&](const int64_t* k) { return k[0] == key[0] && k[1] == key[1] && k[2] == key[2]; };
  bool replay = false;
  if (!p->no_graph && p->graph && same(p->graph_key)) {
    replay = true;
  } else if (!p->no_graph && same(p->last_key)) {
    drop_graph(p);
    const long long n0 = g_launches.load(std::memory_order_relaxed);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      p->capturing = true;
      const cudaError_t e1 = enqueue_detect(p, st);
      p->capturing = false;
      const cudaError_t e2 = cudaStreamEndCapture(st, &g);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    // launches enqueued while capturing did not run
    const long long n = g_launches.load(std::memory_order_relaxed) - n0;
    g_launches.fetch_sub(n, std::memory_order_relaxed);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      p->graph = nullptr;
      p->no_graph = true;   // eager from now on
    } else {
      p->graph_launches = n;
      for (int i = 0; i < 3; ++i) p->graph_key[i] = key[i];
      replay = true;
    }
  }
  if (replay) {
    CK(cudaGraphLaunch(p->graph, st));
    count_launches((int)p->graph_launches);
  } else {
    CK(enqueue_detect(p, st));
  }
  for (int i = 0; i < 3; ++i) p->last_key[i] = key[i];
  CK(cudaStreamSynchronize(st));
  for (int k = 0; k < FITRIG_KERNEL_COUNT; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev[2 * k], p->ev[2 * k + 1]) == cudaSuccess) p->ms[k] = ms;
    else (void)cudaGetLastError();
  }
  rc = finish_detect(p, ncand);
  if (rc == FITRIG_ETRUNC && overflow_need(p) > 0 && p->max_selected == 0) {
    const int g = grow_select(p);
    if (g != FITRIG_OK) return g;
    rc = repost(p, st, ncand);
  }
  return rc;
}

// ---------------------------------------------------------------- batches
struct fitrig_batch_s {
  std::vector<fitrig_plan_t> plans;   // in work order (largest first)
  std::vector<int> order;             // plans[k] is the caller's plan order[k]
  FieldDesc* d_fields = nullptr;
  unsigned long long* d_counter = nullptr;
  int64_t nitems = 0;
  bool multi = false;                 // one persistent march for every plan
  StackGeom geom{};
  int grid = 0;
  int storage = 0, rmode = 0;
  uint64_t timeout_ns = 0;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
  float last_ms = 0.f;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // the plans' post-march work (noise, selection, candidates) runs on these
  // streams, plan k on post_st[k % npost]: most of its kernels are bound by
  // latency, so several fields' chains overlap on the device
  static constexpr int kMaxPost = 8;
  int npost = 0;
  cudaStream_t post_st[kMaxPost] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kMaxPost] = {};
};

static cudaError_t enqueue_batch(fitrig_batch_t b, cudaStream_t st) {
  for (fitrig_plan_t p : b->plans) CKE(enqueue_clear(p, st));
  if (b->multi) {
    CKE(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), st));
    CKE(launch_stack_multi(b->d_fields, (int)b->plans.size(), b->nitems, b->d_counter, b->geom,
                           b->grid, b->storage, b->rmode, b->timeout_ns, st));
  } else {
    for (fitrig_plan_t p : b->plans) CKE(enqueue_march(p, st));
  }
  if (b->npost <= 1) {
    for (fitrig_plan_t p : b->plans) CKE(enqueue_post(p, st, false));
    return cudaSuccess;
  }
  CKE(cudaEventRecord(b->fork_ev, st));
  for (int k = 0; k < b->npost; ++k) CKE(cudaStreamWaitEvent(b->post_st[k], b->fork_ev, 0));
  for (size_t i = 0; i < b->plans.size(); ++i)
    CKE(enqueue_post(b->plans[i], b->post_st[i % b->npost], false));
  for (int k = 0; k < b->npost; ++k) {
    CKE(cudaEventRecord(b->join_ev[k], b->post_st[k]));
    CKE(cudaStreamWaitEvent(st, b->join_ev[k], 0));
  }
  return cudaSuccess;
}

FITRIG_API int fitrig_candidates(fitrig_plan_t p, fitrig_candidate* out, int32_t cap,
                                 int32_t* n) {
  if (!p || !n || cap < 0 || (cap > 0 && !out)) return FITRIG_EINVAL;
  if (!p->detected) return FITRIG_ESTATE;
  CK(cudaSetDevice(p->device));
  *n = p->last_ncand;
  const int m = std::min(cap, p->last_ncand);
  if (m > 0) {
    cudaStream_t st = plan_stream(p);
    CK(cudaMemcpyAsync(out, p->d_cand, sizeof(fitrig_candidate) * m, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return cap < p->last_ncand ? FITRIG_ETRUNC : FITRIG_OK;
}

static int read_floats(fitrig_plan_t p, const float* src, int64_t count, float* out, int32_t cap) {
  if (cap < count) return FITRIG_ETRUNC;
  cudaStream_t st = plan_stream(p);
  CK(cudaMemcpyAsync(out, src, sizeof(float) * count, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FITRIG_OK;
}

FITRIG_API int fitrig_unit_values(fitrig_plan_t p, int32_t unit, float* out, int32_t cap) {
  if (!p || !out) return FITRIG_EINVAL;
  if (!p->detected) return FITRIG_ESTATE;
  if (unit < 0 || unit >= p->detected_units) return FITRIG_EINVAL;
  CK(cudaSetDevice(p->device));
  return read_floats(p, p->d_vp + (size_t)unit * p->vstride, p->T, out, cap);
}

static int resolve_max(fitrig_plan_t p, double* M) {
  cudaStream_t st = plan_stream(p);
  unsigned key = 0;
  CK(cudaMemcpyAsync(p->h_pinned + 8, p->d_small, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  key = p->h_pinned[8];
  if (key && std::isinf(f32_from_key(key))) {
    // the fused maximum saw +inf: recompute over finite pixels only
    CK(cudaMemsetAsync(p->d_small, 0, 4, st));
    if (p->coding == FITRIG_CODING_DELTA)
      CK(launch_delta_finite_max(p->d_key, p->kpitch, p->d_stack, p->storage, p->pushed, p->nyu,
                                 p->nxu, p->pitch, p->d_small, nullptr, st));
    else
      CK(launch_finite_max(p->d_stack, p->storage, p->pushed, p->nyu, p->nxu, p->pitch,
                           p->d_small, st));
    CK(cudaMemcpyAsync(p->h_pinned + 8, p->d_small, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    key = p->h_pinned[8];
  }
  const double m = key ? (double)f32_from_key(key) : -INFINITY;
  *M = std::max(m, (double)kGuardC);
  return FITRIG_OK;
}

FITRIG_API int fitrig_global_max(fitrig_plan_t p, double* M) {
  if (!p || !M) return FITRIG_EINVAL;
  if (!p->detected) return FITRIG_ESTATE;
  CK(cudaSetDevice(p->device));
  return resolve_max(p, M);
}

FITRIG_API int fitrig_unit_normaliser(fitrig_plan_t p, int32_t unit, double* M) {
  if (!p || !M) return FITRIG_EINVAL;
  if (!p->detected) return FITRIG_ESTATE;
  if (unit < 0 || unit >= p->detected_units) return FITRIG_EINVAL;
  CK(cudaSetDevice(p->device));
  if (!p->d_mrun) return resolve_max(p, M);
  cudaStream_t st = plan_stream(p);
  CK(cudaMemcpyAsync(M, p->d_mrun + unit, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FITRIG_OK;
}

FITRIG_API int fitrig_tlisi(fitrig_plan_t p, int32_t unit, float* out, int32_t cap) {
  if (!p || !out) return FITRIG_EINVAL;
  if (!p->detected) return FITRIG_ESTATE;
  if (unit < 0 || unit >= p->detected_units) return FITRIG_EINVAL;
  if (cap < p->T) return FITRIG_ETRUNC;
  CK(cudaSetDevice(p->device));
  double M;
  int rc = resolve_max(p, &M);
  if (rc != FITRIG_OK) return rc;
  cudaStream_t st = plan_stream(p);
  if (!p->d_report) CK(dmalloc(p, &p->d_report, sizeof(float) * p->T));
  CK(launch_tlisi_from_values(p->d_vp + (size_t)unit * p->vstride, p->T, p->d_small,
                              p->d_mrun ? p->d_mrun + unit : nullptr, p->d_report,
                              st));
  return read_floats(p, p->d_report, p->T, out, cap);
}

FITRIG_API int fitrig_noise_params(fitrig_plan_t p, int32_t unit, double* centre,
                                   double* scale) {
  if (!p || !centre || !scale) return FITRIG_EINVAL;
  if (!p->detected) return FITRIG_ESTATE;
  int slot;
  if (unit == -1) {
    if (!(p->detected_branch & FITRIG_BRANCH_FREQ)) return FITRIG_ESTATE;
    slot = p->detected_units;
  } else {
    if (!(p->detected_branch & FITRIG_BRANCH_IMAGE)) return FITRIG_ESTATE;
    if (unit < 0 || unit >= p->detected_units) return FITRIG_EINVAL;
    slot = unit;
  }
  CK(cudaSetDevice(p->device));
  double v[2];
  cudaStream_t st = plan_stream(p);
  CK(cudaMemcpyAsync(v, p->d_cs + 2 * slot, sizeof(v), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *centre = v[0];
  *scale = v[1];
  return FITRIG_OK;
}

FITRIG_API int fitrig_spectrum(fitrig_plan_t p, float* eta, int32_t* bin, int32_t cap) {
  if (!p) return FITRIG_EINVAL;
  if (!p->detected || !(p->detected_branch & FITRIG_BRANCH_FREQ)) return FITRIG_ESTATE;
  if (cap < p->T) return FITRIG_ETRUNC;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = plan_stream(p);
  if (eta) CK(cudaMemcpyAsync(eta, p->d_eta, sizeof(float) * p->T, cudaMemcpyDeviceToHost, st));
  if (bin) CK(cudaMemcpyAsync(bin, p->d_bin, sizeof(int) * p->T, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FITRIG_OK;
}

FITRIG_API int fitrig_tile_grid(fitrig_plan_t p, int32_t* ty, int32_t* tx) {
  if (!p || !ty || !tx) return FITRIG_EINVAL;
  *ty = p->Ty;
  *tx = p->Tx;
  return FITRIG_OK;
}

FITRIG_API int fitrig_kernel_ms(fitrig_plan_t p, int kernel, float* ms) {
  if (!p || !ms || kernel < 0 || kernel >= FITRIG_KERNEL_COUNT) return FITRIG_EINVAL;
  if (!p->detected) return FITRIG_ESTATE;
  *ms = p->ms[kernel];
  return FITRIG_OK;
}

FITRIG_API int fitrig_stack_device_ptr(fitrig_plan_t p, int32_t s, void** ptr,
                                       int64_t* row_pitch_elems) {
  if (!p || !ptr || !row_pitch_elems || s < 0 || s >= p->L) return FITRIG_EINVAL;
  CK(cudaSetDevice(p->device));
  int rc = ensure_allocated(p);
  if (rc != FITRIG_OK) return rc;
  if (s == 0 && p->coding == FITRIG_CODING_DELTA) {   // the FP32 key frame
    *ptr = p->d_key;
    *row_pitch_elems = p->kpitch;
    return FITRIG_OK;
  }
  *ptr = p->d_stack + p->slice_bytes * s;
  *row_pitch_elems = p->pitch;
  return FITRIG_OK;
}

FITRIG_API int fitrig_spectrum_map(const float* dev_cube, int32_t n, int64_t T, int64_t stride,
                                   int32_t harmonics, float* dev_eta, int32_t* dev_bin,
                                   int32_t method, int64_t stream, float* ms) {
  if (!dev_cube || !dev_eta || !dev_bin || T < 1 || stride < T) return FITRIG_EINVAL;
  if (n < 2 || n > spectrum_max_n()) return FITRIG_EINVAL;
  if (harmonics < 1 || harmonics > 32 || (harmonics & (harmonics - 1))) return FITRIG_EINVAL;
  if (method < FITRIG_SPECTRUM_AUTO || method > FITRIG_SPECTRUM_RADIX) return FITRIG_EINVAL;
  const bool pow2 = n >= 128 && (n & (n - 1)) == 0;
  if (method == FITRIG_SPECTRUM_RADIX && !pow2) return FITRIG_EUNSUPPORTED;
  if (T > (int64_t)UINT32_MAX) return FITRIG_EUNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const std::vector<float2> tw = spectrum_twiddles(n);
  float2* d_tw = nullptr;
  CK(cudaMalloc(&d_tw, sizeof(float2) * tw.size()));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemcpyAsync(d_tw, tw.data(), sizeof(float2) * tw.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    const int m = method == FITRIG_SPECTRUM_DIRECT ? kSpectrumDirect
                  : method == FITRIG_SPECTRUM_RADIX ? kSpectrumRadix : kSpectrumAuto;
    if (method == FITRIG_SPECTRUM_DIRECT && !pow2)   // the table is already the direct kernels'
      e = launch_spectrum(dev_cube, n, T, stride, d_tw, nullptr, harmonics, dev_eta, dev_bin, st);
    else
      e = launch_spectrum_method(dev_cube, n, T, stride, d_tw, nullptr, harmonics, dev_eta,
                                 dev_bin, m, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_tw);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return FITRIG_ECUDA;
  }
  if (ms) *ms = t;
  return FITRIG_OK;
}

FITRIG_API int fitrig_threshold_map(const float* dev_map, int64_t n, double nsigma,
                                    int noise_mode, int64_t stream, int64_t* nexceed,
                                    double* centre, double* scale) {
  if (!dev_map || n < 1 || !nexceed || !(nsigma > 0.0)) return FITRIG_EINVAL;
  if (noise_mode != FITRIG_NOISE_MEANSTD && noise_mode != FITRIG_NOISE_MEDMAD) return FITRIG_EINVAL;
  if (n > (int64_t)INT32_MAX) return FITRIG_EUNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nblk = 152 * 4;
  void* scratch = nullptr;
  const size_t nb = (noise_scratch_bytes(1, nblk) + 255) / 256 * 256;   // keeps the tail 8-byte aligned
  const size_t extra = 256 + sizeof(int) * (nblk * 8 + 2) + sizeof(long long) * 2 + 64;
  const size_t ntail = (extra + 255) / 256 * 256;
  const size_t nsplit = noise_mode == FITRIG_NOISE_MEDMAD ? noise_split_bytes(1, n) : 0;
  CK(cudaMalloc(&scratch, nb + ntail + nsplit));
  NoiseScratch ns;
  noise_scratch_carve(scratch, 1, nblk, &ns);
  if (nsplit) noise_split_carve(static_cast<char*>(scratch) + nb + ntail, 1, n, &ns);
  char* tail = static_cast<char*>(scratch) + nb;
  double* cs = reinterpret_cast<double*>(tail);
  float* thr = reinterpret_cast<float*>(tail + 16);
  unsigned long long* inval = reinterpret_cast<unsigned long long*>(tail + 32);
  long long* total = reinterpret_cast<long long*>(tail + 48);
  double* inv = reinterpret_cast<double*>(tail + 56);
  int* blkcnt = reinterpret_cast<int*>(tail + 64);
  ns.invalid = inval;
  int rc = FITRIG_OK;
  double h[2] = {0, 0};
  long long cnt = 0;
  cudaError_t e = cudaMemsetAsync(inval, 0, 8, st);
  if (e == cudaSuccess) e = launch_noise(dev_map, 1, n, n, noise_mode, ns, cs, st);
  if (e == cudaSuccess) e = launch_thresholds(cs, 1, nsigma, thr, inv, st);
  if (e == cudaSuccess) e = launch_count_selected(dev_map, 1, n, thr, nblk, blkcnt, total, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, cs, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, total, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    rc = FITRIG_ECUDA;
  }
  cudaFree(scratch);
  if (rc != FITRIG_OK) return rc;
  *nexceed = cnt;
  if (centre) *centre = h[0];
  if (scale) *scale = h[1];
  return FITRIG_OK;
}

FITRIG_API int fitrig_autotune(int window, int storage, int32_t* tile_rows, int32_t* stages,
                               float* best_ms) {
  if (!tile_rows || !stages || !best_ms) return FITRIG_EINVAL;
  if (storage != FITRIG_F32 && storage != FITRIG_BF16 && storage != FITRIG_F16) return FITRIG_EINVAL;
  if (window < 3 || window > 6) return FITRIG_EUNSUPPORTED;
  int tby = 0, ns = 0;
  const int rc = tuned_shape(window, storage, &tby, &ns);
  if (rc != FITRIG_OK) return rc;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  *tile_rows = tby;
  *stages = ns;
  *best_ms = g_tuned[{window, storage}].second;
  return FITRIG_OK;
}

FITRIG_API int fitrig_batch_create(const fitrig_plan_t* plans, int32_t nplans,
                                   fitrig_batch_t* out) {
  if (!plans || nplans < 1 || !out) return FITRIG_EINVAL;
  *out = nullptr;
  fitrig_plan_t p0 = plans[0];
  for (int i = 0; i < nplans; ++i) {
    fitrig_plan_t p = plans[i];
    if (!p) return FITRIG_EINVAL;
    for (int j = 0; j < i; ++j)
      if (plans[j] == p) return FITRIG_EINVAL;   // a plan may appear once
    const int rc = detect_ready(p);
    if (rc != FITRIG_OK) return rc;
    if (!p->allocated || p->device != p0->device) return FITRIG_ESTATE;
  }
  fitrig_batch_t b = new (std::nothrow) fitrig_batch_s();
  if (!b) return FITRIG_ENOMEM;
  b->device = p0->device;
  b->stream = plan_stream(p0);
  b->storage = p0->storage;
  b->rmode = p0->rmode;
  b->timeout_ns = p0->timeout_ns;
  // largest fields first, so the persistent march ends evenly
  std::vector<int> idx(nplans);
  for (int i = 0; i < nplans; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    return (double)plans[x]->pushed * plans[x]->T > (double)plans[y]->pushed * plans[y]->T;
  });
  for (int i : idx) {
    b->plans.push_back(plans[i]);
    b->order.push_back(i);
  }
  // one persistent launch needs the same thread-per-tile march for all (and
  // plain stored values: difference-coded plans march one by one)
  b->multi = true;
  for (fitrig_plan_t p : b->plans)
    if (p->stride != FITRIG_STRIDE_TILE || p->geom.R != 0 || p->w != p0->w ||
        p->coding != FITRIG_CODING_VALUE ||
        p->storage != p0->storage || p->rmode != p0->rmode || p->geom.TBY != p0->geom.TBY ||
        p->geom.stages != p0->geom.stages)
      b->multi = false;
  cudaSetDevice(b->device);
  if (b->multi) {
    b->geom = p0->geom;
    std::vector<FieldDesc> fd(b->plans.size());
    int64_t items = 0;
    for (size_t k = 0; k < b->plans.size(); ++k) {
      fitrig_plan_t p = b->plans[k];
      FieldDesc& d = fd[k];
      memset(&d, 0, sizeof(d));
      d.tmap = p->tmap;
      d.zrot = 0;
      d.vp = p->d_vp;
      d.arg = p->d_arg;
      d.gmax = p->d_small;
      d.smax = p->d_smax;
      d.status = p->d_small + 1;
      d.nx = p->nxu;
      d.ny = p->nyu;
      d.L = p->pushed;
      d.Tx = p->Tx;
      d.Ty = p->Ty;
      d.gridX = p->geom.gridX;
      d.vstride = p->vstride;
      d.item0 = items;
      items += (int64_t)p->geom.gridX * p->geom.gridY;
    }
    b->nitems = items;
    const int per_sm = multi_blocks_per_sm(b->geom, b->storage, b->rmode);
    b->grid = 152 * std::max(1, per_sm);
    if (cudaMalloc(&b->d_fields, sizeof(FieldDesc) * fd.size()) != cudaSuccess ||
        cudaMalloc(&b->d_counter, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemcpy(b->d_fields, fd.data(), sizeof(FieldDesc) * fd.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      (void)cudaGetLastError();
      fitrig_batch_destroy(b);
      return FITRIG_ENOMEM;
    }
  }
  if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) {
    (void)cudaGetLastError();
    fitrig_batch_destroy(b);
    return FITRIG_ECUDA;
  }
  b->npost = (int)std::min<size_t>(b->plans.size(), fitrig_batch_s::kMaxPost);
  if (b->npost > 1) {
    bool ok = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < b->npost; ++k)
      ok = cudaStreamCreateWithFlags(&b->post_st[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      (void)cudaGetLastError();
      fitrig_batch_destroy(b);
      return FITRIG_ECUDA;
    }
  }
  *out = b;
  return FITRIG_OK;
}

FITRIG_API int fitrig_batch_detect(fitrig_batch_t b, int32_t* ncand) {
  if (!b || !ncand) return FITRIG_EINVAL;
  CK(cudaSetDevice(b->device));
  cudaStream_t st = b->stream;
  for (fitrig_plan_t p : b->plans) {
    const int rc = detect_ready(p);
    if (rc != FITRIG_OK) return rc;
  }
  if (!b->exec) {
    // one eager pass (sets kernel attributes, checks every launch and sizes
    // the selection lists), then capture the same stream work once
    CK(enqueue_batch(b, st));
    CK(cudaStreamSynchronize(st));
    for (fitrig_plan_t p : b->plans) {
      if (overflow_need(p) > 0 && p->max_selected == 0) {
        const int g = grow_select(p);
        if (g != FITRIG_OK) return g;
      }
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = enqueue_batch(b, st);
    const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      (void)cudaGetLastError();
      return FITRIG_ECUDA;
    }
    const cudaError_t e3 = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
      b->exec = nullptr;
      (void)cudaGetLastError();
      return FITRIG_ECUDA;
    }
  }
  CK(cudaEventRecord(b->ev0, st));
  CK(cudaGraphLaunch(b->exec, st));
  CK(cudaEventRecord(b->ev1, st));
  CK(cudaStreamSynchronize(st));
  cudaEventElapsedTime(&b->last_ms, b->ev0, b->ev1);
  int worst = FITRIG_OK;
  for (size_t k = 0; k < b->plans.size(); ++k) {
    fitrig_plan_t p = b->plans[k];
    int32_t n = 0;
    int rc = finish_detect(p, &n);
    if (rc == FITRIG_ETRUNC && overflow_need(p) > 0 && p->max_selected == 0) {
      // more selected tiles than on the first run: grow, finish this plan
      // eagerly, and capture the graph again on the next call
      const int g = grow_select(p);
      if (g != FITRIG_OK) return g;
      rc = repost(p, st, &n);
      if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
    }
    ncand[b->order[k]] = n;
    if (rc != FITRIG_OK && (worst == FITRIG_OK || worst == FITRIG_ENONFINITE)) worst = rc;
  }
  return worst;
}

FITRIG_API int fitrig_batch_ms(fitrig_batch_t b, float* ms) {
  if (!b || !ms) return FITRIG_EINVAL;
  *ms = b->last_ms;
  return FITRIG_OK;
}

FITRIG_API int fitrig_batch_destroy(fitrig_batch_t b) {
  if (!b) return FITRIG_EINVAL;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->d_fields) cudaFree(b->d_fields);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  for (int k = 0; k < fitrig_batch_s::kMaxPost; ++k) {
    if (b->post_st[k]) cudaStreamSynchronize(b->post_st[k]);
    if (b->post_st[k]) cudaStreamDestroy(b->post_st[k]);
    if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
  }
  delete b;
  return FITRIG_OK;
}

// ---------------------------------------------------------------- serving
// A server owns fields that stream snapshots.  Each active field is a plan
// whose stack is a ring of three slots: the latest three snapshots stay on the
// device, and every arriving snapshot completes one unit, whose trigger runs
// on the field's own stream right away.  Fields overlap on the GPU through
// their streams; admission reserves each field's device bytes against the
// budget, and fields that do not fit wait in FIFO order until retirements free
// enough memory.  Results are collected in stream order by a host callback
// that stamps the completion time.
namespace {

int64_t monotonic_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

enum { kFieldQueued = 0, kFieldActive = 1, kFieldRetired = 2 };

struct ServerField {
  int id = 0;
  int state = kFieldQueued;
  int nx = 0, ny = 0, w = 0, storage = 0, noise = 0;
  int nwin = 0;                     // frequency-branch window in units (0: image only)
  double tau = 0.0;
  fitrig_plan_t plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t copied = nullptr;
  int64_t received = 0;             // snapshots pushed so far
  int64_t bytes = 0;                // device bytes reserved
  fitrig_candidate* h_cands = nullptr;   // mapped pinned host buffer
  fitrig_candidate* d_cands = nullptr;   // its device alias
  int32_t cand_cap = 0;
  // GPU timestamps of the current unit (mapped, after the candidates): the
  // copy's start and end and the trigger's end; the unit's callback reads
  // them before the next unit's stamps run (stream order)
  long long* h_stamps = nullptr;
  long long* d_stamps = nullptr;
};

struct ServerResult {
  fitrig_result r;
  std::vector<fitrig_candidate> cands;
};

}  // namespace

struct fitrig_server_s {
  int64_t budget = 0, used = 0;
  int max_fields = 0;
  int device = 0;
  std::mutex mtx;                     // fields, admission, enqueue
  std::vector<ServerField*> fields;   // index = field id
  std::deque<int> waiting;            // FIFO of queued field ids
  int active = 0;
  std::mutex rmtx;                    // results only (never held across CUDA calls)
  std::deque<ServerResult> results;
};

namespace {

struct UnitTicket {
  fitrig_server_s* srv;
  ServerField* f;
  int32_t unit;
  int64_t t_arrival;
  int64_t t_push;
  int64_t t_enqueued;
};

constexpr int32_t kServeCandCap = 1 << 16;

// Host callback, in stream order after a unit's trigger and export.
void CUDART_CB unit_done(void* arg) {
  UnitTicket* t = static_cast<UnitTicket*>(arg);
  ServerField* f = t->f;
  fitrig_plan_t p = f->plan;
  ServerResult res;
  res.r.field = f->id;
  res.r.unit = t->unit;
  const unsigned flags = p->h_pinned[1];
  const int n = (int)p->h_pinned[2];
  unsigned long long invalid;
  memcpy(&invalid, p->h_pinned + 4, 8);
  res.r.ncand = n;
  res.r.status = (flags & kErrTimeout) ? FITRIG_ETIMEOUT
                 : (flags & (kErrCapacity | kErrCcLimit)) || n > f->cand_cap ? FITRIG_ETRUNC
                 : invalid ? FITRIG_ENONFINITE : FITRIG_OK;
  const int m = std::min(n, f->cand_cap);
  res.cands.assign(f->h_cands, f->h_cands + m);
  for (auto& c : res.cands) c.snapshot = t->unit;   // absolute unit index
  res.r.ncand = m;
  res.r.t_arrival_ns = t->t_arrival;
  res.r.t_done_ns = monotonic_ns();
  res.r.cand_offset = 0;
  res.r.t_push_ns = t->t_push;
  res.r.t_enqueued_ns = t->t_enqueued;
  const volatile long long* gs = f->h_stamps;
  res.r.copy_ms = (float)((double)(gs[1] - gs[0]) * 1e-6);
  res.r.trigger_ms = (float)((double)(gs[2] - gs[1]) * 1e-6);
  {
    std::lock_guard<std::mutex> lk(t->srv->rmtx);
    t->srv->results.push_back(std::move(res));
  }
  delete t;
}

void free_field(ServerField* f) {
  if (f->plan) fitrig_plan_destroy(f->plan);
  f->plan = nullptr;
  if (f->h_cands) cudaFreeHost(f->h_cands);
  f->h_cands = nullptr;
  if (f->copied) cudaEventDestroy(f->copied);
  f->copied = nullptr;
}

// Creates the field's plan and buffers; FITRIG_EBUSY if it does not fit.
int activate(fitrig_server_s* s, ServerField* f) {
  fitrig_plan_t p = nullptr;
  int rc = fitrig_plan_create(f->nx, f->ny, 3, f->w, f->tau, FITRIG_BRANCH_IMAGE, &p);
  if (rc != FITRIG_OK) return rc;
  if ((rc = fitrig_plan_set(p, FITRIG_OPT_STORAGE, f->storage)) != FITRIG_OK ||
      (rc = fitrig_plan_set(p, FITRIG_OPT_NOISE, f->noise)) != FITRIG_OK) {
    fitrig_plan_destroy(p);
    return rc;
  }
  p->ring = true;
  if (f->nwin > 0) p->branch = FITRIG_BRANCH_BOTH;   // eta takes the slot after the unit
  rc = ensure_allocated(p);
  if (rc == FITRIG_OK && f->nwin > 0) {
    if (cudaMalloc(&p->d_hist, sizeof(float) * (size_t)f->nwin * p->vstride) != cudaSuccess ||
        cudaMalloc(&p->d_hwts, sizeof(float) * f->nwin) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = FITRIG_ENOMEM;
    } else {
      p->bytes += (int64_t)(sizeof(float) * ((size_t)f->nwin * p->vstride + f->nwin));
      rc = make_twiddles(p, f->nwin, &p->d_htw);
      p->hist_n = f->nwin;
    }
  }
  const int64_t need = p->bytes;
  if (rc != FITRIG_OK || s->used + need > s->budget) {
    fitrig_plan_destroy(p);
    return rc != FITRIG_OK && rc != FITRIG_ENOMEM ? rc : FITRIG_EBUSY;
  }
  f->plan = p;
  f->stream = plan_stream(p);
  f->cand_cap = kServeCandCap;
  if (cudaHostAlloc(&f->h_cands, sizeof(fitrig_candidate) * f->cand_cap + 64, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&f->d_cands, f->h_cands, 0) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->copied, cudaEventDisableTiming) != cudaSuccess ||
      cudaMemsetAsync(p->d_small, 0, 16, f->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    free_field(f);
    return FITRIG_ENOMEM;
  }
  f->h_stamps = reinterpret_cast<long long*>(f->h_cands + f->cand_cap);
  f->d_stamps = reinterpret_cast<long long*>(f->d_cands + f->cand_cap);
  f->bytes = need;
  s->used += need;
  f->state = kFieldActive;
  ++s->active;
  return FITRIG_OK;
}

// Activates waiting fields in FIFO order while they fit.
void admit_waiting(fitrig_server_s* s) {
  while (!s->waiting.empty() && s->active < s->max_fields) {
    ServerField* f = s->fields[s->waiting.front()];
    if (activate(s, f) != FITRIG_OK) break;
    s->waiting.pop_front();
  }
}

}  // namespace

FITRIG_API int fitrig_server_create(int64_t hbm_budget_bytes, int max_fields, fitrig_server_t* out) {
  if (!out || hbm_budget_bytes <= 0 || max_fields < 1) return FITRIG_EINVAL;
  *out = nullptr;
  fitrig_server_t s = new (std::nothrow) fitrig_server_s();
  if (!s) return FITRIG_ENOMEM;
  s->budget = hbm_budget_bytes;
  s->max_fields = max_fields;
  cudaGetDevice(&s->device);
  *out = s;
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_admit(fitrig_server_t s, int nx, int ny, int window, double nsigma,
                                   int storage, int noise, int32_t* field_id) {
  if (!s || !field_id) return FITRIG_EINVAL;
  if (nx < 1 || ny < 1 || window < 1 || window > std::min(nx, ny) || !(nsigma > 0.0)) return FITRIG_EINVAL;
  if (storage != FITRIG_F32 && storage != FITRIG_BF16 && storage != FITRIG_F16) return FITRIG_EINVAL;
  if (noise != FITRIG_NOISE_MEANSTD && noise != FITRIG_NOISE_MEDMAD) return FITRIG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mtx);
  CK(cudaSetDevice(s->device));
  ServerField* f = new (std::nothrow) ServerField();
  if (!f) return FITRIG_ENOMEM;
  f->id = (int)s->fields.size();
  f->nx = nx;
  f->ny = ny;
  f->w = window;
  f->tau = nsigma;
  f->storage = storage;
  f->noise = noise;
  s->fields.push_back(f);
  *field_id = f->id;
  int rc = FITRIG_EBUSY;
  if (s->waiting.empty() && s->active < s->max_fields) rc = activate(s, f);
  if (rc == FITRIG_EBUSY) {
    s->waiting.push_back(f->id);
    return FITRIG_EBUSY;   // queued: becomes active when memory frees
  }
  if (rc != FITRIG_OK) {
    f->state = kFieldRetired;
    return rc;
  }
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_admit_freq(fitrig_server_t s, int nx, int ny, int window,
                                        double nsigma, int storage, int noise, int freq_units,
                                        int32_t* field_id) {
  if (!s || !field_id) return FITRIG_EINVAL;
  if (freq_units < 2) return FITRIG_EINVAL;
  if (freq_units > 256) return FITRIG_EUNSUPPORTED;
  if (nx < 1 || ny < 1 || window < 1 || window > std::min(nx, ny) || !(nsigma > 0.0)) return FITRIG_EINVAL;
  if (storage != FITRIG_F32 && storage != FITRIG_BF16 && storage != FITRIG_F16) return FITRIG_EINVAL;
  if (noise != FITRIG_NOISE_MEANSTD && noise != FITRIG_NOISE_MEDMAD) return FITRIG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mtx);
  CK(cudaSetDevice(s->device));
  ServerField* f = new (std::nothrow) ServerField();
  if (!f) return FITRIG_ENOMEM;
  f->id = (int)s->fields.size();
  f->nx = nx;
  f->ny = ny;
  f->w = window;
  f->tau = nsigma;
  f->storage = storage;
  f->noise = noise;
  f->nwin = freq_units;
  s->fields.push_back(f);
  *field_id = f->id;
  int rc = FITRIG_EBUSY;
  if (s->waiting.empty() && s->active < s->max_fields) rc = activate(s, f);
  if (rc == FITRIG_EBUSY) {
    s->waiting.push_back(f->id);
    return FITRIG_EBUSY;
  }
  if (rc != FITRIG_OK) {
    f->state = kFieldRetired;
    return rc;
  }
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_field_state(fitrig_server_t s, int32_t field, int32_t* state) {
  if (!s || !state) return FITRIG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mtx);
  if (field < 0 || field >= (int)s->fields.size()) return FITRIG_EINVAL;
  *state = s->fields[field]->state;
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_push(fitrig_server_t s, int32_t field, const void* data, int dtype,
                                  int64_t t_arrival_ns) {
  if (!s || !data) return FITRIG_EINVAL;
  if (dtype != FITRIG_F32 && dtype != FITRIG_BF16 && dtype != FITRIG_F16) return FITRIG_EINVAL;
  const int64_t t_push = monotonic_ns();
  cudaEvent_t copied = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mtx);
    if (field < 0 || field >= (int)s->fields.size()) return FITRIG_EINVAL;
    ServerField* f = s->fields[field];
    if (f->state == kFieldQueued) return FITRIG_EBUSY;
    if (f->state != kFieldActive) return FITRIG_ESTATE;
    CK(cudaSetDevice(s->device));
    fitrig_plan_t p = f->plan;
    cudaStream_t st = f->stream;
    const int slot = (int)(f->received % 3);
    const int eb = elem_bytes(p->storage), ib = elem_bytes(dtype);
    char* dst = p->d_stack + p->slice_bytes * slot;
    const bool unit = f->received + 1 >= 3;   // this snapshot completes a unit
    if (unit) CK(launch_stamp(f->d_stamps + 0, st));
    if (dtype == p->storage) {
      CK(cudaMemcpy2DAsync(dst, p->pitch * eb, data, (size_t)p->nx * ib, (size_t)p->nx * ib, p->ny,
                           cudaMemcpyDefault, st));
    } else {
      if (!p->d_staging) CK(dmalloc(p, &p->d_staging, (size_t)p->nx * p->ny * 4));
      CK(cudaMemcpyAsync(p->d_staging, data, (size_t)p->nx * p->ny * ib, cudaMemcpyDefault, st));
      CK(launch_convert(p->d_staging, dtype, p->nx, dst, p->storage, p->pitch, p->ny, p->nx, st));
    }
    if (unit) CK(launch_stamp(f->d_stamps + 1, st));
    CK(cudaEventRecord(f->copied, st));
    copied = f->copied;
    f->received += 1;
    if (f->received >= 3) {
      // the unit whose last snapshot just arrived
      p->pushed = 3;
      p->zrot = (int)((f->received - 3) % 3);
      CK(enqueue_clear(p, st));
      CK(enqueue_march(p, st));
      if (p->hist_n > 0) {
        // the unit's tile statistics and weight into the ring of the last hist_n
        const int64_t slot = p->hist_units % p->hist_n;
        CK(cudaMemcpyAsync(p->d_hist + slot * p->vstride, p->d_vp, sizeof(float) * p->vstride,
                           cudaMemcpyDeviceToDevice, st));
        CK(launch_unit_weight(p->d_small, p->d_hwts + slot, st));
        p->hist_units += 1;
        p->freq_ready = p->hist_units >= p->hist_n;
      }
      CK(enqueue_post(p, st, false));
      CK(launch_export_candidates(p->d_cand, reinterpret_cast<int*>(p->d_small + 2), f->d_cands,
                                  f->cand_cap, st));
      CK(launch_stamp(f->d_stamps + 2, st));
      UnitTicket* t = new (std::nothrow)
          UnitTicket{s, f, (int32_t)(f->received - 3), t_arrival_ns, t_push, monotonic_ns()};
      if (!t) return FITRIG_ENOMEM;
      CK(cudaLaunchHostFunc(st, unit_done, t));
    }
  }
  // the caller's buffer is free once the copy is done
  CK(cudaEventSynchronize(copied));
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_poll(fitrig_server_t s, fitrig_result* out, int32_t cap,
                                  fitrig_candidate* cands, int32_t cand_cap, int32_t* n,
                                  int32_t* ncands) {
  if (!s || !n || !ncands || cap < 0 || cand_cap < 0) return FITRIG_EINVAL;
  *n = 0;
  *ncands = 0;
  std::lock_guard<std::mutex> lk(s->rmtx);
  int32_t k = 0, c = 0;
  while (!s->results.empty() && k < cap) {
    ServerResult& r = s->results.front();
    if (c + (int32_t)r.cands.size() > cand_cap) break;
    r.r.cand_offset = c;
    out[k++] = r.r;
    if (!r.cands.empty()) memcpy(cands + c, r.cands.data(), sizeof(fitrig_candidate) * r.cands.size());
    c += (int32_t)r.cands.size();
    s->results.pop_front();
  }
  *n = k;
  *ncands = c;
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_drain(fitrig_server_t s) {
  if (!s) return FITRIG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mtx);
  for (ServerField* f : s->fields)
    if (f->state == kFieldActive) CK(cudaStreamSynchronize(f->stream));
  return FITRIG_OK;
}

// ---- checkpoint / resume of a serving field
namespace {
struct FieldImage {            // header of an exported field (host byte order)
  char magic[8];               // "FITRIGF1"
  int32_t nx, ny, w, storage, noise, nwin;
  double tau;
  int64_t received, hist_units;
  uint32_t gmax_key, nsnaps;   // running-maximum key; snapshots that follow (0..2)
  int64_t slice_bytes, hist_bytes;
};
constexpr char kFieldMagic[8] = {'F', 'I', 'T', 'R', 'I', 'G', 'F', '1'};

int64_t field_image_bytes(const ServerField* f, const fitrig_plan_t p) {
  const int64_t ns = std::min<int64_t>(2, f->received);
  const int64_t hist = p->hist_n ? (int64_t)sizeof(float) * ((int64_t)p->hist_n * p->vstride + p->hist_n) : 0;
  return (int64_t)sizeof(FieldImage) + ns * (int64_t)p->slice_bytes + hist;
}
}  // namespace

FITRIG_API int fitrig_server_field_export(fitrig_server_t s, int32_t field, void* out, int64_t cap,
                                          int64_t* size) {
  if (!s || !size) return FITRIG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mtx);
  if (field < 0 || field >= (int)s->fields.size()) return FITRIG_EINVAL;
  ServerField* f = s->fields[field];
  if (f->state != kFieldActive) return FITRIG_ESTATE;
  fitrig_plan_t p = f->plan;
  *size = field_image_bytes(f, p);
  if (!out || cap < *size) return FITRIG_ETRUNC;
  CK(cudaSetDevice(s->device));
  CK(cudaStreamSynchronize(f->stream));   // every pushed unit is complete
  FieldImage h{};
  memcpy(h.magic, kFieldMagic, 8);
  h.nx = f->nx;
  h.ny = f->ny;
  h.w = f->w;
  h.storage = f->storage;
  h.noise = f->noise;
  h.nwin = f->nwin;
  h.tau = f->tau;
  h.received = f->received;
  h.hist_units = p->hist_units;
  h.nsnaps = (uint32_t)std::min<int64_t>(2, f->received);
  h.slice_bytes = (int64_t)p->slice_bytes;
  h.hist_bytes = p->hist_n ? (int64_t)sizeof(float) * ((int64_t)p->hist_n * p->vstride + p->hist_n) : 0;
  CK(cudaMemcpy(&h.gmax_key, p->d_small, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  char* o = static_cast<char*>(out);
  memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  for (int64_t r = f->received - h.nsnaps; r < f->received; ++r) {   // oldest first
    CK(cudaMemcpy(o, p->d_stack + p->slice_bytes * (r % 3), p->slice_bytes, cudaMemcpyDeviceToHost));
    o += p->slice_bytes;
  }
  if (p->hist_n) {
    CK(cudaMemcpy(o, p->d_hist, sizeof(float) * (size_t)p->hist_n * p->vstride, cudaMemcpyDeviceToHost));
    o += sizeof(float) * (size_t)p->hist_n * p->vstride;
    CK(cudaMemcpy(o, p->d_hwts, sizeof(float) * p->hist_n, cudaMemcpyDeviceToHost));
  }
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_field_import(fitrig_server_t s, const void* image, int64_t size,
                                          int32_t* field_id) {
  if (!s || !image || !field_id || size < (int64_t)sizeof(FieldImage)) return FITRIG_EINVAL;
  FieldImage h;
  memcpy(&h, image, sizeof(h));
  if (memcmp(h.magic, kFieldMagic, 8) != 0 || h.nsnaps > 2 || h.received < 0 ||
      h.nsnaps != (uint32_t)std::min<int64_t>(2, h.received) || h.hist_units < 0 ||
      size != (int64_t)sizeof(h) + (int64_t)h.nsnaps * h.slice_bytes + h.hist_bytes)
    return FITRIG_EINVAL;
  if (h.nx < 1 || h.ny < 1 || h.w < 1 || h.w > std::min(h.nx, h.ny) || !(h.tau > 0.0) ||
      (h.storage != FITRIG_F32 && h.storage != FITRIG_BF16 && h.storage != FITRIG_F16) ||
      (h.noise != FITRIG_NOISE_MEANSTD && h.noise != FITRIG_NOISE_MEDMAD) || h.nwin < 0 || h.nwin > 256)
    return FITRIG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mtx);
  CK(cudaSetDevice(s->device));
  if (!s->waiting.empty() || s->active >= s->max_fields) return FITRIG_EBUSY;
  ServerField* f = new (std::nothrow) ServerField();
  if (!f) return FITRIG_ENOMEM;
  f->nx = h.nx;
  f->ny = h.ny;
  f->w = h.w;
  f->tau = h.tau;
  f->storage = h.storage;
  f->noise = h.noise;
  f->nwin = h.nwin;
  const int rc = activate(s, f);   // nothing is queued by an import
  if (rc != FITRIG_OK) {
    delete f;
    return rc;
  }
  fitrig_plan_t p = f->plan;
  const int64_t hist = p->hist_n ? (int64_t)sizeof(float) * ((int64_t)p->hist_n * p->vstride + p->hist_n) : 0;
  bool ok = h.slice_bytes == (int64_t)p->slice_bytes && h.hist_bytes == hist;
  const char* in = static_cast<const char*>(image) + sizeof(h);
  for (int64_t r = h.received - h.nsnaps; ok && r < h.received; ++r) {
    ok = cudaMemcpy(p->d_stack + p->slice_bytes * (r % 3), in, p->slice_bytes,
                    cudaMemcpyHostToDevice) == cudaSuccess;
    in += p->slice_bytes;
  }
  if (ok && p->hist_n) {
    ok = cudaMemcpy(p->d_hist, in, sizeof(float) * (size_t)p->hist_n * p->vstride,
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->d_hwts, in + sizeof(float) * (size_t)p->hist_n * p->vstride,
                    sizeof(float) * p->hist_n, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  ok = ok && cudaMemcpy(p->d_small, &h.gmax_key, sizeof(uint32_t), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    s->used -= f->bytes;
    --s->active;
    free_field(f);
    delete f;
    return FITRIG_EINVAL;
  }
  f->received = h.received;
  p->hist_units = h.hist_units;
  p->freq_ready = p->hist_n > 0 && p->hist_units >= p->hist_n;
  f->id = (int)s->fields.size();
  s->fields.push_back(f);
  *field_id = f->id;
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_retire(fitrig_server_t s, int32_t field) {
  if (!s) return FITRIG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mtx);
  if (field < 0 || field >= (int)s->fields.size()) return FITRIG_EINVAL;
  ServerField* f = s->fields[field];
  if (f->state == kFieldQueued) {
    for (auto it = s->waiting.begin(); it != s->waiting.end(); ++it)
      if (*it == field) {
        s->waiting.erase(it);
        break;
      }
    f->state = kFieldRetired;
    return FITRIG_OK;
  }
  if (f->state != kFieldActive) return FITRIG_ESTATE;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(f->stream);   // its pending results are delivered
  free_field(f);
  s->used -= f->bytes;
  f->bytes = 0;
  f->state = kFieldRetired;
  --s->active;
  admit_waiting(s);
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_usage(fitrig_server_t s, int64_t* used_bytes, int32_t* active,
                                   int32_t* waiting) {
  if (!s || !used_bytes || !active || !waiting) return FITRIG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mtx);
  *used_bytes = s->used;
  *active = s->active;
  *waiting = (int32_t)s->waiting.size();
  return FITRIG_OK;
}

FITRIG_API int fitrig_server_destroy(fitrig_server_t s) {
  if (!s) return FITRIG_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mtx);
    cudaSetDevice(s->device);
    for (ServerField* f : s->fields) {
      if (f->state == kFieldActive) {
        cudaStreamSynchronize(f->stream);
        free_field(f);
      }
      delete f;
    }
    s->fields.clear();
  }
  delete s;
  return FITRIG_OK;
}

FITRIG_API int fitrig_wait_probe(int64_t timeout_ns, int64_t stream) {
  if (timeout_ns <= 0 || timeout_ns > 10000000000ll) return FITRIG_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned* d = nullptr;
  unsigned h = 0;
  CK(cudaMalloc(&d, sizeof(unsigned)));
  cudaError_t e = launch_wait_probe((uint64_t)timeout_ns, d, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return FITRIG_ECUDA;
  }
  return h ? FITRIG_ETIMEOUT : FITRIG_OK;
}

FITRIG_API int fitrig_launch_count(int64_t* count) {
  if (!count) return FITRIG_EINVAL;
  *count = g_launches.load(std::memory_order_relaxed);
  return FITRIG_OK;
}

FITRIG_API int fitrig_plan_destroy(fitrig_plan_t p) {
  if (!p) return FITRIG_EINVAL;
  cudaSetDevice(p->device);
  if (p->allocated || p->d_stack) {
    cudaStreamSynchronize(plan_stream(p));
  }
  free_all(p);
  for (int i = 0; i < 2 * FITRIG_KERNEL_COUNT; ++i)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  for (cudaStream_t c : p->copy_st)
    if (c) cudaStreamDestroy(c);
  for (cudaEvent_t c : p->copy_ev)
    if (c) cudaEventDestroy(c);
  if (p->own_stream) cudaStreamDestroy(p->own_stream);
  if (p->side_st) cudaStreamDestroy(p->side_st);
  if (p->fork_ev) cudaEventDestroy(p->fork_ev);
  if (p->join_ev) cudaEventDestroy(p->join_ev);
  delete p;
  return FITRIG_OK;
}

}  // extern "C"
