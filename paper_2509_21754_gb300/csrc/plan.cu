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
  uint64_t timeout_ns = 2000000000ull;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  // derived
  int Tx = 0, Ty = 0, nxu = 0, nyu = 0, units = 0;
  int64_t T = 0;
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
  unsigned* d_small = nullptr;   // [0] gmax key, [1] status flags, [2] ncand
  unsigned long long* d_invalid = nullptr;
  double* d_cs = nullptr;        // (units + 1) x (centre, scale)
  float* d_thr = nullptr;        // units + 1
  void* d_noise = nullptr;
  NoiseScratch ns_img{}, ns_freq{};
  void* d_sel = nullptr;
  SelectScratch sel{};
  fitrig_candidate* d_cand = nullptr;
  fitrig_candidate* d_cand_tmp = nullptr;
  int64_t cand_cap = 0;
  float* d_eta = nullptr;
  int* d_bin = nullptr;
  float2* d_tw = nullptr;
  void* d_staging = nullptr;
  float* d_report = nullptr;
  unsigned* h_pinned = nullptr;   // [0..3] readback words
  CUtensorMap tmap;
  cudaEvent_t ev[2 * FITRIG_KERNEL_COUNT] = {};
  float ms[FITRIG_KERNEL_COUNT] = {};
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

static int select_capacity(fitrig_plan_t p) {
  const int64_t all = (int64_t)p->units * p->T;
  const int64_t cap = std::min<int64_t>(all, (int64_t)(4 << 20) + all / 64);
  return (int)std::max<int64_t>(cap, 1);
}

static void free_all(fitrig_plan_t p) {
  void* ptrs[] = {p->d_stack, p->d_vp,  p->d_small, p->d_invalid,  p->d_cs,
                  p->d_thr,   p->d_noise, p->d_sel, p->d_cand,     p->d_cand_tmp,
                  p->d_eta,   p->d_bin, p->d_tw,    p->d_staging,  p->d_report};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->h_pinned) cudaFreeHost(p->h_pinned);
  p->h_pinned = nullptr;
  p->allocated = false;
}

static int allocate(fitrig_plan_t p) {
  if (p->allocated) return FITRIG_OK;
  const int eb = elem_bytes(p->storage);
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
    if (!stack_geometry(p->w, eb, &p->geom)) return FITRIG_EUNSUPPORTED;
    p->geom.gridX = (p->Tx + p->geom.TBX - 1) / p->geom.TBX;
    p->geom.gridY = (p->Ty + p->geom.TBY - 1) / p->geom.TBY;
    if (p->geom.gridY > 65535) return FITRIG_EUNSUPPORTED;
    boxW = p->geom.boxW;
    boxH = p->geom.BH;
  }
  const int U = p->units;
  CK(cudaMalloc(&p->d_stack, p->slice_bytes * p->L));
  CK(cudaMalloc(&p->d_vp, sizeof(float) * (size_t)U * p->T));
  CK(cudaMalloc(&p->d_small, 64));
  CK(cudaMalloc(&p->d_invalid, sizeof(unsigned long long)));
  CK(cudaMalloc(&p->d_cs, sizeof(double) * 2 * (U + 1)));
  CK(cudaMalloc(&p->d_thr, sizeof(float) * (U + 1)));
  const int nblk_img = std::max(1, std::min(1024, (152 * 4 + U - 1) / U));
  const int nblk_freq = 152 * 4;
  const size_t nb = std::max(noise_scratch_bytes(U, nblk_img), noise_scratch_bytes(1, nblk_freq));
  CK(cudaMalloc(&p->d_noise, nb));
  noise_scratch_carve(p->d_noise, U, nblk_img, &p->ns_img);
  noise_scratch_carve(p->d_noise, 1, nblk_freq, &p->ns_freq);
  p->ns_img.invalid = p->d_invalid;
  p->ns_freq.invalid = p->d_invalid;
  // selection lists
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
  const size_t o_cnt = carve(sizeof(int) * s.nblk), o_off = carve(sizeof(int) * (s.nblk + 1));
  const size_t o_items = carve(sizeof(SelItem) * cap), o_nsel = carve(sizeof(int));
  const size_t o_par = carve(sizeof(int) * cap), o_cm = carve(sizeof(unsigned long long) * cap);
  const size_t o_pk = carve(sizeof(int) * cap);
  const size_t o_pl = carve(sizeof(int) * cap), o_np = carve(sizeof(int));
  const size_t map_n = (size_t)std::max<int64_t>(1, (int64_t)U * p->T);
  const size_t o_map = carve(sizeof(int) * map_n);
  CK(cudaMalloc(&p->d_sel, bytes));
  CK(cudaMemset(p->d_sel, 0, bytes));
  char* b = static_cast<char*>(p->d_sel);
  s.blkcnt = reinterpret_cast<int*>(b + o_cnt);
  s.blkoff = reinterpret_cast<int*>(b + o_off);
  s.items = reinterpret_cast<SelItem*>(b + o_items);
  s.nsel = reinterpret_cast<int*>(b + o_nsel);
  s.parent = reinterpret_cast<int*>(b + o_par);
  s.compmax = reinterpret_cast<unsigned long long*>(b + o_cm);
  s.peak = reinterpret_cast<int*>(b + o_pk);
  s.plist = reinterpret_cast<int*>(b + o_pl);
  s.npeak = reinterpret_cast<int*>(b + o_np);
  s.map = reinterpret_cast<int*>(b + o_map);
  p->cand_cap = s.capacity;
  CK(cudaMalloc(&p->d_cand, sizeof(fitrig_candidate) * cap));
  CK(cudaMalloc(&p->d_cand_tmp, sizeof(fitrig_candidate) * cap));
  if (p->branch & FITRIG_BRANCH_FREQ) {
    CK(cudaMalloc(&p->d_eta, sizeof(float) * p->T));
    CK(cudaMalloc(&p->d_bin, sizeof(int) * p->T));
    const int n = U, H = (n - 1) / 2, K = n / 2;
    std::vector<float2> tw((size_t)std::max(1, K * H));
    for (int k = 1; k <= K; ++k)
      for (int q = 1; q <= H; ++q) {
        const double ang = 2.0 * M_PI * (double)(((int64_t)k * q) % n) / (double)n;
        tw[(size_t)(k - 1) * H + (q - 1)] = make_float2((float)std::cos(ang), (float)std::sin(ang));
      }
    CK(cudaMalloc(&p->d_tw, sizeof(float2) * tw.size()));
    CK(cudaMemcpy(p->d_tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice));
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
  if ((branch & FITRIG_BRANCH_FREQ) && nsnap - 2 > 256) return FITRIG_EUNSUPPORTED;
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
  if (cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
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
    case FITRIG_OPT_TIMEOUT_NS:
      if (value <= 0) return FITRIG_EINVAL;
      p->timeout_ns = (uint64_t)value;
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
    case FITRIG_OPT_NOISE:
      if (value != FITRIG_NOISE_MEANSTD && value != FITRIG_NOISE_MEDMAD) return FITRIG_EINVAL;
      p->noise = (int)value;
      return FITRIG_OK;
    case FITRIG_OPT_RMODE:
      if (value != FITRIG_RMODE_ABS && value != FITRIG_RMODE_SIGNED) return FITRIG_EINVAL;
      p->rmode = (int)value;
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

FITRIG_API int fitrig_push_snapshot(fitrig_plan_t p, const void* data, int dtype, int on_device,
                                    int64_t row_pitch_elems) {
  if (!p || !data) return FITRIG_EINVAL;
  if (dtype != FITRIG_F32 && dtype != FITRIG_BF16 && dtype != FITRIG_F16) return FITRIG_EINVAL;
  const int64_t rp = row_pitch_elems ? row_pitch_elems : p->nx;
  if (rp < p->nx) return FITRIG_EINVAL;
  if (p->pushed >= p->L) return FITRIG_ESTATE;
  CK(cudaSetDevice(p->device));
  int rc = ensure_allocated(p);
  if (rc != FITRIG_OK) return rc;
  cudaStream_t st = plan_stream(p);
  const int eb = elem_bytes(p->storage), ib = elem_bytes(dtype);
  char* dst = p->d_stack + p->slice_bytes * p->pushed;
  if (dtype == p->storage) {
    CK(cudaMemcpy2DAsync(dst, p->pitch * eb, data, rp * ib, (size_t)p->nx * ib, p->ny,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  } else {
    const void* src = data;
    int64_t sp = rp;
    if (!on_device) {
      if (!p->d_staging) CK(cudaMalloc(&p->d_staging, (size_t)p->nx * p->ny * 4));
      CK(cudaMemcpy2DAsync(p->d_staging, (size_t)p->nx * ib, data, rp * ib, (size_t)p->nx * ib,
                           p->ny, cudaMemcpyHostToDevice, st));
      src = p->d_staging;
      sp = p->nx;
    }
    CK(launch_convert(src, dtype, sp, dst, p->storage, p->pitch, p->ny, p->nx, st));
  }
  if (!on_device) CK(cudaStreamSynchronize(st));
  p->pushed += 1;
  p->detected = false;
  return FITRIG_OK;
}

FITRIG_API int fitrig_plan_reset(fitrig_plan_t p) {
  if (!p) return FITRIG_EINVAL;
  p->pushed = 0;
  p->detected = false;
  return FITRIG_OK;
}

static void rec(fitrig_plan_t p, int k, int end, cudaStream_t st) {
  cudaEventRecord(p->ev[2 * k + end], st);
}

FITRIG_API int fitrig_detect(fitrig_plan_t p, int32_t* ncand) {
  if (!p || !ncand) return FITRIG_EINVAL;
  *ncand = 0;
  if (p->pushed < 3) return FITRIG_ESTATE;
  if ((p->branch & FITRIG_BRANCH_FREQ) && p->pushed != p->L) return FITRIG_ESTATE;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = plan_stream(p);
  const int P = p->pushed, U = P - 2;
  unsigned* gmax = p->d_small;
  unsigned* status = p->d_small + 1;
  int* nout = reinterpret_cast<int*>(p->d_small + 2);
  CK(cudaMemsetAsync(p->d_small, 0, 16, st));
  CK(cudaMemsetAsync(p->d_invalid, 0, sizeof(unsigned long long), st));
  rec(p, FITRIG_KERNEL_DETECT, 0, st);
  rec(p, FITRIG_KERNEL_STACK, 0, st);
  StackArgs a;
  a.nx = p->nxu;
  a.ny = p->nyu;
  a.nsnap = P;
  a.Tx = p->Tx;
  a.Ty = p->Ty;
  a.T = p->T;
  a.vp = p->d_vp;
  a.gmax = gmax;
  a.status = status;
  a.timeout_ns = p->timeout_ns;
  a.g = p->geom;
  if (p->stride == FITRIG_STRIDE_SLIDING) {
    SlideArgs sa;
    sa.nx = p->nx;
    sa.ny = p->ny;
    sa.nsnap = P;
    sa.vp = p->d_vp;
    sa.gmax = gmax;
    sa.status = status;
    sa.timeout_ns = p->timeout_ns;
    sa.g = p->sgeom;
    CK(launch_slide(&p->tmap, sa, p->storage, p->rmode, st));
  } else {
    CK(launch_stack(&p->tmap, a, p->storage, p->rmode, st));
  }
  rec(p, FITRIG_KERNEL_STACK, 1, st);
  CandArgs ca;
  ca.nx = p->nxu;
  ca.ny = p->nyu;
  ca.w = p->stride == FITRIG_STRIDE_SLIDING ? 1 : p->w;   // pixels are 1 x 1 tiles
  ca.Tx = p->Tx;
  ca.Ty = p->Ty;
  ca.T = p->T;
  ca.stack = p->d_stack;
  ca.storage = p->storage;
  ca.pitch = p->pitch;
  ca.slice = (int64_t)p->pitch * p->ny;
  ca.eta = p->d_eta;
  ca.bin = p->d_bin;
  ca.out = p->d_cand;
  ca.nout = nout;
  ca.cap = p->cand_cap;
  // frequency branch first: its candidates (snapshot -1) lead the sorted list
  if (p->branch & FITRIG_BRANCH_FREQ) {
    rec(p, FITRIG_KERNEL_SPECTRUM, 0, st);
    CK(launch_spectrum(p->d_vp, U, p->T, p->d_tw, p->d_eta, p->d_bin, st));
    rec(p, FITRIG_KERNEL_SPECTRUM, 1, st);
    double* cs = p->d_cs + 2 * U;
    CK(launch_noise(p->d_eta, 1, p->T, p->noise, p->ns_freq, cs, st));
    CK(launch_thresholds(cs, 1, p->tau, p->d_thr + U, st));
    CK(launch_select(p->d_eta, 1, p->T, p->d_thr + U, cs, p->sel, status, st));
    CK(launch_components(p->Tx, p->Ty, p->T, p->sel, status, st));
    ca.branch = FITRIG_BRANCH_FREQ;
    CK(launch_emit_candidates(ca, p->sel, nout, p->d_cand_tmp, status, st));
  }
  if (p->branch & FITRIG_BRANCH_IMAGE) {
    rec(p, FITRIG_KERNEL_NOISE, 0, st);
    CK(launch_noise(p->d_vp, U, p->T, p->noise, p->ns_img, p->d_cs, st));
    CK(launch_thresholds(p->d_cs, U, p->tau, p->d_thr, st));
    rec(p, FITRIG_KERNEL_NOISE, 1, st);
    rec(p, FITRIG_KERNEL_SELECT, 0, st);
    CK(launch_select(p->d_vp, U, p->T, p->d_thr, p->d_cs, p->sel, status, st));
    CK(launch_components(p->Tx, p->Ty, p->T, p->sel, status, st));
    ca.branch = FITRIG_BRANCH_IMAGE;
    CK(launch_emit_candidates(ca, p->sel, nout, p->d_cand_tmp, status, st));
    rec(p, FITRIG_KERNEL_SELECT, 1, st);
  }
  CK(launch_clamp_count(nout, (int)p->cand_cap, status, st));
  rec(p, FITRIG_KERNEL_DETECT, 1, st);
  CK(cudaMemcpyAsync(p->h_pinned, p->d_small, 16, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(p->h_pinned + 4, p->d_invalid, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int k = 0; k < FITRIG_KERNEL_COUNT; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev[2 * k], p->ev[2 * k + 1]) == cudaSuccess) p->ms[k] = ms;
    else (void)cudaGetLastError();
  }
  const unsigned flags = p->h_pinned[1];
  const int n = (int)p->h_pinned[2];
  unsigned long long invalid;
  memcpy(&invalid, p->h_pinned + 4, 8);
  p->last_ncand = n;
  p->detected = true;
  p->detected_branch = p->branch;
  p->detected_units = U;
  *ncand = n;
  if (flags & kErrTimeout) return FITRIG_ETIMEOUT;
  if (flags & (kErrCapacity | kErrCcLimit)) return FITRIG_ETRUNC;
  if (invalid) return FITRIG_ENONFINITE;
  return FITRIG_OK;
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
  return read_floats(p, p->d_vp + (size_t)unit * p->T, p->T, out, cap);
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
    CK(launch_finite_max(p->d_stack, p->storage, p->pushed, p->nyu, p->nxu, p->pitch, p->d_small,
                         st));
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
  if (!p->d_report) CK(cudaMalloc(&p->d_report, sizeof(float) * p->T));
  CK(launch_tlisi_from_values(p->d_vp + (size_t)unit * p->T, p->T, p->d_small, p->d_report, st));
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
  *ptr = p->d_stack + p->slice_bytes * s;
  *row_pitch_elems = p->pitch;
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
  const size_t extra = 256 + sizeof(int) * (nblk + 2) + sizeof(long long) * 2 + 64;
  CK(cudaMalloc(&scratch, nb + extra));
  NoiseScratch ns;
  noise_scratch_carve(scratch, 1, nblk, &ns);
  char* tail = static_cast<char*>(scratch) + nb;
  double* cs = reinterpret_cast<double*>(tail);
  float* thr = reinterpret_cast<float*>(tail + 16);
  unsigned long long* inval = reinterpret_cast<unsigned long long*>(tail + 32);
  long long* total = reinterpret_cast<long long*>(tail + 48);
  int* blkcnt = reinterpret_cast<int*>(tail + 64);
  ns.invalid = inval;
  int rc = FITRIG_OK;
  double h[2] = {0, 0};
  long long cnt = 0;
  cudaError_t e = cudaMemsetAsync(inval, 0, 8, st);
  if (e == cudaSuccess) e = launch_noise(dev_map, 1, n, noise_mode, ns, cs, st);
  if (e == cudaSuccess) e = launch_thresholds(cs, 1, nsigma, thr, st);
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
  if (p->own_stream) cudaStreamDestroy(p->own_stream);
  delete p;
  return FITRIG_OK;
}

}  // extern "C"
