// fitrig_noise_static: the per-group noise estimate (mean/std or median/MAD)
// of caller-provided device maps, with all of its working memory in one
// file-scope device array instead of memory it allocates.
//
// Who needs this: a caller that must not call cudaMalloc -- for example a
// real-time trigger loop that cannot afford an allocation that may block or
// synchronise the device mid-stream, or a host program whose device memory is
// owned by another allocator that forbids raw allocations.  Such a caller
// passes its input maps and its output buffer; this entry point allocates
// nothing (no cudaMalloc, cudaFree or allocating library call).
//
// The array is held by every GPU that loads the library until the process
// exits.  Every call on a device shares it and it keeps the last call's
// contents, so each call clears what must start at zero; calls that overlap
// on the GPU (e.g. on two streams at once) race on it and must not be issued.
// The first call on a device (and the first after a device reset) looks up
// the array's device address (a host-side symbol is only a stand-in for it);
// make that first call before any stream capture.  Each map is split over
// 608 / groups blocks (at least one), so a call with many groups reads each
// map with few blocks: correct, but far below the memory bandwidth for large
// maps.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kMaxGroups = FITRIG_NOISE_STATIC_MAX_GROUPS;
constexpr int kBlocks = 152 * 4;   // blocks per map pass, split over the groups
constexpr int kMaxDevices = 64;

// Layout (bytes, 256-aligned sections):
//   part  double [kBlocks + kMaxGroups]     per-block partial sums
//   cnt   int    [kBlocks + kMaxGroups]     per-block counts
//   hist  uint   [kMaxGroups][2048]         radix histograms
//   rsel  uint   [kMaxGroups][4]            radix-select state
//   shift float  [kMaxGroups]               FP32 means of the second pass
constexpr size_t kSlots = kBlocks + kMaxGroups;
constexpr size_t kOffCnt = ((kSlots * 8 + 255) / 256) * 256;
constexpr size_t kOffHist = kOffCnt + ((kSlots * 4 + 255) / 256) * 256;
constexpr size_t kOffRsel = kOffHist + (size_t)kMaxGroups * 2048 * 4;
constexpr size_t kOffShift = kOffRsel + ((kMaxGroups * 16 + 255) / 256) * 256;
constexpr size_t kScratchBytes = kOffShift + ((kMaxGroups * 4 + 255) / 256) * 256;

__device__ __align__(256) static unsigned char g_noise_scratch[kScratchBytes];

std::mutex g_setup_mutex;

// The cached address belongs to one CUDA context: a device reset (or the
// primary context being released and created again) reloads the module, and
// the array may then sit elsewhere.  Each device's entry therefore records
// the unique ID of the context it was looked up in (cuCtxGetId, never reused
// within a process) and is looked up again when the current context differs.
struct ScratchEntry {
  unsigned long long ctx_id = 0;
  bool valid = false;
  unsigned char* addr = nullptr;
};
ScratchEntry g_scratch[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

template <typename Fn>
Fn driver_fn(const char* name, int version) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return reinterpret_cast<Fn>(p);
}

// Unique ID of the calling thread's current context on device `dev`
// (cudaSetDevice makes the device's primary context current and initialises
// it; it allocates nothing).
int current_context_id(int dev, unsigned long long* id) {
  static CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent", 12000);
  static CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId", 12000);
  if (!get_current || !get_id) return FITRIG_EUNSUPPORTED;
  if (cudaSetDevice(dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return FITRIG_ECUDA;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return FITRIG_ECUDA;
  return get_id(ctx, id) == CUDA_SUCCESS ? FITRIG_OK : FITRIG_ECUDA;
}

// Device address of the scratch array in the current device's current
// context (looked up once per context).
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FITRIG_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return FITRIG_EUNSUPPORTED;
  unsigned long long ctx = 0;
  const int rc = current_context_id(dev, &ctx);
  if (rc != FITRIG_OK) return rc;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchEntry& e = g_scratch[dev];
  if (!e.valid || e.ctx_id != ctx) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noise_scratch);
    if (err != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return FITRIG_ECUDA;
    }
    e.addr = static_cast<unsigned char*>(p);
    e.ctx_id = ctx;
    e.valid = true;
  }
  *out = e.addr;
  return FITRIG_OK;
}

}  // namespace

extern "C" FITRIG_API int fitrig_noise_static(const float* dev_values, int32_t groups, int64_t n,
                                              int noise_mode, double* dev_centre_scale,
                                              int64_t stream) {
  if (!dev_values || !dev_centre_scale || n < 1 || groups < 1) return FITRIG_EINVAL;
  if (groups > kMaxGroups) return FITRIG_EINVAL;   // beyond the static scratch
  if (n > (int64_t)INT32_MAX) return FITRIG_EINVAL;
  if (noise_mode != FITRIG_NOISE_MEANSTD && noise_mode != FITRIG_NOISE_MEDMAD) return FITRIG_EINVAL;
  unsigned char* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != FITRIG_OK) return rc;
  fitrig::NoiseScratch s;
  s.nblk = kBlocks / groups > 0 ? kBlocks / groups : 1;
  s.part = reinterpret_cast<double*>(base);
  s.cnt = reinterpret_cast<int*>(base + kOffCnt);
  s.hist = reinterpret_cast<unsigned*>(base + kOffHist);
  s.rsel = reinterpret_cast<unsigned*>(base + kOffRsel);
  s.shift = reinterpret_cast<float*>(base + kOffShift);
  s.invalid = nullptr;
  // launch_noise clears the histogram and select state it needs before use;
  // the mean/std partials are fully overwritten by each pass.
  const cudaError_t e = fitrig::launch_noise(dev_values, groups, n, n, noise_mode, s,
                                             dev_centre_scale,
                                             reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return FITRIG_ECUDA;
  }
  return FITRIG_OK;
}
