// Noise estimates of a map of tile statistics, per group (unit).
//
// MEANSTD (Sec. 2.4.1: "mean and standard deviation of the tLISI matrix"):
// two passes, the mean first and then the sum of squared deviations from it.
// Each thread accumulates its strided share in FP32 with Kahan compensation,
// blocks reduce in FP64 in a fixed tree and the per-block partials are merged
// in FP64 in block order, so results are deterministic.  The population
// standard deviation is used.
//
// MEDMAD (robust reading): the lower median (rank floor((n-1)/2)) of the finite
// values and the lower median of |v - median| computed in FP32, each found by
// an exact radix select over order-preserving 32-bit keys in three digit passes
// (11, 11 and 10 bits) with integer histograms; scale = 1.482602218505602 MAD.
// Both medians are bit-exact elements of the (derived) value arrays.
#include <cfloat>
#include <cmath>

#include "internal.cuh"

namespace fitrig {

constexpr int kNoiseThreads = 256;
constexpr int kBins = 2048;

size_t noise_scratch_bytes(int groups, int nblk) {
  size_t b = 0;
  b += (size_t)groups * nblk * sizeof(double);
  b += (size_t)groups * nblk * sizeof(int);
  b = (b + 255) / 256 * 256;
  b += (size_t)groups * kBins * sizeof(unsigned);
  b += (size_t)groups * 4 * sizeof(unsigned);
  b += (size_t)groups * sizeof(float);
  return (b + 255) / 256 * 256;   // callers may carve more after this
}

void noise_scratch_carve(void* base, int groups, int nblk, NoiseScratch* s) {
  char* p = static_cast<char*>(base);
  s->nblk = nblk;
  s->part = reinterpret_cast<double*>(p);
  p += (size_t)groups * nblk * sizeof(double);
  s->cnt = reinterpret_cast<int*>(p);
  p += (size_t)groups * nblk * sizeof(int);
  size_t off = (size_t)(p - static_cast<char*>(base));
  off = (off + 255) / 256 * 256;
  p = static_cast<char*>(base) + off;
  s->hist = reinterpret_cast<unsigned*>(p);
  p += (size_t)groups * kBins * sizeof(unsigned);
  s->rsel = reinterpret_cast<unsigned*>(p);
  p += (size_t)groups * 4 * sizeof(unsigned);
  s->shift = reinterpret_cast<float*>(p);
}

// ---------------------------------------------------------------- MEANSTD
// Partial sums of v (sq == 0) or of (v - shift[g])^2 (sq == 1) over finite v.
__global__ void __launch_bounds__(kNoiseThreads) k_sum_pass(const float* __restrict__ vals,
                                                            int64_t n, int nblk, int sq,
                                                            const float* __restrict__ shift,
                                                            double* part, int* cnt) {
  __shared__ double sh[kNoiseThreads];
  __shared__ int shc[kNoiseThreads];
  const int g = blockIdx.y;
  const float* v = vals + (size_t)g * n;
  const float m = sq ? shift[g] : 0.f;
  float s = 0.f, comp = 0.f;
  int c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)nblk * blockDim.x) {
    const float x = v[i];
    if (!isfinite(x)) continue;
    float term = x;
    if (sq) {
      const float d = x - m;
      term = d * d;
    }
    const float y = term - comp;
    const float t = s + y;
    comp = (t - s) - y;
    s = t;
    ++c;
  }
  sh[threadIdx.x] = (double)s - (double)comp;
  shc[threadIdx.x] = c;
  __syncthreads();
  for (int d = kNoiseThreads / 2; d > 0; d >>= 1) {
    if (threadIdx.x < d) {
      sh[threadIdx.x] += sh[threadIdx.x + d];
      shc[threadIdx.x] += shc[threadIdx.x + d];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[(size_t)g * nblk + blockIdx.x] = sh[0];
    cnt[(size_t)g * nblk + blockIdx.x] = shc[0];
  }
}

// stage 0: mean -> cs[2g], shift[g] = (float)mean.  stage 1: population std.
__global__ void k_sum_final(int groups, int64_t n, int nblk, int stage, const double* part,
                            const int* cnt, float* shift, double* cs,
                            unsigned long long* invalid) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= groups) return;
  double s = 0.0;
  long long c = 0;
  for (int b = 0; b < nblk; ++b) {
    s += part[(size_t)g * nblk + b];
    c += cnt[(size_t)g * nblk + b];
  }
  if (stage == 0) {
    if (invalid && c < n) atomicAdd(invalid, (unsigned long long)(n - c));
    const double mean = c > 0 ? s / (double)c : NAN;
    cs[2 * g] = mean;
    shift[g] = c > 0 ? (float)mean : 0.f;
  } else {
    if (c == 0) {
      cs[2 * g + 1] = 0.0;
      return;
    }
    // sum (v - a)^2 = sum (v - mean)^2 + c (mean - a)^2 with a = (float)mean
    const double off = cs[2 * g] - (double)shift[g];
    double var = s / (double)c - off * off;
    cs[2 * g + 1] = var > 0.0 ? sqrt(var) : 0.0;
  }
}

// ---------------------------------------------------------------- MEDMAD
// rsel[g*4 + 0] = key prefix, +1 = remaining rank, +2 = number of finite values,
// +3 = 1 if the group is degenerate (no finite values).
__device__ __forceinline__ bool rs_key(float v, int mad, float med, uint32_t* key) {
  if (!isfinite(v)) return false;
  *key = mad ? f32_key(fabsf(v - med)) : f32_key(v);
  return true;
}

__global__ void __launch_bounds__(kNoiseThreads) k_rs_hist(const float* __restrict__ vals,
                                                           int64_t n, int nblk, int pass,
                                                           int mad, const unsigned* rsel,
                                                           const double* cs, unsigned* hist) {
  __shared__ unsigned sh[kBins];
  const int g = blockIdx.y;
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const unsigned prefix = rsel[4 * g + 0];
  const bool degenerate = rsel[4 * g + 3] != 0;
  const float med = mad ? (float)cs[2 * g] : 0.f;
  const float* v = vals + (size_t)g * n;
  if (!degenerate) {
    // The trip count depends only on the block, so every lane of a warp reaches
    // the warp-wide match below together.
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)nblk * blockDim.x) {
      const int64_t i = base + threadIdx.x;
      uint32_t key = 0;
      const bool ok = i < n && rs_key(v[i], mad, med, &key);
      if (pass == 0) {
        // the leading digit is concentrated (exponent bits): aggregate per warp
        const unsigned bin = ok ? (key >> 21) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (ok && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1))
          atomicAdd(&sh[bin], (unsigned)__popc(peers));
      } else if (pass == 1) {
        if (ok && (key >> 21) == prefix) atomicAdd(&sh[(key >> 10) & 2047u], 1u);
      } else {
        if (ok && (key >> 10) == prefix) atomicAdd(&sh[key & 1023u], 1u);
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[(size_t)g * kBins + b], sh[b]);
}

// One block per group: locate the digit holding the target rank (block-wide
// scan of the histogram), clear the histogram for the next pass, and finish
// the value after the last digit.
constexpr int kSelectThreads = 256;

__global__ void __launch_bounds__(kSelectThreads) k_rs_select(int groups, int64_t n, int pass,
                                                              int mad, unsigned* hist,
                                                              unsigned* rsel, double* cs,
                                                              unsigned long long* invalid) {
  __shared__ unsigned long long scan[kSelectThreads];
  __shared__ int found_bin;
  __shared__ unsigned found_below;
  const int g = blockIdx.x;
  const int tid = threadIdx.x;
  unsigned* h = hist + (size_t)g * kBins;
  unsigned* st = rsel + 4 * g;
  const int nb = pass == 2 ? 1024 : 2048;
  const int per = nb / kSelectThreads;
  unsigned local[8];
  unsigned long long mine = 0;
  for (int i = 0; i < per; ++i) {
    local[i] = h[tid * per + i];
    mine += local[i];
  }
  scan[tid] = mine;
  __syncthreads();
  for (int d = 1; d < kSelectThreads; d <<= 1) {
    const unsigned long long add = tid >= d ? scan[tid - d] : 0ull;
    __syncthreads();
    scan[tid] += add;
    __syncthreads();
  }
  const unsigned long long total = scan[kSelectThreads - 1];
  const unsigned long long before = scan[tid] - mine;
  for (int i = 0; i < per; ++i) h[tid * per + i] = 0;   // ready for the next pass
  if (pass == 0 && tid == 0) {
    if (!mad) {
      st[2] = (unsigned)total;
      if (invalid && (int64_t)total < n) atomicAdd(invalid, (unsigned long long)(n - (int64_t)total));
    }
    st[3] = total == 0 ? 1u : 0u;
    st[1] = total == 0 ? 0u : (unsigned)((total - 1) / 2);
  }
  __syncthreads();
  if (st[3]) {
    if (tid == 0 && pass == 2) {
      if (!mad) cs[2 * g] = NAN;
      cs[2 * g + 1] = 0.0;
    }
    return;
  }
  const unsigned k = st[1];
  if ((unsigned long long)k >= before && (unsigned long long)k < before + mine) {
    unsigned long long cum = before;
    for (int i = 0; i < per; ++i) {
      if (k < cum + local[i]) {
        found_bin = tid * per + i;
        found_below = (unsigned)cum;
        break;
      }
      cum += local[i];
    }
  }
  __syncthreads();
  if (tid != 0) return;
  const unsigned sel = (unsigned)found_bin;
  st[1] = k - found_below;
  if (pass == 0) {
    st[0] = sel;
  } else if (pass == 1) {
    st[0] = (st[0] << 11) | sel;
  } else {
    const uint32_t key = (st[0] << 10) | sel;
    const float val = f32_from_key(key);
    if (!mad) cs[2 * g] = (double)val;
    else cs[2 * g + 1] = kMadToSigma * (double)val;
    st[0] = 0;
  }
}

static int noise_blocks(int groups, const NoiseScratch& s) {
  (void)groups;
  return s.nblk;
}

cudaError_t launch_noise(const float* vals, int groups, int64_t n, int mode,
                         const NoiseScratch& s, double* cs, cudaStream_t st) {
  const int nblk = noise_blocks(groups, s);
  dim3 grid(nblk, groups);
  if (mode == FITRIG_NOISE_MEANSTD) {
    k_sum_pass<<<grid, kNoiseThreads, 0, st>>>(vals, n, nblk, 0, s.shift, s.part, s.cnt);
    k_sum_final<<<(groups + 127) / 128, 128, 0, st>>>(groups, n, nblk, 0, s.part, s.cnt, s.shift,
                                                      cs, s.invalid);
    k_sum_pass<<<grid, kNoiseThreads, 0, st>>>(vals, n, nblk, 1, s.shift, s.part, s.cnt);
    k_sum_final<<<(groups + 127) / 128, 128, 0, st>>>(groups, n, nblk, 1, s.part, s.cnt, s.shift,
                                                      cs, nullptr);
    count_launches(4);
    return cudaGetLastError();
  }
  if (mode != FITRIG_NOISE_MEDMAD) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(s.rsel, 0, (size_t)groups * 4 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.hist, 0, (size_t)groups * kBins * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  for (int mad = 0; mad < 2; ++mad) {
    for (int pass = 0; pass < 3; ++pass) {
      k_rs_hist<<<grid, kNoiseThreads, 0, st>>>(vals, n, nblk, pass, mad, s.rsel, cs, s.hist);
      k_rs_select<<<groups, kSelectThreads, 0, st>>>(groups, n, pass, mad, s.hist, s.rsel, cs,
                                                     s.invalid);
    }
  }
  count_launches(12);
  return cudaGetLastError();
}

__global__ void k_thresholds(const double* cs, int groups, double tau, float* thr) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= groups) return;
  const double c = cs[2 * g], s = cs[2 * g + 1];
  if (!(s > 0.0) || !isfinite(c) || !isfinite(s)) {
    thr[g] = INFINITY;   // degenerate spread: nothing is selected
    return;
  }
  // largest float <= c + tau*s, so (float v > thr) <=> ((double)v > c + tau*s)
  thr[g] = __double2float_rd(c + tau * s);
}

cudaError_t launch_thresholds(const double* cs, int groups, double tau, float* thr,
                              cudaStream_t st) {
  k_thresholds<<<(groups + 127) / 128, 128, 0, st>>>(cs, groups, tau, thr);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace fitrig
