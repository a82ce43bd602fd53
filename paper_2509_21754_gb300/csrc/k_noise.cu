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
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "internal.cuh"

namespace cg = cooperative_groups;

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
__device__ __forceinline__ void kahan_add(float term, float& s, float& comp) {
  const float y = term - comp;
  const float t = s + y;
  comp = (t - s) - y;
  s = t;
}

// Partial sums of v (sq == 0) or of (v - shift[g])^2 (sq == 1) over finite v.
// Group g's values start at vals + g * stride; VEC loads four at a time (the
// caller guarantees 16-byte alignment and stride % 4 == 0).
template <bool VEC>
__global__ void __launch_bounds__(kNoiseThreads) k_sum_pass(const float* __restrict__ vals,
                                                            int64_t stride, int nblk, int sq,
                                                            const float* __restrict__ shift,
                                                            double* part, int* cnt) {
  __shared__ double sh[kNoiseThreads];
  __shared__ int shc[kNoiseThreads];
  const int g = blockIdx.y;
  const float* v = vals + (size_t)g * stride;
  const float m = sq ? shift[g] : 0.f;
  float s = 0.f, comp = 0.f;
  int c = 0;
  auto take = [&](float x) {
    if (!isfinite(x)) return;
    float term = x;
    if (sq) {
      const float d = x - m;
      term = d * d;
    }
    kahan_add(term, s, comp);
    ++c;
  };
  if (VEC) {
    const float4* v4 = reinterpret_cast<const float4*>(v);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < stride / 4;
         i += (int64_t)nblk * blockDim.x) {
      const float4 q = v4[i];
      take(q.x);
      take(q.y);
      take(q.z);
      take(q.w);
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < stride;
         i += (int64_t)nblk * blockDim.x)
      take(v[i]);
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

__device__ __forceinline__ void rs_count(unsigned* sh, int pass, unsigned prefix, bool ok,
                                         uint32_t key) {
  if (pass == 0) {
    // the leading digit is concentrated (exponent bits): up to two leader
    // rounds add the lanes that share a leader's bin with one atomic each
    // (ballots, not match instructions, whose unit is slow), the rest add
    // their own
    const unsigned lane = threadIdx.x & 31;
    const unsigned bin = ok ? (key >> 21) : 0xffffffffu;
    unsigned left = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int round = 0; round < 2; ++round) {
      if (!left) break;
      const int lead = __ffs(left) - 1;
      const unsigned lb = __shfl_sync(0xffffffffu, bin, lead);
      const unsigned same = __ballot_sync(0xffffffffu, ok && bin == lb) & left;
      if ((int)lane == lead) atomicAdd(&sh[lb], (unsigned)__popc(same));
      left &= ~same;
    }
    if ((left >> lane) & 1u) atomicAdd(&sh[bin], 1u);
  } else if (pass == 1) {
    if (ok && (key >> 21) == prefix) atomicAdd(&sh[(key >> 10) & 2047u], 1u);
  } else {
    if (ok && (key >> 10) == prefix) atomicAdd(&sh[key & 1023u], 1u);
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kNoiseThreads) k_rs_hist(const float* __restrict__ vals,
                                                           int64_t stride, int nblk, int pass,
                                                           int mad, const unsigned* rsel,
                                                           const double* cs, unsigned* hist) {
  __shared__ unsigned sh[kBins];
  const int g = blockIdx.y;
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const unsigned prefix = rsel[4 * g + 0];
  const bool degenerate = rsel[4 * g + 3] != 0;
  const float med = mad ? (float)cs[2 * g] : 0.f;
  const float* v = vals + (size_t)g * stride;
  if (!degenerate) {
    // Trip counts depend only on the block, so every lane of a warp reaches the
    // warp-wide ballots in rs_count together.
    const int64_t nv = VEC ? stride / 4 : stride;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nv;
         base += (int64_t)nblk * blockDim.x) {
      const int64_t i = base + threadIdx.x;
      if (VEC) {
        float4 q = make_float4(NAN, NAN, NAN, NAN);
        if (i < nv) q = reinterpret_cast<const float4*>(v)[i];
        uint32_t k0 = 0, k1 = 0, k2 = 0, k3 = 0;
        const bool o0 = rs_key(q.x, mad, med, &k0), o1 = rs_key(q.y, mad, med, &k1);
        const bool o2 = rs_key(q.z, mad, med, &k2), o3 = rs_key(q.w, mad, med, &k3);
        rs_count(sh, pass, prefix, o0, k0);
        rs_count(sh, pass, prefix, o1, k1);
        rs_count(sh, pass, prefix, o2, k2);
        rs_count(sh, pass, prefix, o3, k3);
      } else {
        uint32_t key = 0;
        const bool ok = i < nv && rs_key(v[i], mad, med, &key);
        rs_count(sh, pass, prefix, ok, key);
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

// ---------------------------------------------------------------- MEDMAD, cluster form
// One thread-block cluster of 8 CTAs per group finds the median and then the
// MAD, every group of the map in the same launch, by range-binned selection
// over the order-preserving keys:
//   * a first sweep takes the minimum and maximum key (and the count) of the
//     group's finite values;
//   * a binning round counts the keys inside the current inclusive range
//     [lo, hi] in 4096 linear bins (digit = (key - lo) >> shift); the bin
//     holding the target rank becomes the new range and the rank is reduced by
//     the counts below it;
//   * once the range holds at most 20 Ki keys, one more pass over the group
//     copies exactly those keys into the CTAs' shared memory, and the
//     remaining rounds bin the copies instead of the whole map;
//   * the range ends as a single key: the exact order statistic;
//   * the MAD repeats this on the keys of |v - median| (FP32), whose range is
//     [0, max(|vmax - median|, |vmin - median|)].
// Each CTA bins its share into its own histogram, plus 64 coarse counts (64
// bins each).  After one cluster barrier every CTA reads the eight CTAs'
// coarse counts and then the 64 fine counts of the coarse bin that holds the
// rank through distributed shared memory and finds the new range itself, so
// all CTAs hold the same state without a leader.  The histograms are double
// buffered: a CTA rewrites a buffer only after the next barrier, when every
// CTA has finished reading it.  Integer counting only: the result is the
// element a sort would give.
constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 256;
constexpr int kClusterBins = 4096;
constexpr int kCoarse = 64;                                     // coarse bins of 64 fine bins
constexpr int kCollectPerCta = 5120;                            // keys kept per CTA
constexpr unsigned long long kCollectAll = kClusterCtas * kCollectPerCta / 2;
constexpr int64_t kClusterMaxPerGroup = 8 << 20;   // larger maps use the grid-wide passes

struct RangeState {
  unsigned long long lo, hi;   // inclusive key range
  unsigned long long rank;     // rank of the target inside the range
  unsigned long long count;    // keys inside the range
  unsigned shift;              // digit = (key - lo) >> shift
  unsigned done;
};

__device__ __forceinline__ unsigned range_shift(unsigned long long lo, unsigned long long hi) {
  const unsigned long long width = hi - lo + 1;   // <= 2^32
  unsigned s = 0;
  while ((width - 1) >> s >= (unsigned long long)kClusterBins) ++s;
  return s;
}

// Inclusive warp scan of two counts per lane (entries 2*lane, 2*lane+1); finds
// the entry holding `rank`.  Returns the entry and the count before it.
__device__ __forceinline__ void warp_find64(const unsigned* cnt, unsigned long long rank,
                                            int* entry, unsigned long long* below,
                                            unsigned* size) {
  const int lane = threadIdx.x & 31;
  const unsigned a = cnt[2 * lane], b = cnt[2 * lane + 1];
  unsigned long long incl = (unsigned long long)a + b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned long long excl = incl - a - b;
  int e = -1;
  unsigned long long bl = 0;
  unsigned sz = 0;
  if (rank >= excl && rank < excl + a) {
    e = 2 * lane;
    bl = excl;
    sz = a;
  } else if (rank >= excl + a && rank < incl) {
    e = 2 * lane + 1;
    bl = excl + a;
    sz = b;
  }
  const unsigned who = __ballot_sync(0xffffffffu, e >= 0);
  const int src = who ? __ffs(who) - 1 : 0;
  // the rank always lies inside the counted range; the clamp only keeps the
  // indices derived from `entry` in bounds
  *entry = max(0, __shfl_sync(0xffffffffu, e, src));
  *below = __shfl_sync(0xffffffffu, bl, src);
  *size = __shfl_sync(0xffffffffu, sz, src);
}

// (four CTAs per SM: the clusters of a whole map are resident at once)
template <bool VEC>
__global__ void __launch_bounds__(kClusterThreads, 4) k_medmad_cluster(const float* __restrict__ vals,
                                                                    int64_t stride, int64_t n,
                                                                    int g0, double* cs,
                                                                    unsigned long long* invalid,
                                                                    int skip_done) {
  pdl_begin();
  __shared__ unsigned hist[2][kClusterBins];
  __shared__ unsigned coarse[2][kCoarse];
  __shared__ uint32_t keep[kCollectPerCta];
  __shared__ unsigned nkeep, overflow;
  __shared__ unsigned long long red[kClusterThreads / 32][3];
  __shared__ unsigned sum64[kCoarse];
  __shared__ RangeState st;
  __shared__ unsigned long long mm[3];   // this CTA's min key, max key, count
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const int g = g0 + blockIdx.y;
  // after the bracketed kernel: only the groups it left (scale -1) remain; the
  // test reads one value, so every CTA of the cluster leaves together
  if (skip_done && cs[2 * g + 1] >= 0.0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* v = vals + (size_t)g * stride;
  const int64_t nv = VEC ? stride / 4 : stride;
  const int64_t step = (int64_t)kClusterCtas * blockDim.x;

  // visit every finite value of this CTA's share as an order-preserving key;
  // four loads are issued before their keys are used, so that each thread
  // keeps several requests in flight (the passes are latency-bound otherwise)
  auto for_keys = [&](int mad, float med, auto&& fn) {
    auto take = [&](float e) {
      uint32_t key;
      if (rs_key(e, mad, med, &key)) fn(key);
    };
    int64_t i = (int64_t)rank * blockDim.x + tid;
    if (VEC) {
      const float4* v4 = reinterpret_cast<const float4*>(v);
      for (; i + 3 * step < nv; i += 4 * step) {
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = v4[i + u * step];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          take(q[u].x);
          take(q[u].y);
          take(q[u].z);
          take(q[u].w);
        }
      }
      for (; i < nv; i += step) {
        const float4 q = v4[i];
        take(q.x);
        take(q.y);
        take(q.z);
        take(q.w);
      }
    } else {
      for (; i + 3 * step < nv; i += 4 * step) {
        float q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = v[i + u * step];
#pragma unroll
        for (int u = 0; u < 4; ++u) take(q[u]);
      }
      for (; i < nv; i += step) take(v[i]);
    }
  };

  // ---- sweep 0: min, max and count of the keys (each CTA its share; every
  // CTA then combines all shares through distributed shared memory)
  {
    unsigned long long kmin = ~0ull, kmax = 0ull, cnt = 0;
    for_keys(0, 0.f, [&](uint32_t key) {
      kmin = key < kmin ? key : kmin;
      kmax = key > kmax ? key : kmax;
      ++cnt;
    });
    for (int o = 16; o > 0; o >>= 1) {
      kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
      kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
      red[warp][0] = kmin;
      red[warp][1] = kmax;
      red[warp][2] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kClusterThreads / 32; ++w) {
        kmin = min(kmin, red[w][0]);
        kmax = max(kmax, red[w][1]);
        cnt += red[w][2];
      }
      mm[0] = kmin;
      mm[1] = kmax;
      mm[2] = cnt;
    }
  }
  cl.sync();   // every CTA's share is summarised
  unsigned long long gmin = ~0ull, gmax = 0ull, total = 0;
  for (int r = 0; r < kClusterCtas; ++r) {
    const unsigned long long* o = cl.map_shared_rank(mm, r);
    gmin = min(gmin, o[0]);
    gmax = max(gmax, o[1]);
    total += o[2];
  }
  if (total == 0) {
    if (rank == 0 && tid == 0) {
      cs[2 * g] = NAN;
      cs[2 * g + 1] = 0.0;
      if (invalid && n > 0) atomicAdd(invalid, (unsigned long long)n);
    }
    cl.sync();   // nobody leaves while others still read its shared memory
    return;
  }
  if (rank == 0 && tid == 0 && invalid && (int64_t)total < n)
    atomicAdd(invalid, (unsigned long long)(n - (int64_t)total));

  float med = 0.f;
  int buf = 0;
  for (int mad = 0; mad < 2; ++mad) {
    if (tid == 0) {
      if (mad == 0) {
        st.lo = gmin;
        st.hi = gmax;
      } else {
        const float vmin = f32_from_key((uint32_t)gmin), vmax = f32_from_key((uint32_t)gmax);
        st.lo = f32_key(0.f);
        st.hi = f32_key(fmaxf(fabsf(vmax - med), fabsf(vmin - med)));
      }
      st.rank = (total - 1) / 2;
      st.count = total;
      st.shift = range_shift(st.lo, st.hi);
      st.done = st.lo == st.hi;
    }
    __syncthreads();
    bool kept = false;        // the keys of the current range sit in `keep`
    bool no_copy = false;     // a copy pass overflowed: bin the whole map instead
    for (int round = 0; round < 12; ++round) {
      const RangeState r = st;   // the same in every CTA
      if (r.done) break;
      if (!kept && !no_copy && r.count <= kCollectAll) {
        // copy pass: the keys inside [lo, hi] into this CTA's shared memory
        if (tid == 0) {
          nkeep = 0;
          overflow = 0;
        }
        __syncthreads();
        for_keys(mad, med, [&](uint32_t key) {
          if (key >= r.lo && key <= r.hi) {
            const unsigned at = atomicAdd(&nkeep, 1u);
            if (at < (unsigned)kCollectPerCta) keep[at] = key;
            else overflow = 1u;
          }
        });
        cl.sync();         // every CTA's copy and overflow flag are final
        unsigned any = 0;
        for (int c = 0; c < kClusterCtas; ++c) any |= *cl.map_shared_rank(&overflow, c);
        kept = any == 0;   // the same decision in every CTA
        no_copy = !kept;
        // (the flags are next written in the MAD's copy pass, after further
        // cluster barriers, so no barrier is needed before moving on)
        continue;
      }
      unsigned* h = hist[buf];
      unsigned* co = coarse[buf];
      for (int b = tid; b < kClusterBins; b += blockDim.x) h[b] = 0;
      __syncthreads();
      auto bin = [&](uint32_t key) {
        if (key >= r.lo && key <= r.hi) atomicAdd(&h[(unsigned)((key - r.lo) >> r.shift)], 1u);
      };
      if (kept) {
        const unsigned m = nkeep;
        for (unsigned i = tid; i < m; i += blockDim.x) bin(keep[i]);
      } else {
        for_keys(mad, med, bin);
      }
      __syncthreads();
      // coarse counts: 4 threads per coarse bin of 64 fine bins
      {
        const int c = tid >> 2, part = tid & 3;
        unsigned sum = 0;
#pragma unroll 4
        for (int i = 0; i < 16; ++i) sum += h[c * 64 + part * 16 + i];
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        if (part == 0) co[c] = sum;
      }
      cl.sync();           // every CTA's histogram and coarse counts are complete
      // the cluster's coarse counts, then the fine counts inside the coarse bin
      if (tid < kCoarse) {
        unsigned t = 0;
        for (int c = 0; c < kClusterCtas; ++c) t += cl.map_shared_rank(co, c)[tid];
        sum64[tid] = t;
      }
      __syncthreads();
      int cbin;
      unsigned long long cbelow;
      unsigned csize;
      if (warp == 0) {
        warp_find64(sum64, r.rank, &cbin, &cbelow, &csize);
        if (lane == 0) {
          red[0][0] = (unsigned long long)cbin;
          red[0][1] = cbelow;
        }
      }
      __syncthreads();
      cbin = (int)red[0][0];
      cbelow = red[0][1];
      if (tid < kCoarse) {
        unsigned t = 0;
        for (int c = 0; c < kClusterCtas; ++c) t += cl.map_shared_rank(h, c)[cbin * 64 + tid];
        sum64[tid] = t;
      }
      __syncthreads();
      if (warp == 0) {
        int fbin;
        unsigned long long fbelow;
        unsigned fsize;
        warp_find64(sum64, r.rank - cbelow, &fbin, &fbelow, &fsize);
        if (lane == 0) {
          const unsigned long long b = (unsigned long long)(cbin * 64 + fbin);
          const unsigned long long lo = r.lo + (b << r.shift);
          const unsigned long long hi = min(r.hi, lo + ((1ull << r.shift) - 1));
          st.lo = lo;
          st.hi = hi;
          st.rank = r.rank - cbelow - fbelow;
          st.count = fsize;
          st.shift = range_shift(lo, hi);
          st.done = lo == hi;
        }
      }
      __syncthreads();     // the new range is visible to the whole CTA
      buf ^= 1;
    }
    const float val = f32_from_key((uint32_t)st.lo);
    if (mad == 0) {
      med = val;
      if (rank == 0 && tid == 0) cs[2 * g] = (double)val;
    } else if (rank == 0 && tid == 0) {
      cs[2 * g + 1] = kMadToSigma * (double)val;
    }
    __syncthreads();       // everyone has read st before it is reset
  }
  cl.sync();               // nobody leaves while others may still read its histograms
}

// ---------------------------------------------------------------- MEDMAD, bracketed form
// One thread-block cluster of 8 CTAs per group, for maps of moderate size.
// The exact lower median and MAD are found with two passes over the map
// instead of one pass per radix digit:
//   * every CTA bins the same fixed, evenly spread sample of the group (up to
//     288 runs of 32 consecutive values) twice -- over the sample's key range,
//     then over the bins holding the targets -- and so finds the same sample
//     quantiles A <= B at ranks 1/2 -+ delta of the sample;
//   * one pass, each CTA over its share, counts the finite values and the
//     keys below A, and copies the keys in [A, B] into its shared memory;
//   * if the median's rank lies among the copies of the cluster, rounds of
//     2048-bin histograms over the copies (summed over the cluster through
//     distributed shared memory) select it exactly;
//   * the same sample as keys of |v - median| (FP32, the exact median) gives
//     the MAD's bracket [m_lo, m_hi]; a second pass counts the values with
//     |v - median| <= m_lo and copies those strictly between, and the MAD is
//     selected among the copies the same way.
// Every count is exact, so the result is the element a sort would give; the
// sample only decides how much is copied.  When a bracket misses its rank or
// the copies do not fit, the group is marked (scale -1) and the multi-pass
// cluster kernel above, launched next, computes it instead.
constexpr int kFastThreads = 256;
constexpr int kFastWarps = kFastThreads / 32;
constexpr int kFastBins = 2048;                    // 64 coarse bins of 32
constexpr int kFastPool = 9 * 1024;                // keys copied per CTA
constexpr int kFastRuns = kFastPool / 32;          // sample runs of 32 values
constexpr int64_t kFastMaxPerGroup = 2 << 20;
constexpr uint32_t kFinLo = 0x00800000u;   // key of -FLT_MAX
constexpr uint32_t kFinHi = 0xff7fffffu;   // key of +FLT_MAX
constexpr uint32_t kNoKey = 0xffffffffu;   // above every finite key (a NaN's)

// Finiteness from the exponent bits (an integer test, so that no floating-
// point rewriting of NaN or infinity can change which values are ranked).
__device__ __forceinline__ bool finite_bits(float x) {
  return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

struct FastFind {
  unsigned long long below;   // keys before the bin
  unsigned bin, size;
};

__device__ __forceinline__ unsigned fast_shift(unsigned long long lo, unsigned long long hi) {
  const unsigned long long width = hi - lo + 1;   // <= 2^32
  unsigned s = 0;
  while ((width - 1) >> s >= (unsigned long long)kFastBins) ++s;
  return s;
}

// Exclusive scan of one CTA's 2048 bins (eight per thread); returns, for
// each of up to three ranks, the bin holding it.  Every thread must call it.
__device__ void fast_find(const unsigned* h, const unsigned long long* rank, int nr, FastFind* out,
                          unsigned long long* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned c[8];
  unsigned mine = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    c[i] = h[8 * tid + i];
    mine += c[i];
  }
  unsigned long long incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  unsigned long long before = incl - mine;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  for (int r = 0; r < nr; ++r) {
    const unsigned long long k = rank[r];
    if (k >= before && k < before + mine) {
      unsigned long long cum = before;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (k >= cum && k < cum + c[i]) out[r] = FastFind{cum, (unsigned)(8 * tid + i), c[i]};
        cum += c[i];
      }
    }
  }
  __syncthreads();
}

// Sample quantiles of the n keys in pool (range [kmin, kmax]) at ranks
// t[0] <= t[nt-1]: a histogram over the whole range, then one over the bins
// holding the first and last target.  Returns the lower edge of the first
// target's final bin and the upper edge of the last one's.  CTA-local.
__device__ void fast_quantiles(const uint32_t* pool, unsigned n, unsigned kmin, unsigned kmax,
                               const unsigned long long* t, int nt, unsigned* hist,
                               unsigned long long* wsum, FastFind* res, uint32_t* qlo,
                               uint32_t* qhi) {
  unsigned long long lo = kmin, hi = kmax;
  unsigned long long rk[2] = {t[0], t[nt - 1]};
  for (int round = 0; round < 2; ++round) {
    const unsigned sh = fast_shift(lo, hi);
    for (int b = threadIdx.x; b < kFastBins; b += kFastThreads) hist[b] = 0;
    if (threadIdx.x < 2) res[threadIdx.x] = FastFind{0ull, 0u, 0u};
    __syncthreads();
    for (unsigned i = threadIdx.x; i < n; i += kFastThreads) {
      const uint32_t k = pool[i];
      if (k >= lo && k <= hi) atomicAdd(&hist[(unsigned)((k - lo) >> sh)], 1u);
    }
    __syncthreads();
    fast_find(hist, rk, 2, res, wsum);
    const FastFind f0 = res[0], f1 = res[1];
    const unsigned long long nlo = lo + ((unsigned long long)f0.bin << sh);
    const unsigned long long nhi = min(hi, lo + ((unsigned long long)f1.bin << sh) + ((1ull << sh) - 1));
    rk[0] -= f0.below;
    rk[1] -= f0.below;
    lo = nlo;
    hi = nhi;
    __syncthreads();   // res and hist are rewritten next round
  }
  *qlo = (uint32_t)lo;
  *qhi = (uint32_t)hi;
}

// Sample ranks 1/2 -+ delta of n sample keys (delta = 4.5 standard errors of
// a sample median, counting each run of 32 values as half as informative).
__device__ __forceinline__ void fast_targets(unsigned ns, unsigned long long* t) {
  const double d = 4.5 * 0.5 / sqrt(0.5 * (double)ns) + 1.0 / (double)ns;
  const double m = (double)(ns - 1);
  const double a = floor((0.5 - d) * m), b = ceil((0.5 + d) * m);
  t[0] = a < 0.0 ? 0ull : (unsigned long long)a;
  t[1] = b > m ? (unsigned long long)m : (unsigned long long)b;
}

// Warp 0: the entry of 32 counts (one per lane) holding `rank`.
__device__ __forceinline__ void warp_find32(unsigned c, unsigned long long rank, int* entry,
                                            unsigned long long* below, unsigned* size) {
  const int lane = threadIdx.x & 31;
  unsigned long long incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned long long excl = incl - c;
  const bool hit = rank >= excl && rank < incl;
  const unsigned who = __ballot_sync(0xffffffffu, hit);
  const int src = who ? __ffs(who) - 1 : 0;
  *entry = src;
  *below = __shfl_sync(0xffffffffu, excl, src);
  *size = __shfl_sync(0xffffffffu, c, src);
}

template <bool VEC>
__global__ void __launch_bounds__(kFastThreads, 4) k_medmad_fast(const float* __restrict__ vals,
                                                                 int64_t stride, int64_t n, int g0,
                                                                 double* cs,
                                                                 unsigned long long* invalid) {
  __shared__ uint32_t pool[kFastPool];
  __shared__ unsigned hist[2][kFastBins];
  __shared__ unsigned coarse[2][64];
  __shared__ unsigned sum64[64];
  __shared__ unsigned long long wsum[kFastWarps];
  __shared__ FastFind res[2];
  __shared__ unsigned cnt, kmin, kmax;
  __shared__ unsigned long long mine[3];   // this CTA's pass counts: finite, low, copies
  __shared__ unsigned long long sel[3];    // cluster selection state: lo, hi, rank
  cg::cluster_group cl = cg::this_cluster();
  const unsigned crank = cl.block_rank();
  const int g = g0 + blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* v = vals + (size_t)g * stride;
  const int64_t nv = VEC ? stride / 4 : stride;
  // sample slots: one run of 32 values per 32 slots
  const unsigned slots = 32u * (unsigned)min((stride + 31) / 32, (int64_t)kFastRuns);
  int buf = 0;

  auto reset = [&]() {
    if (tid == 0) {
      cnt = 0;
      kmin = 0xffffffffu;
      kmax = 0;
      mine[0] = mine[1] = mine[2] = 0;
    }
    __syncthreads();
  };
  // the sample (the same runs in every CTA) as keys of v or of |v - med|:
  // run c fills slots 32c .. 32c+31; a value that is not finite leaves key 0,
  // below every finite key, which the ranges of the quantile rounds exclude
  auto sample = [&](bool mad, float med) -> unsigned {
    const int64_t runs = (stride + 31) / 32;
    const int64_t use = runs < kFastRuns ? runs : kFastRuns;
    unsigned lmin = 0xffffffffu, lmax = 0u, nfin = 0;
    for (int64_t c = warp; c < use; c += kFastWarps) {   // every run into L2 first
      const int64_t i = (c * runs / use) * 32 + lane;
      if (i < stride) asm volatile("prefetch.global.L2 [%0];" ::"l"((const void*)(v + i)));
    }
    constexpr int B = 12;
    for (int64_t c0 = warp; c0 < use; c0 += B * kFastWarps) {
      float x[B];
      bool in[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int64_t c = c0 + b * kFastWarps;
        const int64_t i = (c * runs / use) * 32 + lane;
        in[b] = c < use && i < stride;
        x[b] = in[b] ? v[i] : 0.f;
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int64_t c = c0 + b * kFastWarps;
        const float y = mad ? fabsf(x[b] - med) : x[b];
        const bool ok = in[b] && finite_bits(x[b]) && finite_bits(y);
        const uint32_t key = ok ? f32_key(y) : 0u;
        if (c < use) pool[c * 32 + lane] = key;
        if (ok) {
          lmin = min(lmin, key);
          lmax = max(lmax, key);
          ++nfin;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
      lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
      nfin += __shfl_xor_sync(0xffffffffu, nfin, o);
    }
    if (lane == 0) {
      atomicMin(&kmin, lmin);
      atomicMax(&kmax, lmax);
      atomicAdd(&cnt, nfin);
    }
    __syncthreads();
    return cnt;
  };
  // One pass over this CTA's share.  keyof(x) maps a value to the key that is
  // ranked (the key of v, or of |v - median|); over keys, the finite values
  // are exactly [kFinLo, kFinHi], so a key below `low` (finite) is counted and
  // a key in [clo, chi] (finite) is copied.  Each thread counts its copies of
  // a batch first, so a warp reserves their slots with one atomic.  The
  // cluster's totals of (finite, low, copies) are returned in tot.
  auto pass = [&](auto&& keyof, uint32_t low, uint32_t clo, uint32_t chi,
                  unsigned long long* tot) {
    unsigned nf = 0, c0 = 0;
    constexpr int U = VEC ? 3 : 8;   // vectors per batch (registers allow 12 keys)
    constexpr int E = VEC ? 4 * U : U;
    constexpr int NV = VEC ? 4 : 1;
    const int step = kClusterCtas * kFastThreads;
    const int nvi = (int)nv;
    const uint32_t cw = chi - clo;
    // one batch of raw values; the next batch is loaded before the current one
    // is classified, so that two batches of loads overlap the work
    float cur[E], nxt[E];
    auto load = [&](float (&x)[E], int w0) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = w0 + lane + u * step;
        if (VEC) {
          const float4 q = i < nvi ? reinterpret_cast<const float4*>(v)[i]
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
          x[4 * u] = q.x;
          x[4 * u + 1] = q.y;
          x[4 * u + 2] = q.z;
          x[4 * u + 3] = q.w;
        } else {
          x[u] = i < nvi ? v[i] : 0.f;
        }
      }
    };
    // the trip count depends on the warp only (the shuffles below need every lane)
    int w0 = (int)crank * kFastThreads + warp * 32;
    if (w0 < nvi) load(cur, w0);
    for (; w0 < nvi; w0 += U * step) {
      const int wn = w0 + U * step;
      if (wn < nvi) load(nxt, wn);
      uint32_t key[E];
      // slots past the end take kNoKey, which no class contains
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = w0 + lane + (e / NV) * step;
        key[e] = i < nvi ? keyof(cur[e]) : kNoKey;
      }
      unsigned ncp = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const bool fin = key[e] - kFinLo <= kFinHi - kFinLo;
        nf += fin;
        c0 += fin && key[e] < low;
        ncp += key[e] - clo <= cw;
      }
      unsigned incl = ncp;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned wtot = __shfl_sync(0xffffffffu, incl, 31);
      if (wtot) {   // warp-uniform
        unsigned base = 0;
        if (lane == 31) base = atomicAdd(&cnt, wtot);
        unsigned pos = __shfl_sync(0xffffffffu, base, 31) + incl - ncp;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const bool cp = key[e] - clo <= cw;
          if (cp && pos < (unsigned)kFastPool) pool[pos] = key[e];
          pos += cp;
        }
      }
#pragma unroll
      for (int e = 0; e < E; ++e) cur[e] = nxt[e];
    }
    unsigned long long nf64 = nf, c064 = c0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nf64 += __shfl_xor_sync(0xffffffffu, nf64, o);
      c064 += __shfl_xor_sync(0xffffffffu, c064, o);
    }
    if (lane == 0) {
      atomicAdd(&mine[0], nf64);
      atomicAdd(&mine[1], c064);
    }
    __syncthreads();
    if (tid == 0) mine[2] = cnt;
    cl.sync();   // every CTA's counts are final
    tot[0] = tot[1] = tot[2] = 0;
    bool over = false;
    for (int r = 0; r < kClusterCtas; ++r) {
      const unsigned long long* o = cl.map_shared_rank(mine, r);
      tot[0] += o[0];
      tot[1] += o[1];
      tot[2] += o[2];
      over |= o[2] > (unsigned long long)kFastPool;
    }
    if (over) tot[2] = ~0ull;   // a copy did not fit
  };
  // the rank-th smallest copy (counted from lo) of the cluster inside [lo, hi]
  auto select = [&](unsigned long long lo, unsigned long long hi, unsigned long long rank) {
    const unsigned n = min(cnt, (unsigned)kFastPool);
    for (int round = 0; round < 8 && lo < hi; ++round) {
      const unsigned sh = fast_shift(lo, hi);
      unsigned* h = hist[buf];
      unsigned* co = coarse[buf];
      for (int b = tid; b < kFastBins; b += kFastThreads) h[b] = 0;
      __syncthreads();
      for (unsigned i = tid; i < n; i += kFastThreads) {
        const uint32_t k = pool[i];
        if (k >= lo && k <= hi) atomicAdd(&h[(unsigned)((k - lo) >> sh)], 1u);
      }
      __syncthreads();
      {
        const int c = tid >> 2, part = tid & 3;   // 64 coarse bins of 32
        unsigned sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) sum += h[c * 32 + part * 8 + i];
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        if (part == 0) co[c] = sum;
      }
      cl.sync();   // every CTA's histogram and coarse counts are complete
      if (tid < 64) {
        unsigned t = 0;
        for (int r = 0; r < kClusterCtas; ++r) t += cl.map_shared_rank(co, r)[tid];
        sum64[tid] = t;
      }
      __syncthreads();
      if (warp == 0) {
        int cbin;
        unsigned long long cbelow;
        unsigned csize;
        warp_find64(sum64, rank, &cbin, &cbelow, &csize);
        unsigned f = 0;
        for (int r = 0; r < kClusterCtas; ++r) f += cl.map_shared_rank(h, r)[cbin * 32 + lane];
        int fbin;
        unsigned long long fbelow;
        unsigned fsize;
        warp_find32(f, rank - cbelow, &fbin, &fbelow, &fsize);
        if (lane == 0) {
          const unsigned long long nlo = lo + ((unsigned long long)(cbin * 32 + fbin) << sh);
          sel[0] = nlo;
          sel[1] = min(hi, nlo + ((1ull << sh) - 1));
          sel[2] = rank - cbelow - fbelow;
        }
      }
      __syncthreads();
      lo = sel[0];
      hi = sel[1];
      rank = sel[2];
      __syncthreads();   // sel is rewritten next round
      buf ^= 1;
    }
    return (uint32_t)lo;
  };
  auto leave = [&](bool fail) {
    if (fail && crank == 0 && tid == 0) cs[2 * g + 1] = -1.0;   // the cluster kernel takes it
    cl.sync();   // nobody leaves while others may still read its shared memory
  };

  // ---- median bracket from the sample (the same in every CTA)
  reset();
  unsigned ns = sample(false, 0.f);
  uint32_t kA = 0, kB = 0;
  if (ns > 0) {
    unsigned long long t[2];
    fast_targets(ns, t);
    fast_quantiles(pool, slots, kmin, kmax, t, 2, hist[1], wsum, res, &kA, &kB);
  }
  // ---- pass 1: finite count, keys below A, copies of [A, B]
  reset();
  unsigned long long tot[3];
  pass([](float x) { return f32_key(x); }, kA, kA, kB, tot);
  const unsigned long long nf = tot[0];
  if (nf == 0) {
    if (crank == 0 && tid == 0) {
      cs[2 * g] = NAN;
      cs[2 * g + 1] = 0.0;
      if (invalid && n > 0) atomicAdd(invalid, (unsigned long long)n);
    }
    leave(false);
    return;
  }
  const unsigned long long R = (nf - 1) / 2;
  if (ns == 0 || tot[2] == ~0ull || R < tot[1] || R >= tot[1] + tot[2]) {
    leave(true);
    return;
  }
  const float med = f32_from_key(select(kA, kB, R - tot[1]));
  // ---- MAD bracket from the sample of |v - median|
  cl.sync();   // every CTA is done with its copies before they are replaced
  reset();
  ns = sample(true, med);
  uint32_t mlo = 0, mhi = 0xffffffffu;
  if (ns > 0) {
    unsigned long long t[2];
    fast_targets(ns, t);
    fast_quantiles(pool, slots, kmin, kmax, t, 2, hist[buf], wsum, res, &mlo, &mhi);
  }
  // ---- pass 2: |v - median| <= m_lo counted, (m_lo, m_hi) copied
  cl.sync();   // no CTA still reads the previous counts
  if (ns == 0 || mhi <= mlo + 1u) {   // no key strictly inside: the bracket cannot hold the MAD
    leave(true);
    return;
  }
  reset();
  pass([&](float x) { return finite_bits(x) ? f32_key(fabsf(x - med)) : kNoKey; }, mlo + 1,
       mlo + 1, mhi - 1, tot);
  if (ns == 0 || tot[2] == ~0ull || R < tot[1] || R >= tot[1] + tot[2]) {
    leave(true);
    return;
  }
  const float mad = f32_from_key(select((unsigned long long)mlo + 1, (unsigned long long)mhi - 1,
                                        R - tot[1]));
  if (crank == 0 && tid == 0) {
    cs[2 * g] = (double)med;
    cs[2 * g + 1] = kMadToSigma * (double)mad;
    if (invalid && (int64_t)nf < n) atomicAdd(invalid, (unsigned long long)(n - (int64_t)nf));
  }
  leave(false);
}

template <bool VEC>
static cudaError_t launch_fast_t(const float* vals, int groups, int64_t stride, int64_t n,
                                 double* cs, unsigned long long* invalid, cudaStream_t st) {
  for (int g0 = 0; g0 < groups; g0 += 65535) {
    const int gb = std::min(65535, groups - g0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas, gb, 1);
    cfg.blockDim = dim3(kFastThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_medmad_fast<VEC>, vals, stride, n, g0, cs, invalid);
    count_launches(1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t launch_medmad_cluster(const float* vals, int groups, int64_t stride,
                                         int64_t n, bool vec, double* cs,
                                         unsigned long long* invalid, int skip_done,
                                         cudaStream_t st) {
  for (int g0 = 0; g0 < groups; g0 += 65535) {
    const int gb = std::min(65535, groups - g0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas, gb, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // starts with pdl_begin()
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    const cudaError_t e =
        vec ? cudaLaunchKernelEx(&cfg, k_medmad_cluster<true>, vals, stride, n, g0, cs, invalid,
                                 skip_done)
            : cudaLaunchKernelEx(&cfg, k_medmad_cluster<false>, vals, stride, n, g0, cs, invalid,
                                 skip_done);
    count_launches(1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- MEDMAD, split form
// For plans, which own scratch memory: the bracketed selection above with its
// pieces in separate launches, so that the passes over the maps run on every
// SM at memory bandwidth instead of in one 8-CTA cluster per map:
//   1. k_split_bracket (one CTA per map): a fixed, evenly spread sample of up
//      to kSplitRuns runs of 32 values; two histogram rounds over the sample
//      keys give quantiles A <= B at ranks 1/2 -+ delta, which bracket the
//      median;
//   2. k_split_pass (one CTA per chunk of kSplitChunk values): counts the
//      finite values and the keys below A, and writes the keys in [A, B] into
//      the chunk's own slot of the copy buffer, counting them in a 2048-bin
//      histogram over [A, B].  A chunk's counts go to its own entry of a count
//      array, so a CTA waits on no global atomic: its loads are issued first
//      (beside the read of the map's state) and one barrier places its warps'
//      copies;
//   3. k_split_select (one CTA per map): sums the chunks' counts; the
//      histogram gives the bin holding the median's rank; the copies inside
//      that bin are gathered into shared memory and the median is selected
//      among them exactly; the same sample as keys of |v - median| (FP32)
//      then brackets the MAD as (m_lo, m_hi);
//   4. k_split_pass again on the keys of |v - median| (those <= m_lo counted,
//      those strictly inside the bracket copied) and 5. k_split_select for the
//      MAD.
// Every count is exact, so the results are the elements a sort gives; the
// sample only decides how much is copied.  A map whose bracket misses its
// rank, a chunk of which has more copies than its slot holds, or whose rank
// bin holds too many copies is marked (scale -1) and the cluster kernel,
// launched last, finishes it.
constexpr int kSplitRuns = 512;
constexpr int kSplitPool = kSplitRuns * 32;     // sample keys (64 KB of shared memory)
constexpr int kSplitChunk = 4096;               // values per CTA of a pass
constexpr int kSplitSlot = 1024;                // copies a chunk keeps (a quarter of its values)
constexpr int kSplitMaxChunks = (int)(kFastMaxPerGroup / kSplitChunk);
constexpr int kSplitPassThreads = 128;
constexpr int kSplitThreads = 1024;             // bracket and select kernels
constexpr int kSplitBins = 2048;
constexpr int kSplitGather = 8192;              // copies of the rank's bin kept in shared memory
static_assert(kSplitMaxChunks <= kSplitThreads, "one chunk count per select thread");

struct SplitState {
  uint32_t lo, hi;     // copy range of the current pass (inclusive keys)
  uint32_t nfin;       // finite values (set by the median's select)
  uint32_t stage;      // 0: median pass, 1: MAD pass, 2: finished, 3: left to the cluster form
  float med;
  uint32_t nsample;    // finite sample values
  uint32_t pad[2];
};
static_assert(sizeof(SplitState) == 32, "SplitState layout");

static int split_chunks(int64_t stride) { return (int)((stride + kSplitChunk - 1) / kSplitChunk); }

static size_t split_head(int groups) {
  return ((size_t)groups * (sizeof(SplitState) + kSplitBins * sizeof(unsigned)) + 255) / 256 * 256;
}

size_t noise_split_bytes(int groups, int64_t stride) {
  if (stride > kFastMaxPerGroup || groups > 65535) return 0;
  const size_t nc = (size_t)groups * (size_t)split_chunks(stride);
  return split_head(groups) + nc * sizeof(uint4) + nc * kSplitSlot * sizeof(uint32_t);
}

void noise_split_carve(void* base, int groups, int64_t stride, NoiseScratch* s) {
  s->split = noise_split_bytes(groups, stride) ? base : nullptr;
  s->split_cap = s->split ? (int64_t)split_chunks(stride) * kSplitSlot : 0;
}

struct SplitPtrs {
  SplitState* st;
  unsigned* hist;      // [groups][kSplitBins]
  uint4* cnt;          // [groups][nchunk]: keys below lo, finite values, copies (unclipped)
  uint32_t* copies;    // [groups][nchunk][kSplitSlot]
  int nchunk;
};

static SplitPtrs split_ptrs(void* base, int groups, int64_t stride) {
  char* p = static_cast<char*>(base);
  SplitPtrs r;
  r.nchunk = split_chunks(stride);
  r.st = reinterpret_cast<SplitState*>(p);
  r.hist = reinterpret_cast<unsigned*>(p + (size_t)groups * sizeof(SplitState));
  p += split_head(groups);
  r.cnt = reinterpret_cast<uint4*>(p);
  p += (size_t)groups * r.nchunk * sizeof(uint4);
  r.copies = reinterpret_cast<uint32_t*>(p);
  return r;
}

// Bin width (as a shift) of kSplitBins bins over the inclusive key range
// [lo, hi] (0 for an empty range, which holds no key).
static_assert(kSplitBins == 2048, "split_shift assumes 11-bit bins");
__device__ __forceinline__ unsigned split_shift(uint32_t lo, uint32_t hi) {
  if (hi < lo) return 0;
  const uint32_t top = (hi - lo) >> 11;   // span >> s < 2048  <=>  s >= bit length of (span >> 11)
  return top ? 32u - (unsigned)__clz(top) : 0u;
}

// Block-wide (kSplitThreads): the bin of h[0..kSplitBins) holding `rank`
// and the count before it.  Every thread must call it; the result is in
// every thread.  Returns false when the rank lies beyond the total.
__device__ bool split_find(const unsigned* h, unsigned long long rank, unsigned* bin,
                           unsigned long long* below, unsigned long long* wsum,
                           unsigned long long* found) {
  constexpr int per = kSplitBins / kSplitThreads;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned c[per];
  unsigned long long mine = 0;
#pragma unroll
  for (int i = 0; i < per; ++i) {
    c[i] = h[per * tid + i];
    mine += c[i];
  }
  unsigned long long incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  if (tid == 0) found[0] = ~0ull;
  __syncthreads();
  // the warps before this one, summed across the lanes
  unsigned long long ws = lane < warp ? wsum[lane] : 0ull;
#pragma unroll
  for (int o = 16; o; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
  const unsigned long long before = incl - mine + ws;
  if (rank >= before && rank < before + mine) {
    unsigned long long cum = before;
#pragma unroll
    for (int i = 0; i < per; ++i) {
      if (rank >= cum && rank < cum + c[i]) {
        found[0] = (unsigned long long)(per * tid + i);
        found[1] = cum;
      }
      cum += c[i];
    }
  }
  __syncthreads();
  const bool ok = found[0] != ~0ull;
  *bin = (unsigned)found[0];
  *below = found[1];
  __syncthreads();   // found and wsum are reused by the next call
  return ok;
}

// The sample: up to kSplitRuns runs of 32 consecutive values, evenly spread
// over the map (the same runs in every call), as keys of v (mad = false) or
// of |v - med| in FP32.  A value that is not finite leaves key 0, below every
// finite key.  Returns the number of finite sample values; kminmax gets their
// smallest and largest key.  Every thread must call it.
__device__ unsigned split_sample(const float* v, int64_t stride, bool mad, float med,
                                 uint32_t* pool, unsigned* slots, uint32_t* kminmax,
                                 unsigned* nfin_sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = kSplitThreads / 32;
  constexpr int per_warp = kSplitRuns / nwarps;   // runs a warp reads (16)
  static_assert(per_warp <= 32, "one run start per lane");
  // the split form takes maps of at most 2 Mi values, so 32-bit arithmetic
  // holds c * runs; lane l of warp w computes the start of run w + 32 l once
  // (no division per run)
  const uint32_t runs = (uint32_t)((stride + 31) / 32);
  const uint32_t use = runs < (uint32_t)kSplitRuns ? runs : (uint32_t)kSplitRuns;
  const uint32_t cl = (uint32_t)warp + (uint32_t)nwarps * (uint32_t)lane;
  const uint32_t start = cl < use ? cl * runs / use * 32u : 0u;
  if (tid == 0) {
    kminmax[0] = 0xffffffffu;
    kminmax[1] = 0u;
    *nfin_sh = 0;
    *slots = use * 32u;
  }
  for (int k = 0; k < per_warp; ++k) {   // every run into L2 first
    const uint32_t c = (uint32_t)warp + (uint32_t)nwarps * (uint32_t)k;
    const int64_t i = (int64_t)__shfl_sync(0xffffffffu, start, k) + lane;
    if (c < use && i < stride) asm volatile("prefetch.global.L2 [%0];" ::"l"((const void*)(v + i)));
  }
  __syncthreads();
  uint32_t lmin = 0xffffffffu, lmax = 0u;
  unsigned nf = 0;
  constexpr int B = 8;
  for (int k0 = 0; k0 < per_warp; k0 += B) {
    const int64_t c0 = warp + (int64_t)nwarps * k0;
    float x[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int64_t c = c0 + (int64_t)b * nwarps;
      const int64_t i = (int64_t)__shfl_sync(0xffffffffu, start, k0 + b) + lane;
      x[b] = (c < use && i < stride) ? v[i] : NAN;
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int64_t c = c0 + (int64_t)b * nwarps;
      if (c >= use) break;
      uint32_t key = 0;
      if (finite_bits(x[b])) {
        key = mad ? f32_key(fabsf(x[b] - med)) : f32_key(x[b]);
        lmin = min(lmin, key);
        lmax = max(lmax, key);
        ++nf;
      }
      pool[c * 32 + lane] = key;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    nf += __shfl_xor_sync(0xffffffffu, nf, o);
  }
  if (lane == 0) {
    atomicMin(&kminmax[0], lmin);
    atomicMax(&kminmax[1], lmax);
    atomicAdd(nfin_sh, nf);
  }
  __syncthreads();
  return *nfin_sh;
}

// Sample ranks 1/2 -+ delta of ns sample values (delta = 4.5 standard errors of
// a sample median, a run of 32 values counting as half as informative).
// The ranks only decide how much the passes copy, so FP32 is enough (FP64 is
// slow on this part, and every thread evaluates this).
__device__ __forceinline__ void split_targets(unsigned ns, unsigned long long* t) {
  const float d = 4.5f * 0.5f * rsqrtf(0.5f * (float)ns) + 1.0f / (float)ns;
  const float m = (float)(ns - 1);
  const float a = floorf((0.5f - d) * m), b = ceilf((0.5f + d) * m);
  t[0] = a < 0.f ? 0ull : (unsigned long long)a;
  t[1] = b > m ? (unsigned long long)(ns - 1) : (unsigned long long)b;
}

// Sample quantiles at ranks t[0] <= t[1] among the finite sample keys (range
// [kmin, kmax]): one histogram over the range, one over the bins holding the
// two targets; returns the lower edge of t[0]'s final bin and the upper edge
// of t[1]'s.  Every thread must call it.
__device__ void split_quantiles(const uint32_t* pool, unsigned slots, uint32_t kmin, uint32_t kmax,
                                const unsigned long long* t, unsigned* hist,
                                unsigned long long* wsum, unsigned long long* found,
                                uint32_t* qlo, uint32_t* qhi) {
  uint32_t lo = kmin, hi = kmax;
  unsigned long long r0 = t[0], r1 = t[1];
  for (int round = 0; round < 2; ++round) {
    const unsigned sh = split_shift(lo, hi);
    for (int b = threadIdx.x; b < kSplitBins; b += kSplitThreads) hist[b] = 0;
    __syncthreads();
    for (unsigned i = threadIdx.x; i < slots; i += kSplitThreads) {
      const uint32_t k = pool[i];
      if (k >= lo && k <= hi) atomicAdd(&hist[(k - lo) >> sh], 1u);
    }
    __syncthreads();
    unsigned b0, b1;
    unsigned long long w0, w1;
    split_find(hist, r0, &b0, &w0, wsum, found);
    split_find(hist, r1, &b1, &w1, wsum, found);
    const uint32_t nlo = lo + (b0 << sh);
    const unsigned long long top = (unsigned long long)lo + ((unsigned long long)(b1 + 1) << sh) - 1;
    const uint32_t nhi = top < hi ? (uint32_t)top : hi;
    r0 -= w0;
    r1 -= w0;
    lo = nlo;
    hi = nhi;
    __syncthreads();
  }
  *qlo = lo;
  *qhi = hi;
}

// 1. The median's bracket from the sample; clears the map's counters and
// histogram.
__global__ void __launch_bounds__(kSplitThreads) k_split_bracket(const float* __restrict__ vals,
                                                                 int64_t stride, SplitState* st,
                                                                 unsigned* hist_g) {
  pdl_begin();
  extern __shared__ uint32_t spool[];   // kSplitPool
  __shared__ unsigned hist[kSplitBins];
  __shared__ unsigned long long wsum[kSplitThreads / 32], found[2];
  __shared__ uint32_t kmm[2];
  __shared__ unsigned slots, nfin;
  const int g = blockIdx.x;
  const float* v = vals + (size_t)g * stride;
  unsigned* hg = hist_g + (size_t)g * kSplitBins;
  for (int b = threadIdx.x; b < kSplitBins; b += kSplitThreads) hg[b] = 0;
  const unsigned ns = split_sample(v, stride, false, 0.f, spool, &slots, kmm, &nfin);
  uint32_t A = 1, B = 0;   // empty range when the sample has no finite value
  if (ns > 0) {
    unsigned long long t[2];
    split_targets(ns, t);
    split_quantiles(spool, slots, kmm[0], kmm[1], t, hist, wsum, found, &A, &B);
  }
  if (threadIdx.x == 0) {
    SplitState s;
    s.lo = A;
    s.hi = B;
    s.nfin = 0;
    s.stage = 0;
    s.med = 0.f;
    s.nsample = ns;
    s.pad[0] = s.pad[1] = 0u;
    st[g] = s;
  }
}

// 2./4. One chunk of one map: counts and copies (see above).  The chunk goes
// into shared memory by asynchronous copies (each thread its own 32 values,
// as eight 16-byte copies when VEC), so that a CTA holds its whole chunk in
// flight without registers and several CTAs per SM stream at once; the map's
// state is read while they land.  Each thread counts in registers and notes
// which of its values are copies in a bit mask; after a warp scan and one
// barrier it writes its copies into the chunk's slot.  Nothing is written
// for a map whose stage is not this pass's.
template <bool VEC, bool MAD>
__global__ void __launch_bounds__(kSplitPassThreads, 12) k_split_pass(const float* __restrict__ vals,
                                                                     int64_t stride,
                                                                     const SplitState* __restrict__ st,
                                                                     unsigned* hist_g, uint4* cnt,
                                                                     uint32_t* copies, int nchunk) {
  pdl_begin();
  constexpr int NW = kSplitPassThreads / 32;
  constexpr int U = kSplitChunk / kSplitPassThreads;   // values per thread (32)
  __shared__ __align__(16) float buf[kSplitChunk];
  __shared__ unsigned wsh[3][NW];   // per warp: copies, keys below lo, finite values
  const int g = blockIdx.y, c = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)c * kSplitChunk;
  const int64_t c1 = c0 + kSplitChunk < stride ? c0 + kSplitChunk : stride;
  const float* v = vals + (size_t)g * stride + c0;
  const int nv = (int)(c1 - c0);
  // value j of this thread sits at chunk offset off(j); the copy of an
  // offset past the map's end is a NaN written here instead
  auto off = [&](int j) -> int {
    return VEC ? ((j >> 2) * kSplitPassThreads + tid) * 4 + (j & 3) : j * kSplitPassThreads + tid;
  };
  if (VEC) {
    // chunk starts are multiples of kSplitChunk values and stride % 4 == 0,
    // so every 16-byte copy is aligned and lies wholly inside or outside
#pragma unroll
    for (int u = 0; u < U / 4; ++u) {
      const int o = off(4 * u);
      if (o < nv) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(buf + o)),
                     "l"(v + o)
                     : "memory");
      } else {
        *reinterpret_cast<float4*>(buf + o) = make_float4(NAN, NAN, NAN, NAN);
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int o = off(u);
      if (o < nv) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(buf + o)), "l"(v + o)
                     : "memory");
      } else {
        buf[o] = NAN;
      }
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  const SplitState s = st[g];   // read while the copies land
  const uint32_t lo = s.lo, hi = s.hi;
  const unsigned sh = split_shift(lo, hi);
  const float med = s.med;
  // order-preserving key from the bits (the same map as f32_key), kNoKey for
  // a value that is not finite; |v - med| is never negative, so its key is
  // its bits with the sign bit set
  auto key_of = [&](float e) -> uint32_t {
    const uint32_t bits = __float_as_uint(e);
    const bool f = (bits & 0x7f800000u) != 0x7f800000u;
    uint32_t key;
    if (MAD) key = __float_as_uint(fabsf(e - med)) | 0x80000000u;
    else key = bits ^ ((uint32_t)((int32_t)bits >> 31) | 0x80000000u);
    return f ? key : kNoKey;
  };
  // copies: lo <= key <= hi as one unsigned compare; an empty bracket (no
  // finite sample value: lo > hi) copies nothing
  const bool any = hi >= lo;
  const uint32_t span = any ? hi - lo : 0u;
  unsigned below = 0, fin = 0;
  uint32_t cmask = 0;
  asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's own copies
  auto classify = [&](float e, int j) {
    const uint32_t key = key_of(e);
    if (!MAD) fin += key != kNoKey;   // the MAD pass keeps the median pass's count
    below += key < lo;
    cmask |= (uint32_t)(any && key - lo <= span) << j;   // never a non-finite value (hi < kNoKey)
  };
  if (VEC) {
#pragma unroll
    for (int u = 0; u < U / 4; ++u) {
      const float4 q = *reinterpret_cast<const float4*>(buf + off(4 * u));
      classify(q.x, 4 * u);
      classify(q.y, 4 * u + 1);
      classify(q.z, 4 * u + 2);
      classify(q.w, 4 * u + 3);
    }
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u) classify(buf[off(u)], u);
  }
  const int nc = __popc(cmask);
  int incl = nc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    below += __shfl_xor_sync(0xffffffffu, below, o);
    if (!MAD) fin += __shfl_xor_sync(0xffffffffu, fin, o);
  }
  if (lane == 31) wsh[0][warp] = (unsigned)incl;
  if (lane == 0) {
    wsh[1][warp] = below;
    wsh[2][warp] = fin;
  }
  __syncthreads();
  if (s.stage != (MAD ? 1u : 0u)) return;   // finished, degenerate or handed on
  unsigned wbase = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const unsigned t = wsh[0][w];
    wbase += w < warp ? t : 0u;
    tot += t;
  }
  if (tid == 0) {
    unsigned tb = 0, tf = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      tb += wsh[1][w];
      tf += wsh[2][w];
    }
    cnt[(size_t)g * nchunk + c] = make_uint4(tb, tf, tot, 0u);
  }
  if (tot > (unsigned)kSplitSlot) return;   // the select hands this map on
  uint32_t* out = copies + ((size_t)g * nchunk + c) * kSplitSlot;
  unsigned* hg = hist_g + (size_t)g * kSplitBins;
  unsigned pos = wbase + (unsigned)(incl - nc);
  for (uint32_t m = cmask; m; m &= m - 1) {
    const uint32_t key = key_of(buf[off(__ffs(m) - 1)]);
    out[pos++] = key;
    atomicAdd(&hg[(key - lo) >> sh], 1u);
  }
}

// 3./5. Exact selection among the copies; after the median, the MAD's bracket.
template <bool MAD>
__global__ void __launch_bounds__(kSplitThreads) k_split_select(const float* __restrict__ vals,
                                                                int64_t stride, int64_t n,
                                                                SplitState* st, unsigned* hist_g,
                                                                const uint4* __restrict__ cnt,
                                                                const uint32_t* __restrict__ copies,
                                                                int nchunk, double* cs,
                                                                unsigned long long* invalid) {
  pdl_begin();
  extern __shared__ uint32_t spool[];   // kSplitPool (the sample, median stage), the gathered bin
  __shared__ unsigned hist[kSplitBins];
  __shared__ unsigned long long wsum[kSplitThreads / 32], found[2];
  __shared__ uint32_t kmm[2];
  __shared__ unsigned slots, nfin_sh, ngather;
  __shared__ unsigned ccount[kSplitMaxChunks];   // copies of each chunk (unclipped)
  __shared__ unsigned long long tsum[3];         // keys below lo, finite values, copies
  __shared__ unsigned tover;                     // a chunk overflowed its slot
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SplitState s = st[g];
  if (s.stage != (MAD ? 1u : 0u)) return;
  unsigned* hg = hist_g + (size_t)g * kSplitBins;
  auto hand_on = [&]() {   // the cluster kernel computes this map
    if (tid == 0) {
      cs[2 * g + 1] = -1.0;
      st[g].stage = 3;
    }
  };
  // the chunks' counts (and the pass histogram, read beside them)
  if (tid == 0) {
    tsum[0] = tsum[1] = tsum[2] = 0ull;
    tover = 0u;
    ngather = 0u;
  }
  for (int b = tid; b < kSplitBins; b += kSplitThreads) hist[b] = hg[b];
  uint4 q = make_uint4(0u, 0u, 0u, 0u);
  if (tid < nchunk) {
    q = cnt[(size_t)g * nchunk + tid];
    ccount[tid] = q.z;
  }
  unsigned long long cb = q.x, cf = q.y, cc = q.z;
  unsigned over = q.z > (unsigned)kSplitSlot;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    cb += __shfl_xor_sync(0xffffffffu, cb, o);
    cf += __shfl_xor_sync(0xffffffffu, cf, o);
    cc += __shfl_xor_sync(0xffffffffu, cc, o);
    over |= __shfl_xor_sync(0xffffffffu, over, o);
  }
  __syncthreads();   // tsum and tover are initialised
  if (lane == 0 && warp * 32 < nchunk) {
    atomicAdd(&tsum[0], cb);
    atomicAdd(&tsum[1], cf);
    atomicAdd(&tsum[2], cc);
    if (over) atomicOr(&tover, 1u);
  }
  __syncthreads();
  const unsigned long long nbelow = tsum[0], ncopy = tsum[2];
  const unsigned nfin = MAD ? s.nfin : (unsigned)tsum[1];
  if (!MAD && nfin == 0) {
    if (tid == 0) {
      cs[2 * g] = NAN;
      cs[2 * g + 1] = 0.0;
      if (invalid && n > 0) atomicAdd(invalid, (unsigned long long)n);
      st[g].stage = 2;
    }
    return;
  }
  const unsigned long long R = (nfin - 1) / 2;
  if (s.nsample == 0 || tover || R < nbelow || R >= nbelow + ncopy) {
    hand_on();
    return;
  }
  // the bin of the pass histogram holding the rank, then its copies
  unsigned long long rank = R - nbelow;
  const unsigned sh = split_shift(s.lo, s.hi);
  unsigned bin;
  unsigned long long below;
  if (!split_find(hist, rank, &bin, &below, wsum, found)) {
    hand_on();
    return;
  }
  rank -= below;
  uint32_t lo = s.lo + (bin << sh);
  const unsigned long long top = (unsigned long long)lo + (1ull << sh) - 1;
  uint32_t hi = top < s.hi ? (uint32_t)top : s.hi;
  // one warp per chunk slot, eight loads in flight per lane
  constexpr int GB = 8;
  for (int c = warp; c < nchunk; c += kSplitThreads / 32) {
    const unsigned nc = ccount[c];
    const uint32_t* cp = copies + ((size_t)g * nchunk + c) * kSplitSlot;
    for (unsigned j0 = lane; j0 < nc; j0 += GB * 32) {
      uint32_t k[GB];
#pragma unroll
      for (int b = 0; b < GB; ++b) {
        const unsigned j = j0 + b * 32;
        k[b] = j < nc ? cp[j] : 1u;
      }
#pragma unroll
      for (int b = 0; b < GB; ++b) {
        const unsigned j = j0 + b * 32;
        if (j < nc && k[b] >= lo && k[b] <= hi) {
          const unsigned i = atomicAdd(&ngather, 1u);
          if (i < kSplitGather) spool[i] = k[b];
        }
      }
    }
  }
  __syncthreads();
  const unsigned ng = ngather;
  if (ng > kSplitGather) {
    hand_on();
    return;
  }
  // rounds of histograms over the gathered keys until one key remains
  while (lo < hi) {
    const unsigned s2 = split_shift(lo, hi);
    for (int b = tid; b < kSplitBins; b += kSplitThreads) hist[b] = 0;
    __syncthreads();
    for (unsigned i = tid; i < ng; i += kSplitThreads) {
      const uint32_t k = spool[i];
      if (k >= lo && k <= hi) atomicAdd(&hist[(k - lo) >> s2], 1u);
    }
    __syncthreads();
    if (!split_find(hist, rank, &bin, &below, wsum, found)) {
      hand_on();
      return;
    }
    rank -= below;
    const uint32_t nlo = lo + (bin << s2);
    const unsigned long long t2 = (unsigned long long)nlo + (1ull << s2) - 1;
    hi = t2 < hi ? (uint32_t)t2 : hi;
    lo = nlo;
  }
  const float val = f32_from_key(lo);
  if (MAD) {
    if (tid == 0) {
      cs[2 * g] = (double)s.med;
      cs[2 * g + 1] = kMadToSigma * (double)val;
      if (invalid && (int64_t)s.nfin < n) atomicAdd(invalid, (unsigned long long)(n - (int64_t)s.nfin));
      st[g].stage = 2;
    }
    return;
  }
  // the MAD's bracket from the same sample as keys of |v - median|
  __syncthreads();   // the gathered keys are replaced by the sample
  const float* v = vals + (size_t)g * stride;
  const unsigned ns = split_sample(v, stride, true, val, spool, &slots, kmm, &nfin_sh);
  uint32_t mlo = 0, mhi = 0;
  if (ns > 0) {
    unsigned long long t[2];
    split_targets(ns, t);
    split_quantiles(spool, slots, kmm[0], kmm[1], t, hist, wsum, found, &mlo, &mhi);
  }
  if (ns == 0 || mhi <= mlo + 1u) {   // no key strictly inside the bracket
    hand_on();
    return;
  }
  for (int b = tid; b < kSplitBins; b += kSplitThreads) hg[b] = 0;
  if (tid == 0) {
    SplitState n2 = s;
    n2.lo = mlo + 1;       // keys <= m_lo are counted below
    n2.hi = mhi - 1;       // keys strictly inside the bracket are copied
    n2.nfin = nfin;
    n2.stage = 1;
    n2.med = val;
    st[g] = n2;
  }
}

template <bool VEC>
static cudaError_t launch_split_t(const float* vals, int groups, int64_t stride, int64_t n,
                                  const NoiseScratch& ns, double* cs, cudaStream_t st) {
  const SplitPtrs sp = split_ptrs(ns.split, groups, stride);
  if ((int64_t)sp.nchunk * kSplitSlot != ns.split_cap) return cudaErrorInvalidValue;   // carved for another stride
  const size_t dyn = (size_t)kSplitPool * sizeof(uint32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_split_bracket,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_split_select<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)dyn);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_split_select<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)dyn);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const dim3 pgrid((unsigned)sp.nchunk, (unsigned)groups);
  cudaError_t e = launch_pdl(k_split_bracket, dim3(groups), dim3(kSplitThreads), dyn, st, vals,
                             stride, sp.st, sp.hist);
  if (e == cudaSuccess)
    e = launch_pdl(k_split_pass<VEC, false>, pgrid, dim3(kSplitPassThreads), 0, st, vals, stride,
                   sp.st, sp.hist, sp.cnt, sp.copies, sp.nchunk);
  if (e == cudaSuccess)
    e = launch_pdl(k_split_select<false>, dim3(groups), dim3(kSplitThreads), dyn, st, vals, stride,
                   n, sp.st, sp.hist, sp.cnt, sp.copies, sp.nchunk, cs, ns.invalid);
  if (e == cudaSuccess)
    e = launch_pdl(k_split_pass<VEC, true>, pgrid, dim3(kSplitPassThreads), 0, st, vals, stride,
                   sp.st, sp.hist, sp.cnt, sp.copies, sp.nchunk);
  if (e == cudaSuccess)
    e = launch_pdl(k_split_select<true>, dim3(groups), dim3(kSplitThreads), dyn, st, vals, stride,
                   n, sp.st, sp.hist, sp.cnt, sp.copies, sp.nchunk, cs, ns.invalid);
  if (e != cudaSuccess) return e;
  count_launches(5);
  return cudaGetLastError();
}

static int noise_blocks(int groups, const NoiseScratch& s) {
  (void)groups;
  return s.nblk;
}

cudaError_t launch_noise(const float* vals, int groups, int64_t stride, int64_t n, int mode,
                         const NoiseScratch& s, double* cs, cudaStream_t st) {
  const int nblk = noise_blocks(groups, s);
  dim3 grid(nblk, groups);
  const bool vec = (reinterpret_cast<uintptr_t>(vals) % 16 == 0) && (stride % 4 == 0);
  if (mode == FITRIG_NOISE_MEANSTD) {
    for (int stage = 0; stage < 2; ++stage) {
      if (vec)
        k_sum_pass<true><<<grid, kNoiseThreads, 0, st>>>(vals, stride, nblk, stage, s.shift,
                                                         s.part, s.cnt);
      else
        k_sum_pass<false><<<grid, kNoiseThreads, 0, st>>>(vals, stride, nblk, stage, s.shift,
                                                          s.part, s.cnt);
      k_sum_final<<<(groups + 127) / 128, 128, 0, st>>>(groups, n, nblk, stage, s.part, s.cnt,
                                                        s.shift, cs,
                                                        stage == 0 ? s.invalid : nullptr);
    }
    count_launches(4);
    return cudaGetLastError();
  }
  if (mode != FITRIG_NOISE_MEDMAD) return cudaErrorInvalidValue;
  // groups of up to 2 Mi values with split scratch: the split form, then the
  // cluster form for any group it leaves
  if (s.split && s.allow_cluster && stride <= kFastMaxPerGroup && groups <= 65535 &&
      stride <= (int64_t)INT32_MAX) {
    const cudaError_t e = vec ? launch_split_t<true>(vals, groups, stride, n, s, cs, st)
                              : launch_split_t<false>(vals, groups, stride, n, s, cs, st);
    if (e != cudaSuccess) return e;
    return launch_medmad_cluster(vals, groups, stride, n, vec, cs, s.invalid, 1, st);
  }
  // groups of moderate size: one cluster per group, all passes in one launch
  if (stride <= kClusterMaxPerGroup && s.allow_cluster) {
    if (stride > kFastMaxPerGroup)
      return launch_medmad_cluster(vals, groups, stride, n, vec, cs, s.invalid, 0, st);
    // the bracketed form, then the cluster form for any group it leaves
    const cudaError_t e = vec ? launch_fast_t<true>(vals, groups, stride, n, cs, s.invalid, st)
                              : launch_fast_t<false>(vals, groups, stride, n, cs, s.invalid, st);
    if (e != cudaSuccess) return e;
    return launch_medmad_cluster(vals, groups, stride, n, vec, cs, s.invalid, 1, st);
  }
  cudaError_t e = cudaMemsetAsync(s.rsel, 0, (size_t)groups * 4 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.hist, 0, (size_t)groups * kBins * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  for (int mad = 0; mad < 2; ++mad) {
    for (int pass = 0; pass < 3; ++pass) {
      if (vec)
        k_rs_hist<true><<<grid, kNoiseThreads, 0, st>>>(vals, stride, nblk, pass, mad, s.rsel,
                                                        cs, s.hist);
      else
        k_rs_hist<false><<<grid, kNoiseThreads, 0, st>>>(vals, stride, nblk, pass, mad, s.rsel,
                                                         cs, s.hist);
      k_rs_select<<<groups, kSelectThreads, 0, st>>>(groups, n, pass, mad, s.hist, s.rsel, cs,
                                                     s.invalid);
    }
  }
  count_launches(12);
  return cudaGetLastError();
}

__global__ void k_thresholds(const double* cs, int groups, double tau, float* thr,
                             double* inv_scale) {
  pdl_begin();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= groups) return;
  const double c = cs[2 * g], s = cs[2 * g + 1];
  if (!(s > 0.0) || !isfinite(c) || !isfinite(s)) {
    thr[g] = INFINITY;   // degenerate spread: nothing is selected
    inv_scale[g] = 0.0;
    return;
  }
  // largest float <= c + tau*s, so (float v > thr) <=> ((double)v > c + tau*s)
  thr[g] = __double2float_rd(c + tau * s);
  inv_scale[g] = 1.0 / s;
}

cudaError_t launch_thresholds(const double* cs, int groups, double tau, float* thr,
                              double* inv_scale, cudaStream_t st) {
  const cudaError_t e = launch_pdl(k_thresholds, dim3((groups + 127) / 128), dim3(128), 0, st, cs,
                                   groups, tau, thr, inv_scale);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace fitrig
