// Threshold, compaction, components, candidates and their sort.
//
// Selection follows the set {t | z_t > tau} of Sec. 2.4.1 (image branch) and
// Sec. 2.4.2 (eta): z = (v - centre) / scale in FP64.  The comparison is made
// in FP32 against thr = the largest float <= centre + tau * scale, which picks
// exactly the floats v with (double)v > centre + tau * scale.
//
// Compaction is order-preserving (per-block counts, an exclusive scan, and a
// warp-ballot write), so the list of selected tiles is sorted by (unit, t).
// Tiles are merged into 8-connected components per unit (a pulsar spreads over
// one, two or four tiles, Sec. 2.4.2) by a lock-free union-find whose roots
// are always the smallest list index; each component yields one candidate at
// its maximum-z tile (ties: smallest tile index).  The image-branch pixel is
// the tile's arg-max of Delta recomputed from the three snapshots; the
// frequency-branch pixel is the tile centre refined by a parabola through the
// eta of the neighbouring tiles.  Candidates are finally radix-sorted by
// (snapshot, y, x), a unique key, so the output is deterministic.
#include <cfloat>
#include <climits>
#include <cmath>

#include "internal.cuh"

namespace fitrig {

constexpr int kSelThreads = 256;

__device__ __forceinline__ void chunk_range(int64_t N, int nblk, int b, int64_t* lo,
                                            int64_t* hi) {
  const int64_t chunk = (N + nblk - 1) / nblk;
  *lo = (int64_t)b * chunk;
  *hi = *lo + chunk < N ? *lo + chunk : N;
}

// Ordered compaction over the element space [0, groups * stride): each warp
// owns a contiguous chunk of `chunk` elements (a multiple of 128), counts its
// selected entries, and after an exclusive scan of the warp counts writes them
// in order with a warp-level prefix -- no block-wide barriers.  VEC reads four
// entries per lane (16-byte aligned base, stride % 4 == 0).
__device__ __forceinline__ void warp_range(int64_t N, int64_t chunk, int64_t* lo, int64_t* hi) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  *lo = w * chunk;
  *hi = *lo + chunk < N ? *lo + chunk : N;
}

template <bool VEC>
__global__ void __launch_bounds__(kSelThreads) k_sel_count(const float* __restrict__ vals,
                                                           int groups, int64_t stride,
                                                           const float* __restrict__ thr,
                                                           int64_t chunk, int* wcnt) {
  const int64_t N = (int64_t)groups * stride;
  int64_t lo, hi;
  warp_range(N, chunk, &lo, &hi);
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  const int step = VEC ? 4 : 1;
  int64_t i = lo + lane * step;
  int g = lo < N ? (int)(lo / stride) : 0;
  int64_t gend = (int64_t)(g + 1) * stride;
  float th = lo < N ? thr[g] : INFINITY;
  for (; i < hi; i += 32 * step) {
    while (i >= gend) {
      ++g;
      gend += stride;
      th = thr[g];
    }
    if (VEC) {
      const float4 q = *reinterpret_cast<const float4*>(vals + i);
      cnt += (q.x > th) + (q.y > th) + (q.z > th) + (q.w > th);
    } else {
      cnt += vals[i] > th;
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) wcnt[((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5] = cnt;
}

// Exclusive scan of per-warp (or per-block) counts (one block of 1024 threads).
__global__ void __launch_bounds__(1024) k_scan_blocks(int nblk, const int* blkcnt, int* blkoff,
                                                      int* total, int64_t cap,
                                                      unsigned* status, unsigned* want) {
  pdl_begin();
  __shared__ long long sh[1024];
  const int per = (nblk + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  long long local = 0;
  for (int b = b0; b < b0 + per && b < nblk; ++b) local += blkcnt[b];
  sh[threadIdx.x] = local;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const long long add = threadIdx.x >= d ? sh[threadIdx.x - d] : 0;
    __syncthreads();
    sh[threadIdx.x] += add;
    __syncthreads();
  }
  long long run = sh[threadIdx.x] - local;
  for (int b = b0; b < b0 + per && b < nblk; ++b) {
    blkoff[b] = (int)(run < cap ? run : cap);
    run += blkcnt[b];
  }
  if (threadIdx.x == 1023) {
    const long long tot = sh[1023];
    *total = (int)(tot < cap ? tot : cap);
    if (tot > cap) {
      atomicOr(status, kErrCapacity);
      if (want) atomicMax(want, (unsigned)(tot < 0xffffffffll ? tot : 0xffffffffll));
    }
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kSelThreads) k_sel_write(const float* __restrict__ vals,
                                                           int groups, int64_t stride,
                                                           const float* __restrict__ thr,
                                                           int64_t chunk, const int* woff,
                                                           SelItem* items, uint32_t* sbits,
                                                           int* wbase, int64_t cap,
                                                           unsigned* compmax, int* peak) {
  const int64_t N = (int64_t)groups * stride;
  int64_t lo, hi;
  warp_range(N, chunk, &lo, &hi);
  if (lo >= hi) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int step = VEC ? 4 : 1;
  int64_t run = woff[((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5];
  int g = (int)(lo / stride);
  int64_t gend = (int64_t)(g + 1) * stride;
  for (int64_t base = lo; base < hi; base += 32 * step) {
    const int64_t i = base + lane * step;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    unsigned bits = 0;
    if (i < hi) {
      while (i >= gend) {
        ++g;
        gend += stride;
      }
      const float th = thr[g];
      if (VEC) {
        const float4 q = *reinterpret_cast<const float4*>(vals + i);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
        bits = (q.x > th) | ((q.y > th) << 1) | ((q.z > th) << 2) | ((q.w > th) << 3);
      } else {
        v[0] = vals[i];
        bits = v[0] > th;
      }
    }
    const int c = __popc(bits);
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int64_t pos = run + incl - c;
    // bitmap words of this iteration (base is a multiple of 32 elements, of
    // 128 with VEC) and the list index of each word's first selected element
    if (VEC) {
      uint32_t word = bits << (4 * (lane & 7));   // lanes 8w..8w+7 hold word w
      word |= __shfl_xor_sync(0xffffffffu, word, 1);
      word |= __shfl_xor_sync(0xffffffffu, word, 2);
      word |= __shfl_xor_sync(0xffffffffu, word, 4);
      if ((lane & 7) == 0) {
        const int64_t wi = (base >> 5) + (lane >> 3);
        sbits[wi] = word;
        wbase[wi] = (int)min(pos, (int64_t)INT_MAX);
      }
    } else {
      const uint32_t word = __ballot_sync(0xffffffffu, bits != 0);
      if (lane == 0) {
        sbits[base >> 5] = word;
        wbase[base >> 5] = (int)min(pos, (int64_t)INT_MAX);
      }
    }
    if (bits) {
      for (int k = 0; k < step; ++k) {
        if (!(bits >> k & 1u)) continue;
        if (pos < cap) {
          const int64_t e = i + k;
          SelItem it;
          it.group = g;
          it.t = (int32_t)(e - (int64_t)g * stride);
          it.v = v[k];
          items[pos] = it;
          compmax[pos] = 0u;   // component state for launch_components
          peak[pos] = INT_MAX;
        }
        ++pos;
      }
    }
    run += total;
  }
}

static int64_t sel_chunk(int64_t N, int nwarps) {
  int64_t c = (N + nwarps - 1) / nwarps;
  return (c + 127) / 128 * 128;
}

static bool sel_vec(const float* vals, int64_t stride) {
  return (reinterpret_cast<uintptr_t>(vals) % 16 == 0) && (stride % 4 == 0);
}

cudaError_t launch_select(const float* vals, int groups, int64_t stride, const float* thr,
                          const SelectScratch& s, unsigned* status, cudaStream_t st) {
  const int nw = s.nblk * (kSelThreads / 32);
  const int64_t chunk = sel_chunk((int64_t)groups * stride, nw);
  if (sel_vec(vals, stride)) {
    k_sel_count<true><<<s.nblk, kSelThreads, 0, st>>>(vals, groups, stride, thr, chunk, s.blkcnt);
    k_scan_blocks<<<1, 1024, 0, st>>>(nw, s.blkcnt, s.blkoff, s.nsel, s.capacity, status,
                                      s.want);
    k_sel_write<true><<<s.nblk, kSelThreads, 0, st>>>(vals, groups, stride, thr, chunk,
                                                      s.blkoff, s.items, s.bits, s.wbase,
                                                      s.capacity, s.compmax, s.peak);
  } else {
    k_sel_count<false><<<s.nblk, kSelThreads, 0, st>>>(vals, groups, stride, thr, chunk, s.blkcnt);
    k_scan_blocks<<<1, 1024, 0, st>>>(nw, s.blkcnt, s.blkoff, s.nsel, s.capacity, status,
                                      s.want);
    k_sel_write<false><<<s.nblk, kSelThreads, 0, st>>>(vals, groups, stride, thr, chunk,
                                                       s.blkoff, s.items, s.bits, s.wbase,
                                                       s.capacity, s.compmax, s.peak);
  }
  count_launches(3);
  return cudaGetLastError();
}

__global__ void k_sum_counts(int nblk, const int* blkcnt, long long* total) {
  __shared__ long long sh[256];
  long long s = 0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += blkcnt[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = sh[0];
}

cudaError_t launch_count_selected(const float* vals, int groups, int64_t stride, const float* thr,
                                  int nblk, int* wcnt, long long* total, cudaStream_t st) {
  const int nw = nblk * (kSelThreads / 32);
  const int64_t chunk = sel_chunk((int64_t)groups * stride, nw);
  if (sel_vec(vals, stride))
    k_sel_count<true><<<nblk, kSelThreads, 0, st>>>(vals, groups, stride, thr, chunk, wcnt);
  else
    k_sel_count<false><<<nblk, kSelThreads, 0, st>>>(vals, groups, stride, thr, chunk, wcnt);
  k_sum_counts<<<1, 256, 0, st>>>(nw, wcnt, total);
  count_launches(2);
  return cudaGetLastError();
}

__global__ void k_clamp_count(int* n, int cap, unsigned* status) {
  pdl_begin();
  if (*n > cap) {
    *n = cap;
    atomicOr(status, kErrCapacity);
  }
}

cudaError_t launch_clamp_count(int* n, int cap, unsigned* status, cudaStream_t st) {
  const cudaError_t e = launch_pdl(k_clamp_count, dim3(1), dim3(1), 0, st, n, cap, status);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- components
__device__ __forceinline__ int64_t item_key(const SelItem& it, int64_t T) {
  return (int64_t)it.group * T + it.t;
}

__device__ __forceinline__ int find_root(int* parent, int x) {
  volatile int* p = parent;
  int y = p[x];
  while (y != x) {
    const int z = p[y];
    if (z != y) p[x] = z;   // path halving; only non-roots are written
    x = y;
    y = p[x];
  }
  return x;
}

__device__ void unite(int* parent, int a, int b, unsigned* status) {
  for (int it = 0; it < (1 << 20); ++it) {
    a = find_root(parent, a);
    b = find_root(parent, b);
    if (a == b) return;
    const int hi = a > b ? a : b, lo = a > b ? b : a;
    const int old = atomicCAS(&parent[hi], hi, lo);
    if (old == hi) return;
    a = old;
    b = lo;
  }
  atomicOr(status, kErrCcLimit);
}


// Horizontal runs: a selected tile whose left neighbour is selected is the next
// list entry after it.  Each warp takes 32 consecutive entries, finds by
// ballot the nearest run start at or before each lane, and points the entry at
// it; a run that began in an earlier warp points at the entry just before the
// warp, so chains only cross warp boundaries.
__global__ void k_cc_runs(const SelItem* __restrict__ items, const int* nsel, int Tx,
                          int* parent) {
  const int n = *nsel;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n; base += nw * 32) {
    const int i = base + lane;
    bool left = false;
    if (i < n && i > 0) {
      const SelItem me = items[i], pv = items[i - 1];
      left = pv.group == me.group && pv.t == me.t - 1 && (me.t % Tx) != 0;
    }
    const unsigned lmask = __ballot_sync(0xffffffffu, left);
    const unsigned starts = ~lmask & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u));
    if (i < n) {
      int head;
      if (starts) head = base + 31 - __clz(starts);
      else head = base - 1;   // the run started in an earlier warp
      parent[i] = head;
    }
  }
}

// List index of element e when it is selected, else -1.
__device__ __forceinline__ int sel_index(const uint32_t* __restrict__ sbits,
                                         const int* __restrict__ wbase, int64_t e) {
  const uint32_t w = sbits[e >> 5];
  const uint32_t b = 1u << (e & 31);
  if (!(w & b)) return -1;
  return wbase[e >> 5] + __popc(w & (b - 1u));
}

__global__ void k_cc_union(const SelItem* __restrict__ items, const int* nsel, int Tx, int Ty,
                           int64_t T, const uint32_t* __restrict__ sbits,
                           const int* __restrict__ wbase, int* parent, unsigned* status) {
  const int n = *nsel;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const SelItem me = items[i];
    const int ty = me.t / Tx, tx = me.t - (me.t / Tx) * Tx;
    if (ty == 0) continue;
    // left neighbours are joined by the runs; of the row above, the tile right
    // above covers both diagonals when it is selected (they would be in its run)
    const int64_t up = (int64_t)me.group * T + (int64_t)(ty - 1) * Tx + tx;
    // (indices at or past n belong to a list that overflowed its capacity)
    const int j = sel_index(sbits, wbase, up);
    if (j >= 0) {
      if (j < n) unite(parent, i, j, status);
    } else {
      if (tx > 0) {
        const int jl = sel_index(sbits, wbase, up - 1);
        if (jl >= 0 && jl < n) unite(parent, i, jl, status);
      }
      if (tx + 1 < Tx) {
        const int jr = sel_index(sbits, wbase, up + 1);
        if (jr >= 0 && jr < n) unite(parent, i, jr, status);
      }
    }
  }
}

// After the unions the roots no longer change, so each thread finds its
// entry's root without writing, then points the entry at it (a final value,
// so other walks through it stay valid) and raises the component's largest
// value key.  (Path halving here could store an intermediate ancestor over
// another thread's root and leave an entry outside its component's root.)
__global__ void k_cc_flatten_max(const SelItem* __restrict__ items, const int* nsel, int* parent,
                                 unsigned* compmax) {
  const int n = *nsel;
  volatile int* p = parent;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int r = i, y = p[i];
    while (y != r) {
      r = y;
      y = p[r];
    }
    p[i] = r;
    atomicMax(&compmax[r], f32_key(items[i].v));   // a component lies in one group
  }
}

// The peak of each component: its entry of largest value, the smallest list
// index on ties (the list is in tile order).
__global__ void k_cc_peak(const SelItem* __restrict__ items, const int* nsel, const int* parent,
                          const unsigned* compmax, int* peak) {
  const int n = *nsel;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int r = parent[i];
    if (f32_key(items[i].v) == compmax[r]) atomicMin(&peak[r], i);
  }
}

cudaError_t launch_components(int Tx, int Ty, int64_t T, const SelectScratch& s,
                              unsigned* status, cudaStream_t st) {
  // (every entry's compmax / peak were initialised by the compaction)
  const int grid = 152 * 16, thr = 256;
  k_cc_runs<<<grid, thr, 0, st>>>(s.items, s.nsel, Tx, s.parent);
  k_cc_union<<<grid, thr, 0, st>>>(s.items, s.nsel, Tx, Ty, T, s.bits, s.wbase, s.parent,
                                   status);
  k_cc_flatten_max<<<grid, thr, 0, st>>>(s.items, s.nsel, s.parent, s.compmax);
  k_cc_peak<<<grid, thr, 0, st>>>(s.items, s.nsel, s.parent, s.compmax, s.peak);
  count_launches(4);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- block-tiled components
// A streaming kernel first thresholds every tile map into a bitmap (one bit
// per tile).  A CTA then takes one kBlkY x kBlkX block of one group's bitmap
// (with a one-tile halo), labels the block's 8-connected components with a
// shared-memory union-find, and finds each component's peak (largest value,
// smallest tile index on ties) as the largest key (value key << 32) | ~t,
// reading the values of the selected tiles only.  A
// component that reaches a selected tile outside the block is a boundary
// component: it gets a global id, its edge tiles get that id in a dense label
// map, and a second kernel unites the ids of selected neighbours across block
// edges.  Every other component's peak is set in the block's bits of the
// dense peak bitmap directly; the merged boundary components' peaks are
// OR'ed in afterwards, and an ordered compaction of the bitmap gives the peak
// list in (group, t) order.
constexpr int kBlkT = kBlkY * kBlkX;
constexpr int kBlkThreads = 256;
static_assert(kBlkY % 32 == 0 && kBlkY <= 64 && kBlkX == 64, "block geometry");
constexpr int kBlkIds = 2 * kBlkX + 2 * (kBlkY - 2);   // boundary components a block can have
constexpr int kBlkPairs = 4 * kBlkIds;                  // cross-edge pairs a block can record
constexpr int kBlkRing = 2 * kBlkX + 2 * (kBlkY - 2);   // edge tiles of a block

__device__ __forceinline__ int find_s(const int* par, int x) {
  const volatile int* p = par;
  int y = p[x];
  while (y != x) {
    x = y;
    y = p[x];
  }
  return x;
}

// Shared-memory union (roots always link the larger index to the smaller).
__device__ void unite_s(int* par, int a, int b, unsigned* status) {
  for (int it = 0; it < (1 << 16); ++it) {
    a = find_s(par, a);
    b = find_s(par, b);
    if (a == b) return;
    const int hi = a > b ? a : b, lo = a > b ? b : a;
    const int old = atomicCAS(&par[hi], hi, lo);
    if (old == hi) return;
    a = old;
    b = lo;
  }
  atomicOr(status, kErrCcLimit);
}

__device__ __forceinline__ int find_g(const int* par, int x) {
  const volatile int* p = par;
  int y = p[x];
  while (y != x) {
    x = y;
    y = p[x];
  }
  return x;
}

__device__ __forceinline__ unsigned long long peak_key(float v, uint32_t t) {
  return ((unsigned long long)f32_key(v) << 32) | (unsigned long long)(0xffffffffu - t);
}

// The ring position r (0 <= r < kBlkRing) of a block's edge as (ly, lx).
__device__ __forceinline__ void ring_pos(int r, int* ly, int* lx) {
  if (r < kBlkX) {
    *ly = 0;
    *lx = r;
  } else if (r < 2 * kBlkX) {
    *ly = kBlkY - 1;
    *lx = r - kBlkX;
  } else {
    const int q = r - 2 * kBlkX;   // the side columns without the corners
    *ly = 1 + (q >> 1);
    *lx = (q & 1) ? kBlkX - 1 : 0;
  }
}

// Cross-block neighbour pair: group, tile and the direction (0..7) of the
// neighbour, packed as (g << 40) | (t << 3) | dir.
__device__ __forceinline__ void dir_offset(int d, int* dy, int* dx) {
  const int k = d < 4 ? d : d + 1;   // skip the centre of the 3 x 3
  *dy = k / 3 - 1;
  *dx = k % 3 - 1;
}

// Run-based labelling on bit masks.  Row y of the block is a 64-bit mask; a
// run is a maximal sequence of set bits, identified by its first bit, and is a
// node of the shared-memory union-find (node y * 64 + start).  Runs of
// adjacent rows are joined when they touch 8-connectedly (overlap after
// dilating one by a bit on each side).
__device__ __forceinline__ uint64_t run_starts(uint64_t m) { return m & ~(m << 1); }

// First bit of the run of m that contains bit b (b set in m).
__device__ __forceinline__ int run_of(uint64_t m, int b) {
  const uint64_t st = run_starts(m) & (b == 63 ? ~0ull : ((2ull << b) - 1ull));
  return 63 - __clzll((long long)st);
}

// Bits s.. of the run of m starting at s.
__device__ __forceinline__ uint64_t run_bits(uint64_t m, int s) {
  const uint64_t from = m >> s;
  const int len = __ffsll((long long)~from) - 1;   // < 64 unless the run reaches bit 63
  const uint64_t ones = (len <= 0 || len >= 64) ? ~0ull : ((1ull << len) - 1ull);
  return (len == 0 ? 0ull : ones) << s;
}

constexpr int kBlkMaxRuns = kBlkT / 2;   // runs of a block (alternating bits at most)

// Selected-tile bitmap: bit (tx & 31) of word tx / 32 of row (g, ty) is
// v > thr[g] (never for NaN: an invalid tile); bits past the row's end are 0.
// One warp per row: all of the row's loads (coalesced, up to 32 per lane) are
// issued before its ballots.
constexpr int kMaskThreads = 256;
__global__ void __launch_bounds__(kMaskThreads) k_blk_mask(const float* __restrict__ vals,
                                                           int64_t stride, int Tx, int Ty,
                                                           int64_t nrows,
                                                           const float* __restrict__ thr,
                                                           BlockScratch b) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * kMaskThreads + threadIdx.x) >> 5;
  if (r >= nrows) return;
  const int g = (int)(r / Ty), ty = (int)(r - (int64_t)g * Ty);
  const float th = thr[g];
  const float* row = vals + (size_t)g * stride + (int64_t)ty * Tx;
  uint32_t* out = b.sbits + (size_t)r * b.words;
  for (int w0 = 0; w0 < b.words; w0 += 32) {
    float x[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int tx = (w0 + u) * 32 + lane;
      x[u] = tx < Tx ? row[tx] : NAN;
    }
    uint32_t mine = 0;
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const uint32_t bal = __ballot_sync(0xffffffffu, x[u] > th);
      if (lane == u) mine = bal;
    }
    if (w0 + lane < b.words) out[w0 + lane] = mine;
  }
}

__global__ void __launch_bounds__(kBlkThreads, 6) k_blk_cc(const float* __restrict__ vals,
                                                        int64_t stride, int Tx, int Ty,
                                                        BlockScratch b, unsigned* status) {
  pdl_begin();
  __shared__ uint32_t wsh[kBlkY + 2][4];      // bitmap words: rows ty0-1 .. ty0+kBlkY, words w0-1 .. w0+2
  __shared__ unsigned long long mrow[kBlkY];   // the block's rows
  __shared__ unsigned long long htop, hbot;   // halo rows above / below (block columns)
  __shared__ unsigned long long hleft, hright;   // halo columns (bit = block row)
  __shared__ uint32_t hcorner;                // bits: 0 top-left, 1 top-right, 2 bottom-left, 3 bottom-right
  __shared__ int runbase[kBlkY + 1];          // first run of each row; runbase[kBlkY] = runs
  __shared__ uint32_t rinfo[kBlkMaxRuns];     // run: row << 16 | start << 8 | end
  __shared__ __align__(16) short par[kBlkMaxRuns];   // union-find over runs (CAS on aligned words)
  __shared__ unsigned long long pkey[kBlkMaxRuns];   // peak key of each root; its id once known
  __shared__ uint32_t bnd[kBlkMaxRuns / 32];         // boundary flag of each root (bit mask)
  __shared__ uint32_t pw[kBlkY][2];
  __shared__ int nsel_sh, nbnd_sh, npair_sh;
  const int g = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this block's slots: boundary ids bidx * kBlkIds + k, pairs bidx * kBlkPairs + k
  const int64_t bidx = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int tx0 = blockIdx.x * kBlkX, ty0 = blockIdx.y * kBlkY;
  const int w0 = tx0 / 32;
  // 1. the bitmap words of the block's rows and of the halo rows (the words
  // on either side hold the halo columns' bits); outside the map: 0
  const uint32_t* sb = b.sbits + (size_t)g * Ty * b.words;
  for (int q = tid; q < (kBlkY + 2) * 4; q += kBlkThreads) {
    const int r = q >> 2, k = q & 3;
    const int ty = ty0 - 1 + r, w = w0 - 1 + k;
    uint32_t word = 0u;
    if (ty >= 0 && ty < Ty && w >= 0 && w < b.words) word = sb[(size_t)ty * b.words + w];
    wsh[r][k] = word;
  }
  if (tid == 0) {
    hleft = hright = 0ull;
    hcorner = 0u;
    nsel_sh = nbnd_sh = npair_sh = 0;
  }
  if (tid < kBlkY) pw[tid][0] = pw[tid][1] = 0u;
  __syncthreads();
  // 2. rows as 64-bit masks, the halo rows, columns and corners
  if (tid < kBlkY + 2) {
    const int r = tid - 1;   // block row -1 .. kBlkY
    const unsigned long long m = ((unsigned long long)wsh[tid][2] << 32) | wsh[tid][1];
    const bool left = (wsh[tid][0] >> 31) != 0u, right = (wsh[tid][3] & 1u) != 0u;
    if (r < 0) {
      htop = m;
      if (left || right) atomicOr(&hcorner, (left ? 1u : 0u) | (right ? 2u : 0u));
    } else if (r >= kBlkY) {
      hbot = m;
      if (left || right) atomicOr(&hcorner, (left ? 4u : 0u) | (right ? 8u : 0u));
    } else {
      mrow[r] = m;
      if (m) atomicAdd(&nsel_sh, __popcll((long long)m));
      if (left) atomicOr(&hleft, 1ull << r);
      if (right) atomicOr(&hright, 1ull << r);
    }
  }
  __syncthreads();
  // 3. the run list: counts per row, their scan (one thread per row, the
  // first kBlkY / 32 warps), then each row's runs
  __shared__ int wrun[kBlkY / 32];
  int rc = 0, rincl = 0;
  if (tid < kBlkY) {
    rc = __popcll((long long)run_starts(mrow[tid]));
    rincl = rc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, rincl, o);
      if (lane >= o) rincl += y;
    }
    if (lane == 31) wrun[warp] = rincl;
  }
  __syncthreads();
  if (tid < kBlkY) {
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wrun[w];
    const int k0 = before + rincl - rc;
    runbase[tid] = k0;
    if (tid == kBlkY - 1) runbase[kBlkY] = before + rincl;
    const unsigned long long m = mrow[tid];
    int k = k0;
    for (unsigned long long st = run_starts(m); st; st &= st - 1, ++k) {
      const int sb = __ffsll((long long)st) - 1;
      const int eb = 63 - __clzll((long long)run_bits(m, sb));
      rinfo[k] = ((uint32_t)tid << 16) | ((uint32_t)sb << 8) | (uint32_t)eb;
    }
  }
  __syncthreads();
  const int nr = runbase[kBlkY];
  auto run_index = [&](int row, int sb) {   // run of `row` starting at bit sb
    const unsigned long long st = run_starts(mrow[row]);
    return runbase[row] + __popcll((long long)(st & ((1ull << sb) - 1ull)));
  };
  for (int k = tid; k < nr; k += kBlkThreads) {
    par[k] = (short)k;
    pkey[k] = 0ull;
  }
  for (int k = tid; k < kBlkMaxRuns / 32; k += kBlkThreads) bnd[k] = 0u;
  __syncthreads();
  // 4. unions: each run with the touching runs of the row above
  const volatile short* vpar = par;
  auto unite_r = [&](int a, int c) {
    for (int it = 0; it < (1 << 16); ++it) {
      while (vpar[a] != a) a = vpar[a];
      while (vpar[c] != c) c = vpar[c];
      if (a == c) return;
      const int hi = a > c ? a : c, lo = a > c ? c : a;
      // 16-bit compare-and-swap through the aligned 32-bit word
      unsigned* w = reinterpret_cast<unsigned*>(&par[hi & ~1]);
      const unsigned sh = (hi & 1) ? 16u : 0u;
      const unsigned old = *reinterpret_cast<volatile unsigned*>(w);
      if ((int)(short)(old >> sh) != hi) continue;
      const unsigned nw = (old & ~(0xffffu << sh)) | ((unsigned)(unsigned short)lo << sh);
      if (atomicCAS(w, old, nw) == old) return;
    }
    atomicOr(status, kErrCcLimit);
  };
  for (int k = tid; k < nr; k += kBlkThreads) {
    const uint32_t ri = rinfo[k];
    const int row = ri >> 16, sb = (ri >> 8) & 255, eb = ri & 255;
    if (row == 0) continue;
    const unsigned long long rb = (eb == 63 ? ~0ull : ((2ull << eb) - 1ull)) & ~((1ull << sb) - 1ull);
    const unsigned long long u = mrow[row - 1];
    unsigned long long nb = (rb | (rb << 1) | (rb >> 1)) & u;
    while (nb) {
      const int ub = __ffsll((long long)nb) - 1;
      const int us = run_of(u, ub);
      unite_r(k, run_index(row - 1, us));
      nb &= ~run_bits(u, us);
    }
  }
  __syncthreads();
  // 5. per run: its root (read-only), boundary flag, peak key
  int rootv[(kBlkMaxRuns + kBlkThreads - 1) / kBlkThreads];
#pragma unroll
  for (int j = 0; j < (kBlkMaxRuns + kBlkThreads - 1) / kBlkThreads; ++j) {
    const int k = tid + j * kBlkThreads;
    rootv[j] = -1;
    if (k >= nr) continue;
    int r = k;
    while (par[r] != r) r = par[r];
    rootv[j] = r;
    const uint32_t ri = rinfo[k];
    const int row = ri >> 16, sb = (ri >> 8) & 255, eb = ri & 255;
    const unsigned long long rb = (eb == 63 ? ~0ull : ((2ull << eb) - 1ull)) & ~((1ull << sb) - 1ull);
    const unsigned long long dil = rb | (rb << 1) | (rb >> 1);
    bool out = false;
    if (row == 0) out = out || (dil & htop) || (sb == 0 && (hcorner & 1u)) || (eb == 63 && (hcorner & 2u));
    if (row == kBlkY - 1)
      out = out || (dil & hbot) || (sb == 0 && (hcorner & 4u)) || (eb == 63 && (hcorner & 8u));
    // block rows row-1..row+1 as halo-column bits
    const unsigned long long near = row == 0 ? 3ull : (7ull << (row - 1));
    if (sb == 0) out = out || (hleft & near);
    if (eb == 63) out = out || (hright & near);
    if (out) atomicOr(&bnd[r >> 5], 1u << (r & 31));
    unsigned long long key = 0ull;
    const uint32_t t0 = (uint32_t)((ty0 + row) * Tx + tx0);
    const float* vr = vals + (size_t)g * stride + t0;
#pragma unroll 4
    for (int c = sb; c <= eb; ++c) {
      const unsigned long long kc = peak_key(vr[c], t0 + (uint32_t)c);
      key = kc > key ? kc : key;
    }
    atomicMax(&pkey[r], key);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < (kBlkMaxRuns + kBlkThreads - 1) / kBlkThreads; ++j)
    if (rootv[j] >= 0) par[tid + j * kBlkThreads] = (short)rootv[j];   // straight to the root
  // 6. roots: an interior component's peak bit; a boundary component's id
#pragma unroll
  for (int j = 0; j < (kBlkMaxRuns + kBlkThreads - 1) / kBlkThreads; ++j) {
    const int k = tid + j * kBlkThreads;
    if (rootv[j] != k) continue;
    const unsigned long long key = pkey[k];
    if (!((bnd[k >> 5] >> (k & 31)) & 1u)) {
      const uint32_t t = 0xffffffffu - (uint32_t)key;
      const int pty = (int)(t / (uint32_t)Tx), ptx = (int)(t - (uint32_t)pty * (uint32_t)Tx);
      const int ply = pty - ty0, plx = ptx - tx0;
      atomicOr(&pw[ply][plx >> 5], 1u << (plx & 31));
    } else {
      const int slot = atomicAdd(&nbnd_sh, 1);   // < kBlkIds: each owns a ring tile
      const int id = (int)(bidx * kBlkIds + slot);
      b.bpar[id] = id;
      b.bgrp[id] = g;
      b.bkey[id] = key;
      b.rkey[id] = key;
      pkey[k] = (unsigned long long)id;   // only this thread reads or writes a root's slot here
    }
  }
  __syncthreads();
  // 7. edge tiles of boundary components: their label, and each selected
  // neighbour across the block edge with a larger tile index as a pair; the
  // block's peak words; the counts
  auto selected = [&](int ly, int lx) -> bool {   // -1 <= ly <= kBlkY, -1 <= lx <= kBlkX
    if (ly >= 0 && ly < kBlkY) {
      if (lx >= 0 && lx < kBlkX) return (mrow[ly] >> lx) & 1ull;
      return ((lx < 0 ? hleft : hright) >> ly) & 1ull;
    }
    if (lx >= 0 && lx < kBlkX) return ((ly < 0 ? htop : hbot) >> lx) & 1ull;
    return (hcorner >> ((ly < 0 ? 0 : 2) + (lx < 0 ? 0 : 1))) & 1u;
  };
  if (tid < kBlkRing) {
    int ly, lx;
    ring_pos(tid, &ly, &lx);
    if (selected(ly, lx)) {
      const int r = par[run_index(ly, run_of(mrow[ly], lx))];
      if ((bnd[r >> 5] >> (r & 31)) & 1u) {
        const int64_t t = (int64_t)(ty0 + ly) * Tx + (tx0 + lx);
        b.glab[(size_t)g * stride + t] = (int)pkey[r];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
          int dy, dx;
          dir_offset(d, &dy, &dx);
          const int ny = ly + dy, nx = lx + dx;
          const bool outside = ny < 0 || ny >= kBlkY || nx < 0 || nx >= kBlkX;
          if (!outside || !selected(ny, nx)) continue;
          if (dy * Tx + dx <= 0) continue;   // the other tile records it
          const int k = atomicAdd(&npair_sh, 1);   // < kBlkPairs: at most 4 per ring tile
          b.pairs[bidx * kBlkPairs + k] =
              ((unsigned long long)g << 40) | ((unsigned long long)t << 3) | (unsigned)d;
        }
      }
    }
  }
  if (tid < 2 * kBlkY) {
    const int ly = tid >> 1, wx = tid & 1;
    const int ty = ty0 + ly, w = tx0 / 32 + wx;
    if (ty < Ty && w < b.words) b.pbits[((size_t)g * Ty + ty) * b.words + w] = pw[ly][wx];
  }
  __syncthreads();
  if (tid == 0) b.bstat[bidx] = make_int4(nbnd_sh, npair_sh, nsel_sh, 0);
}

// Unions of boundary components across block edges: one warp per block joins
// the component ids of the block's recorded neighbour pairs.
__device__ __forceinline__ bool valid_id(const BlockScratch& b, int64_t nblocks, int id) {
  if (id < 0) return false;
  const int64_t blk = id / kBlkIds;
  return blk < nblocks && (id - blk * kBlkIds) < b.bstat[blk].x;
}

__global__ void k_blk_merge(int64_t stride, int Tx, int64_t nblocks, BlockScratch b,
                            unsigned* status) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; blk < nblocks;
       blk += nw) {
    const int np = b.bstat[blk].y;
    for (int k = lane; k < np; k += 32) {
      const unsigned long long pk = b.pairs[blk * kBlkPairs + k];
      const int g = (int)(pk >> 40);
      const int64_t t = (int64_t)((pk >> 3) & ((1ull << 37) - 1));
      int dy, dx;
      dir_offset((int)(pk & 7u), &dy, &dx);
      const int64_t tn = t + (int64_t)dy * Tx + dx;
      const int* lab = b.glab + (size_t)g * stride;
      // the label map is never cleared: every label read here was written by
      // k_blk_cc of this detect, and the check keeps a stale one harmless
      const int me = lab[t], other = lab[tn];
      if (valid_id(b, nblocks, me) && valid_id(b, nblocks, other)) unite(b.bpar, me, other, status);
    }
  }
}

// Merged peak keys: every boundary component raises its root's key.
__global__ void k_blk_resolve(int64_t nblocks, BlockScratch b) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; blk < nblocks;
       blk += nw) {
    const int n = b.bstat[blk].x;
    for (int k = lane; k < n; k += 32) {
      const int id = (int)(blk * kBlkIds + k);
      const int r = find_g(b.bpar, id);
      if (r != id) atomicMax(&b.rkey[r], b.bkey[id]);
    }
  }
}

// Each merged component's peak bit.
__global__ void k_blk_mark(int Tx, int Ty, int64_t nblocks, BlockScratch b) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; blk < nblocks;
       blk += nw) {
    const int n = b.bstat[blk].x;
    for (int k = lane; k < n; k += 32) {
      const int id = (int)(blk * kBlkIds + k);
      if (b.bpar[id] != id) continue;   // roots never change after the unions
      const uint32_t t = 0xffffffffu - (uint32_t)b.rkey[id];
      const int ty = (int)(t / (uint32_t)Tx), tx = (int)(t - (uint32_t)ty * (uint32_t)Tx);
      atomicOr(&b.pbits[((size_t)b.bgrp[id] * Ty + ty) * b.words + (tx >> 5)], 1u << (tx & 31));
    }
  }
}

// Ordered compaction of the peak bitmap, one warp per tile row and
// kRowsPerCta rows per CTA: each row's peak count and each CTA's sum, the
// scan of the CTAs' sums, then each row's peaks in order.  A row's offset is
// its CTA's offset plus the counts of the CTA's rows before it.
constexpr int kPbThreads = 256;
constexpr int kRowsPerCta = kPbThreads / 32;

__device__ __forceinline__ int64_t row_offset(const BlockScratch& b, int64_t r) {
  const int64_t r0 = r & ~(int64_t)(kRowsPerCta - 1);
  int64_t off = b.blkoff[r0 / kRowsPerCta];
#pragma unroll
  for (int k = 0; k < kRowsPerCta - 1; ++k)
    if (r0 + k < r) off += b.rowcnt[r0 + k];
  return off;
}

__global__ void __launch_bounds__(kPbThreads) k_pbits_count(int64_t nrows, BlockScratch b) {
  pdl_begin();
  __shared__ int wc[kRowsPerCta];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r = (int64_t)blockIdx.x * kRowsPerCta + warp;
  int c = 0;
  if (r < nrows) {
    const uint32_t* row = b.pbits + (size_t)r * b.words;
    for (int w = lane; w < b.words; w += 32) c += __popc(row[w]);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) {
    wc[warp] = c;
    if (r < nrows) b.rowcnt[r] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kRowsPerCta; ++w) t += wc[w];
    b.blkcnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kPbThreads) k_pbits_write(int64_t nrows, int Tx, int Ty,
                                                            const float* __restrict__ vals,
                                                            int64_t stride, BlockScratch b,
                                                            SelItem* peaks, int64_t cap) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * kPbThreads + threadIdx.x) >> 5;
  if (r >= nrows) return;
  const int g = (int)(r / Ty), ty = (int)(r - (int64_t)g * Ty);
  const uint32_t* row = b.pbits + (size_t)r * b.words;
  const float* vg = vals + (size_t)g * stride;
  int64_t run = row_offset(b, r);
  for (int w0 = 0; w0 < b.words; w0 += 32) {
    const int wx = w0 + lane;
    const uint32_t w = wx < b.words ? row[wx] : 0u;
    const int c = __popc(w);
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int64_t pos = run + incl - c;
    run += __shfl_sync(0xffffffffu, incl, 31);
    // every value load of the word first, then the writes
    constexpr int kMaxBits = 8;
    float val[kMaxBits];
    int tt[kMaxBits];
    uint32_t m = w;
    while (m) {
      int nb = 0;
      for (; m && nb < kMaxBits; ++nb) {
        const int bit = __ffs(m) - 1;
        m &= m - 1;
        tt[nb] = ty * Tx + wx * 32 + bit;
        val[nb] = vg[tt[nb]];
      }
      for (int k = 0; k < nb; ++k, ++pos)
        if (pos < cap) peaks[pos] = SelItem{g, tt[k], val[k]};
    }
  }
}

// The selected count (the blocks' sum) against the selection capacity.
__global__ void __launch_bounds__(1024) k_blk_check(int64_t nblocks, BlockScratch b, int64_t cap,
                                                    unsigned* status, unsigned* want) {
  pdl_begin();
  __shared__ long long part[32];
  long long n = 0;
  for (int64_t i = threadIdx.x; i < nblocks; i += 1024) n += b.bstat[i].z;
  for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int w = 0; w < 32; ++w) tot += part[w];
    if (tot > cap) {
      atomicOr(status, kErrCapacity);
      if (want) atomicMax(want, (unsigned)(tot < 0xffffffffll ? tot : 0xffffffffll));
    }
  }
}

static int block_words(int Tx) { return (Tx + 31) / 32; }

static int64_t block_count(int groups, int Tx, int Ty) {
  return (int64_t)groups * ((Ty + kBlkY - 1) / kBlkY) * ((Tx + kBlkX - 1) / kBlkX);
}

size_t block_scratch_bytes(int groups, int Tx, int Ty, int64_t stride) {
  const int64_t cap = block_count(groups, Tx, Ty) * kBlkIds;
  const int64_t nw = (int64_t)groups * Ty * block_words(Tx);
  const int64_t nrows = (int64_t)groups * Ty;
  const int64_t nblk = (nrows + kRowsPerCta - 1) / kRowsPerCta;
  size_t bytes = 0;
  auto add = [&](size_t n) { bytes += (n + 255) / 256 * 256; };
  add(sizeof(int) * (size_t)groups * stride);    // glab
  add(sizeof(int) * cap);                        // bpar
  add(sizeof(int) * cap);                        // bgrp
  add(sizeof(unsigned long long) * cap);         // bkey
  add(sizeof(unsigned long long) * cap);         // rkey
  add(sizeof(uint32_t) * nw);                    // pbits
  add(sizeof(uint32_t) * nw);                    // sbits
  add(sizeof(unsigned long long) * block_count(groups, Tx, Ty) * kBlkPairs);   // pairs
  add(sizeof(int4) * block_count(groups, Tx, Ty));   // bstat
  add(sizeof(int) * 4);                          // counters
  add(sizeof(int) * nblk);                       // blkcnt
  add(sizeof(int) * (nblk + 1));                 // blkoff
  add(sizeof(int) * nrows);                      // rowcnt
  return bytes;
}

void block_scratch_carve(void* base, int groups, int Tx, int Ty, int64_t stride, BlockScratch* b) {
  const int64_t cap = block_count(groups, Tx, Ty) * kBlkIds;
  const int64_t nw = (int64_t)groups * Ty * block_words(Tx);
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t n) {
    char* q = p + off;
    off += (n + 255) / 256 * 256;
    return q;
  };
  b->glab = reinterpret_cast<int*>(take(sizeof(int) * (size_t)groups * stride));
  b->bpar = reinterpret_cast<int*>(take(sizeof(int) * cap));
  b->bgrp = reinterpret_cast<int*>(take(sizeof(int) * cap));
  b->bkey = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * cap));
  b->rkey = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * cap));
  b->pbits = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * nw));
  b->sbits = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * nw));
  b->pairs = reinterpret_cast<unsigned long long*>(
      take(sizeof(unsigned long long) * block_count(groups, Tx, Ty) * kBlkPairs));
  b->bstat = reinterpret_cast<int4*>(take(sizeof(int4) * block_count(groups, Tx, Ty)));
  b->pcap = block_count(groups, Tx, Ty) * kBlkPairs;
  b->counters = reinterpret_cast<int*>(take(sizeof(int) * 4));
  const int64_t nrows = (int64_t)groups * Ty;
  b->nblk = (int)((nrows + kRowsPerCta - 1) / kRowsPerCta);
  b->blkcnt = reinterpret_cast<int*>(take(sizeof(int) * b->nblk));
  b->blkoff = reinterpret_cast<int*>(take(sizeof(int) * (b->nblk + 1)));
  b->rowcnt = reinterpret_cast<int*>(take(sizeof(int) * nrows));
  b->cap = cap;
  b->words = block_words(Tx);
}

cudaError_t launch_block_select(const float* vals, int groups, int64_t stride, int Tx, int Ty,
                                const float* thr, const BlockScratch& b, SelItem* peaks,
                                int64_t cap, unsigned* status, unsigned* want, cudaStream_t st) {
  // peaks == nullptr: the caller emits straight from the rows (launch_emit_rows)
  const int64_t nblocks = block_count(groups, Tx, Ty);
  if (groups < 1 || groups > 65535 || (Ty + kBlkY - 1) / kBlkY > 65535 ||
      (int64_t)Tx * Ty > 0xffffffffll || nblocks * kBlkIds > INT_MAX ||
      nblocks * kBlkIds > b.cap)
    return cudaErrorInvalidValue;
  // (counters[2], the peak count, is written by the scan below; nothing else
  // is read, so no clearing launch sits between the noise and this chain)
  const int64_t nrows = (int64_t)groups * Ty;
  cudaError_t e = launch_pdl(k_blk_mask, dim3((unsigned)((nrows * 32 + kMaskThreads - 1) / kMaskThreads)),
                             dim3(kMaskThreads), 0, st, vals, stride, Tx, Ty, nrows, thr, b);
  const dim3 grid((Tx + kBlkX - 1) / kBlkX, (Ty + kBlkY - 1) / kBlkY, groups);
  if (e == cudaSuccess)
    e = launch_pdl(k_blk_cc, grid, dim3(kBlkThreads), 0, st, vals, stride, Tx, Ty, b, status);
  const unsigned wgrid = (unsigned)std::min<int64_t>((nblocks + 7) / 8, 152 * 16);   // a warp per block
  if (e == cudaSuccess)
    e = launch_pdl(k_blk_merge, dim3(wgrid), dim3(256), 0, st, stride, Tx, nblocks, b, status);
  if (e == cudaSuccess) e = launch_pdl(k_blk_resolve, dim3(wgrid), dim3(256), 0, st, nblocks, b);
  if (e == cudaSuccess)
    e = launch_pdl(k_blk_mark, dim3(wgrid), dim3(256), 0, st, Tx, Ty, nblocks, b);
  if (e != cudaSuccess) return e;
  const int64_t ncta = (nrows + kRowsPerCta - 1) / kRowsPerCta;
  if (ncta > b.nblk) return cudaErrorInvalidValue;   // sized by block_scratch_carve
  const unsigned rgrid = (unsigned)ncta;   // a warp per row
  e = launch_pdl(k_pbits_count, dim3(rgrid), dim3(kPbThreads), 0, st, nrows, b);
  if (e == cudaSuccess)
    e = launch_pdl(k_scan_blocks, dim3(1), dim3(1024), 0, st, (int)ncta, (const int*)b.blkcnt,
                   b.blkoff, &b.counters[2], cap, status, (unsigned*)nullptr);
  if (e == cudaSuccess && peaks)
    e = launch_pdl(k_pbits_write, dim3(rgrid), dim3(kPbThreads), 0, st, nrows, Tx, Ty, vals, stride,
                   b, peaks, cap);
  if (e == cudaSuccess)
    e = launch_pdl(k_blk_check, dim3(1), dim3(1024), 0, st, nblocks, b, cap, status, want);
  if (e != cudaSuccess) return e;
  count_launches(peaks ? 9 : 8);
  return cudaGetLastError();
}

// ---- ordered list of component peaks (sorted by (group, t) like the items)
__global__ void __launch_bounds__(kSelThreads) k_peak_count(const int* nsel, const int* parent,
                                                            const int* peak, int nblk,
                                                            int* blkcnt) {
  __shared__ int wsum[kSelThreads / 32];
  int64_t lo, hi;
  chunk_range(*nsel, nblk, blockIdx.x, &lo, &hi);
  int cnt = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) cnt += peak[parent[i]] == (int)i;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) t += wsum[w];
    blkcnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kSelThreads) k_peak_write(const int* nsel, const int* parent,
                                                            const int* peak, int nblk,
                                                            const int* blkoff, int* plist) {
  __shared__ int wcnt[kSelThreads / 32];
  int64_t lo, hi;
  chunk_range(*nsel, nblk, blockIdx.x, &lo, &hi);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int run = blkoff[blockIdx.x];
  for (int64_t base = lo; base < hi; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool is_peak = i < hi && peak[parent[i]] == (int)i;
    const unsigned bal = __ballot_sync(0xffffffffu, is_peak);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    int before = 0, tile = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) {
      before += w < warp ? wcnt[w] : 0;
      tile += wcnt[w];
    }
    if (is_peak) plist[run + before + __popc(bal & ((1u << lane) - 1u))] = (int)i;
    run += tile;
    __syncthreads();
  }
}

// ---- candidates
// Peak p of an ordered peak list: items[plist[p]], or items[p] without plist.
__device__ __forceinline__ SelItem peak_item(const SelItem* items, const int* plist, int p) {
  return plist ? items[plist[p]] : items[p];
}

__device__ __forceinline__ float load_px(const void* base, int storage, int64_t idx) {
  switch (storage) {
    case FITRIG_BF16: return to_f32(static_cast<const bf16_t*>(base)[idx]);
    case FITRIG_F16: return to_f32(static_cast<const f16_t*>(base)[idx]);
    default: return static_cast<const float*>(base)[idx];
  }
}

__device__ __forceinline__ float parabola(float l, float c, float r) {
  if (!isfinite(l) || !isfinite(c) || !isfinite(r)) return 0.f;
  const float den = l - 2.f * c + r;
  if (!(den < 0.f)) return 0.f;
  const float d = 0.5f * (l - r) / den;
  return fminf(0.5f, fmaxf(-0.5f, d));
}

// Peak offset within [-0.5, 0.5] of the Catmull-Rom cubic spline through the
// samples at -2..2 (m2, m1, c, p1, p2) along one axis of the eta map.  On the
// segment from a (at 0) to b (at 1) with outer neighbours z (at -1) and d (at
// 2):  f(t) = a + t (k1 + t (k2 + t k3)),  k1 = (b - z)/2,
// k2 = (2z - 5a + 4b - d)/2,  k3 = (-z + 3a - 3b + d)/2.  Candidates in order:
// offset 0; the right segment's interior roots of f' (ascending), then +0.5;
// the left segment's (t in [0.5, 1], offset t - 1) roots, then -0.5; strictly
// larger values win.  A missing neighbour at +-1 leaves its side unsearched;
// a missing outer sample is extended linearly.  Roots of f' come from the
// cancellation-free form of the quadratic formula.
__device__ __forceinline__ float cubic_offset(float m2, float m1, float c, float p1, float p2) {
  if (!isfinite(c)) return 0.f;
  float bx = 0.f, bf = c;
  auto segment = [&](float z, float a, float b, float d, float lo, float hi, float shift) {
    const float k1 = 0.5f * (b - z);
    const float k2 = 0.5f * (2.f * z - 5.f * a + 4.f * b - d);
    const float k3 = 0.5f * (-z + 3.f * a - 3.f * b + d);
    auto f = [&](float t) { return a + t * (k1 + t * (k2 + t * k3)); };
    const float A = 3.f * k3, B = 2.f * k2, C = k1;
    const float disc = B * B - 4.f * A * C;
    float r0 = 0.f, r1 = 0.f;
    int nr = 0;
    if (disc >= 0.f) {
      const float q = -0.5f * (B + copysignf(sqrtf(disc), B));
      if (A != 0.f) r0 = q / A, nr = 1;
      if (q != 0.f) {
        if (nr == 0) r0 = C / q;
        else r1 = C / q;
        ++nr;
      }
      if (nr == 2 && r1 < r0) {
        const float t = r0;
        r0 = r1;
        r1 = t;
      }
    }
    if (nr >= 1 && lo < r0 && r0 < hi) {
      const float v = f(r0);
      if (v > bf) bf = v, bx = r0 + shift;
    }
    if (nr == 2 && lo < r1 && r1 < hi) {
      const float v = f(r1);
      if (v > bf) bf = v, bx = r1 + shift;
    }
    const float e = shift == 0.f ? hi : lo;
    const float v = f(e);
    if (v > bf) bf = v, bx = e + shift;
  };
  if (isfinite(p1)) {
    const float d = isfinite(p2) ? p2 : 2.f * p1 - c;
    segment(isfinite(m1) ? m1 : 2.f * c - p1, c, p1, d, 0.f, 0.5f, 0.f);
  }
  if (isfinite(m1)) {
    const float z = isfinite(m2) ? m2 : 2.f * m1 - c;
    segment(z, m1, c, isfinite(p1) ? p1 : 2.f * c - m1, 0.5f, 1.f, -1.f);
  }
  return bx;
}

// The candidate's significance, z = (v - centre) / scale in FP64 (Sec. 2.4.1,
// 2.4.2), rounded to FP32 for the output.
__device__ __forceinline__ float significance(const CandArgs& a, const SelItem& it) {
  return (float)(((double)it.v - a.cs[2 * it.group]) * a.inv[it.group]);
}

// Frequency branch: one thread per peak; tile-centre order is (y, x) order,
// so the peaks' list order is already the output order.
__global__ void k_emit_freq(CandArgs a, const SelItem* __restrict__ items, const int* np_,
                            const int* __restrict__ plist) {
  pdl_begin();
  const int np = *np_;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const SelItem it = peak_item(items, plist, p);
    const int ty = it.t / a.Tx, tx = it.t - (it.t / a.Tx) * a.Tx;
    const int hw = min(a.w, a.ny - ty * a.w), ww = min(a.w, a.nx - tx * a.w);
    const float e = a.eta[it.t];
    const float el = tx > 0 ? a.eta[it.t - 1] : NAN;
    const float er = tx + 1 < a.Tx ? a.eta[it.t + 1] : NAN;
    const float eu = ty > 0 ? a.eta[it.t - a.Tx] : NAN;
    const float ed = ty + 1 < a.Ty ? a.eta[it.t + a.Tx] : NAN;
    fitrig_candidate c;
    c.x = tx * a.w + (ww - 1) / 2;
    c.y = ty * a.w + (hw - 1) / 2;
    c.snapshot = -1;
    c.significance = significance(a, it);
    c.branch = FITRIG_BRANCH_FREQ;
    c.freq_bin = a.bin[it.t];
    float dx, dy;
    if (a.refine == FITRIG_REFINE_CUBIC) {
      const float el2 = tx > 1 ? a.eta[it.t - 2] : NAN;
      const float er2 = tx + 2 < a.Tx ? a.eta[it.t + 2] : NAN;
      const float eu2 = ty > 1 ? a.eta[it.t - 2 * a.Tx] : NAN;
      const float ed2 = ty + 2 < a.Ty ? a.eta[it.t + 2 * a.Tx] : NAN;
      dx = cubic_offset(el2, el, e, er, er2);
      dy = cubic_offset(eu2, eu, e, ed, ed2);
    } else {
      dx = parabola(el, e, er);
      dy = parabola(eu, e, ed);
    }
    c.xf = (float)(tx * a.w) + 0.5f * (float)(ww - 1) + dx * (float)a.w;
    c.yf = (float)(ty * a.w) + 0.5f * (float)(hw - 1) + dy * (float)a.w;
    if (p < a.cap) a.out[p] = c;
  }
}

__device__ __forceinline__ fitrig_candidate image_candidate(const CandArgs& a, const SelItem& it,
                                                            int tx, int ty, int w, int dx, int dy) {
  fitrig_candidate c;
  c.x = tx * w + dx;
  c.y = ty * w + dy;
  c.snapshot = it.group;
  c.significance = significance(a, it);
  c.branch = FITRIG_BRANCH_IMAGE;
  c.freq_bin = -1;
  c.xf = (float)c.x;
  c.yf = (float)c.y;
  return c;
}

// Image branch, step 1 (otherwise): one warp per peak computes the tile's
// arg-max of Delta (ties: smallest row-major index, same FP32 arithmetic as the
// stack march) and writes the candidate in peak-list order to `tmp`.
__global__ void k_emit_image(CandArgs a, const SelItem* __restrict__ items, const int* np_,
                             const int* __restrict__ plist, fitrig_candidate* tmp) {
  pdl_begin();
  const int np = *np_;
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = wid; p < np; p += nw) {
    const SelItem it = peak_item(items, plist, p);
    const int ty = it.t / a.Tx, tx = it.t - (it.t / a.Tx) * a.Tx;
    const int hw = min(a.w, a.ny - ty * a.w), ww = min(a.w, a.nx - tx * a.w);
    int64_t sl[3];   // the unit's three snapshots in the stack
    for (int k = 0; k < 3; ++k)
      sl[k] = (a.zmod > 0 ? (int64_t)((a.zrot + it.group + k) % a.zmod) : (int64_t)(it.group + k)) * a.slice;
    float best = -1.f;
    int bidx = INT_MAX;
    for (int q = lane; q < hw * ww; q += 32) {
      const int dy = q / ww, dx = q - (q / ww) * ww;
      const int64_t off = (int64_t)(ty * a.w + dy) * a.pitch + (tx * a.w + dx);
      float x0, x1, x2;
      if (a.key) {
        // difference-coded stack (plans only: slot = snapshot): decode the
        // pixel in snapshot order with the march's FP32 sums
        x0 = a.key[(int64_t)(ty * a.w + dy) * a.kpitch + (tx * a.w + dx)];
        for (int k = 1; k <= it.group; ++k)
          x0 = __fadd_rn(x0, load_px(a.stack, a.storage, (int64_t)k * a.slice + off));
        x1 = __fadd_rn(x0, load_px(a.stack, a.storage, sl[1] + off));
        x2 = __fadd_rn(x1, load_px(a.stack, a.storage, sl[2] + off));
      } else {
        x0 = load_px(a.stack, a.storage, sl[0] + off);
        x1 = load_px(a.stack, a.storage, sl[1] + off);
        x2 = load_px(a.stack, a.storage, sl[2] + off);
      }
      const float d = fabsf(fabsf(x2 - x1) - fabsf(x1 - x0));
      if (d > best) {
        best = d;
        bidx = q;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) {
        best = ob;
        bidx = oi;
      }
    }
    if (lane == 0) tmp[p] = image_candidate(a, it, tx, ty, a.w, bidx % ww, bidx / ww);
  }
}

// Image branch, step 2: peaks are in (unit, tile row, tile column) order.  Each
// run of peaks sharing (unit, tile row) -- a group -- occupies the same output
// positions once sorted by (y, x); inside a group the order is (dy, tx), so a
// stable counting sort on the in-tile row dy finishes it.  A warp scans 32
// consecutive peaks, finds the group heads among them by ballot, and sorts
// each of those groups (which may run past its 32 entries).  A group's first
// 32 peaks are read once and kept in registers between the count and the
// write (most groups are no longer); later ones are read again.
constexpr int kGroupWarps = 8;
constexpr int kMaxW = 128;

// FROM_ARG: the candidates are formed here from the peak list and the
// march's in-tile arg-max (no intermediate list); otherwise they are read
// from `tmp`, where k_emit_image wrote them.
template <bool FROM_ARG>
__global__ void __launch_bounds__(kGroupWarps * 32) k_group_sort(CandArgs a, const int* np_,
                                                                 const fitrig_candidate* tmp,
                                                                 const SelItem* __restrict__ items,
                                                                 const int* __restrict__ plist,
                                                                 const int* base_) {
  pdl_begin();
  __shared__ int counts[kGroupWarps][kMaxW];
  // one peak: its group (snapshot, tile row) and, for the count and the
  // write, its candidate
  struct Peak {
    SelItem it;   // FROM_ARG
    fitrig_candidate c;
    int snap, row;
  };
  auto head_of = [&](int p, int* snap, int* row) {
    if (FROM_ARG) {
      const SelItem it = peak_item(items, plist, p);
      *snap = it.group;
      *row = it.t / a.Tx;
    } else {
      const fitrig_candidate c = tmp[p];
      *snap = c.snapshot;
      *row = c.y / a.w;
    }
  };
  auto load = [&](int p) -> Peak {
    Peak k;
    if (FROM_ARG) {
      k.it = peak_item(items, plist, p);
      k.snap = k.it.group;
      k.row = k.it.t / a.Tx;
    } else {
      k.c = tmp[p];
      k.snap = k.c.snapshot;
      k.row = k.c.y / a.w;
    }
    return k;
  };
  // the candidate and its in-tile row (FROM_ARG: from the march's arg-max)
  auto finish = [&](Peak& k) -> int {
    if (FROM_ARG) {
      const int ty = k.row, tx = k.it.t - ty * a.Tx;
      const int idx = a.arg[(int64_t)k.it.group * a.stride + k.it.t];
      k.c = image_candidate(a, k.it, tx, ty, a.w, idx % a.w, idx / a.w);
    }
    return k.c.y - k.row * a.w;
  };
  const int np = *np_;
  const int base = base_ ? *base_ : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* cnt = counts[warp];
  const int wid = blockIdx.x * kGroupWarps + warp;
  const int nw = gridDim.x * kGroupWarps;
  for (int p0 = wid * 32; p0 < np; p0 += nw * 32) {
    const int pl = p0 + lane;
    int sn = -1, rw = -1, psn = -2, prw = -2;
    if (pl < np) head_of(pl, &sn, &rw);
    if (lane == 0 && pl > 0 && pl < np) head_of(pl - 1, &psn, &prw);
    const int usn = __shfl_up_sync(0xffffffffu, sn, 1), urw = __shfl_up_sync(0xffffffffu, rw, 1);
    if (lane > 0) {
      psn = usn;
      prw = urw;
    }
    const bool head = pl < np && (sn != psn || rw != prw);
    unsigned heads = __ballot_sync(0xffffffffu, head);
    while (heads) {
      const int hl = __ffs(heads) - 1;
      heads &= heads - 1;
      const int p = p0 + hl;
      const int snap = __shfl_sync(0xffffffffu, sn, hl), gty = __shfl_sync(0xffffffffu, rw, hl);
      for (int k = lane; k < a.w; k += 32) cnt[k] = 0;
      __syncwarp();
      // the group's extent and its count per in-tile row; the first 32 peaks
      // stay in registers
      Peak first;
      int dy0 = kMaxW;
      int end = p;
      for (int q0 = p;; q0 += 32) {
        const int q = q0 + lane;
        Peak k;
        bool in = false;
        if (q < np) {
          k = load(q);
          in = k.snap == snap && k.row == gty;
        }
        int dy = kMaxW;
        if (in) {
          dy = finish(k);
          atomicAdd(&cnt[dy], 1);
        }
        if (q0 == p) {
          first = k;
          dy0 = dy;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, in);   // a prefix of the lanes
        end = q0 + __popc(bal);
        if (bal != 0xffffffffu) break;
      }
      __syncwarp();
      if (lane == 0) {
        int run = 0;
        for (int k = 0; k < a.w; ++k) {
          const int c = cnt[k];
          cnt[k] = run;
          run += c;
        }
      }
      __syncwarp();
      for (int q0 = p; q0 < end; q0 += 32) {
        const int q = q0 + lane;
        const bool valid = q < end;
        Peak k = first;
        int dy = dy0;
        if (q0 != p) {
          dy = kMaxW;
          if (valid) {
            k = load(q);
            dy = finish(k);
          }
        }
        if (!valid) dy = kMaxW;
        // lanes with the same in-tile row: a ballot per row for small
        // windows (the match instruction's unit is slow), a match otherwise;
        // lanes past the group (dy = kMaxW) use none of it
        unsigned peers = 0;
        if (a.w <= 8) {
          for (int d = 0; d < a.w; ++d) {
            const unsigned b = __ballot_sync(0xffffffffu, dy == d);
            if (dy == d) peers = b;
          }
        } else {
          peers = __match_any_sync(0xffffffffu, dy);
        }
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int off = valid ? cnt[dy] : 0;
        __syncwarp();
        if (valid) {
          const int pos = base + p + off + rank;
          if (pos < a.cap) a.out[pos] = k.c;
          if (lane == __ffs(peers) - 1) cnt[dy] = off + __popc(peers);
        }
        __syncwarp();
      }
    }
  }
}

// Image branch with the march's in-tile arg-max, w <= kRowsMaxW and rows of at
// most 32 bitmap words (Tx <= 1024), straight from the peak bitmap: one warp
// per tile row, one word per lane, writes the row's candidates in (snapshot,
// y, x) order.  Inside a tile row that order is (dy, tx), so a peak's place is
// the row's offset (from the scan of the rows' peak counts), the row's peaks
// in lower in-tile rows, and the peaks of its own in-tile row at smaller tx
// (warp scans of each lane's count per in-tile row).  Each lane reads the
// arg-max byte and value of its first kRowsBatch peaks together and keeps
// them; a lane with more reads the rest again.  The same candidates as
// k_group_sort<true> on the compacted peak list, without that list.
constexpr int kRowsMaxW = 8;
constexpr int kRowsBatch = 4;
__global__ void __launch_bounds__(kPbThreads, 4) k_emit_rows(CandArgs a, const float* __restrict__ vals,
                                                          int64_t nrows, BlockScratch b,
                                                          int64_t cap, const int* base_) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * kPbThreads + threadIdx.x) >> 5;
  if (r >= nrows) return;
  const int w = a.w;
  const int g = (int)(r / a.Ty), ty = (int)(r - (int64_t)g * a.Ty);
  const int t0 = ty * a.Tx;
  const uint32_t* row = b.pbits + (size_t)r * b.words;
  const uint8_t* ag = a.arg + (size_t)g * a.stride + t0;
  const float* vg = vals + (size_t)g * a.stride + t0;
  const int64_t roff = row_offset(b, r);
  const int64_t base = *base_;
  // one word per lane: each lane's first kRowsBatch peaks are read once
  // (arg-max byte and value together) and kept; a lane with more reads the
  // rest again
  const uint32_t word = lane < b.words ? row[lane] : 0u;
  int idx[kRowsBatch], tx[kRowsBatch];
  float v[kRowsBatch];
  uint32_t m = word;
#pragma unroll
  for (int k = 0; k < kRowsBatch; ++k) {
    idx[k] = -1;
    tx[k] = 0;
    v[k] = 0.f;
    if (m) {
      tx[k] = lane * 32 + __ffs(m) - 1;
      m &= m - 1;
      idx[k] = ag[tx[k]];
      v[k] = vg[tx[k]];
    }
  }
  const uint32_t rest = m;
  int mine[kRowsMaxW];
#pragma unroll
  for (int d = 0; d < kRowsMaxW; ++d) mine[d] = 0;
#pragma unroll
  for (int k = 0; k < kRowsBatch; ++k) {
    const int dy = idx[k] >= 0 ? idx[k] / w : -1;
#pragma unroll
    for (int d = 0; d < kRowsMaxW; ++d) mine[d] += dy == d;
  }
  for (uint32_t q = rest; q; q &= q - 1) {
    const int dy = ag[lane * 32 + __ffs(q) - 1] / w;
#pragma unroll
    for (int d = 0; d < kRowsMaxW; ++d) mine[d] += dy == d;
  }
  // place of this lane's first peak of each in-tile row: the row's peaks
  // in lower in-tile rows, then the lower lanes' peaks of that row
  int excl[kRowsMaxW];
  int run = 0;
#pragma unroll
  for (int d = 0; d < kRowsMaxW; ++d) {
    int incl = mine[d];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    excl[d] = run + incl - mine[d];
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  auto put = [&](int t, int i, float val) {
    const int dy = i / w, dx = i - dy * w;
    int j = 0;
#pragma unroll
    for (int d = 0; d < kRowsMaxW; ++d)
      if (dy == d) j = excl[d]++;
    const int64_t n = roff + j;   // place among the image candidates
    const int64_t pos = base + n;
    if (n < cap && pos < a.cap) a.out[pos] = image_candidate(a, SelItem{g, t0 + t, val}, t, ty, w, dx, dy);
  };
#pragma unroll
  for (int k = 0; k < kRowsBatch; ++k)
    if (idx[k] >= 0) put(tx[k], idx[k], v[k]);
  for (uint32_t q = rest; q; q &= q - 1) {
    const int t = lane * 32 + __ffs(q) - 1;
    put(t, ag[t], vg[t]);
  }
}

__global__ void k_add_count(int* total, const int* part) {
  pdl_begin();
  *total += *part;
}

// Copies the first min(*n, cap) candidates to mapped host memory, so only the
// candidates that exist cross the host link.
__global__ void k_export(const fitrig_candidate* __restrict__ src, const int* n,
                         fitrig_candidate* dst, int cap) {
  const int m = min(*n, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    dst[i] = src[i];
}

cudaError_t launch_export_candidates(const fitrig_candidate* src, const int* n,
                                     fitrig_candidate* dst, int cap, cudaStream_t st) {
  k_export<<<64, 256, 0, st>>>(src, n, dst, cap);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_emit_peaks(const CandArgs& a, const SelItem* peaks, const int* npeak,
                              int* base, fitrig_candidate* tmp, cudaStream_t st) {
  cudaError_t e;
  if (a.branch == FITRIG_BRANCH_FREQ) {
    e = launch_pdl(k_emit_freq, dim3(152 * 4), dim3(256), 0, st, a, peaks, npeak,
                   (const int*)nullptr);
    count_launches(1);
  } else if (a.arg) {
    e = launch_pdl(k_group_sort<true>, dim3(152 * 4), dim3(kGroupWarps * 32), 0, st, a, npeak,
                   (const fitrig_candidate*)tmp, peaks, (const int*)nullptr, (const int*)base);
    count_launches(1);
  } else {
    e = launch_pdl(k_emit_image, dim3(152 * 4), dim3(256), 0, st, a, peaks, npeak,
                   (const int*)nullptr, tmp);
    if (e == cudaSuccess)
      e = launch_pdl(k_group_sort<false>, dim3(152 * 4), dim3(kGroupWarps * 32), 0, st, a, npeak,
                     (const fitrig_candidate*)tmp, peaks, (const int*)nullptr, (const int*)base);
    count_launches(2);
  }
  if (e == cudaSuccess) e = launch_pdl(k_add_count, dim3(1), dim3(1), 0, st, a.nout, npeak);
  count_launches(1);
  return e;
}

cudaError_t launch_emit_rows(const CandArgs& a, const float* vals, int groups, const BlockScratch& b,
                             int64_t cap, int* base, cudaStream_t st) {
  if (!a.arg || a.w < 1 || a.w > kRowsMaxW || b.words > 32 ||
      ((int64_t)groups * a.Ty + kRowsPerCta - 1) / kRowsPerCta > b.nblk)
    return cudaErrorInvalidValue;
  const int64_t nrows = (int64_t)groups * a.Ty;
  cudaError_t e = launch_pdl(k_emit_rows, dim3((unsigned)((nrows * 32 + kPbThreads - 1) / kPbThreads)),
                             dim3(kPbThreads), 0, st, a, vals, nrows, b, cap, (const int*)base);
  if (e == cudaSuccess)
    e = launch_pdl(k_add_count, dim3(1), dim3(1), 0, st, a.nout, (const int*)&b.counters[2]);
  count_launches(2);
  return e;
}

cudaError_t launch_emit_candidates(const CandArgs& a, const SelectScratch& s, int* base,
                                   fitrig_candidate* tmp, unsigned* status, cudaStream_t st) {
  // ordered list of component peaks
  k_peak_count<<<s.nblk, kSelThreads, 0, st>>>(s.nsel, s.parent, s.peak, s.nblk, s.blkcnt);
  k_scan_blocks<<<1, 1024, 0, st>>>(s.nblk, s.blkcnt, s.blkoff, s.npeak, s.capacity, status,
                                    nullptr);
  k_peak_write<<<s.nblk, kSelThreads, 0, st>>>(s.nsel, s.parent, s.peak, s.nblk, s.blkoff,
                                               s.plist);
  if (a.branch == FITRIG_BRANCH_FREQ) {
    k_emit_freq<<<152 * 4, 256, 0, st>>>(a, s.items, s.npeak, s.plist);
    count_launches(4);
  } else {
    if (a.arg) {
      k_group_sort<true><<<152 * 4, kGroupWarps * 32, 0, st>>>(a, s.npeak, tmp, s.items, s.plist,
                                                               base);
      count_launches(4);
    } else {
      k_emit_image<<<152 * 4, 256, 0, st>>>(a, s.items, s.npeak, s.plist, tmp);
      k_group_sort<false><<<152 * 4, kGroupWarps * 32, 0, st>>>(a, s.npeak, tmp, s.items,
                                                                s.plist, base);
      count_launches(5);
    }
  }
  // running total of candidates
  k_add_count<<<1, 1, 0, st>>>(a.nout, s.npeak);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace fitrig
