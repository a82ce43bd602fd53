// Stack-march tile statistics: one HBM pass over the snapshot stack.
//
// For every tile t and unit s (snapshots s, s+1, s+2) this computes, following
// Eq. (tLISI) and Eq. 3-5 of the paper (Sec. 2.2.4), with the sum form of the
// kernel equation in Sec. 2.3:
//   D^(s)   = |x^(s+1) - x^(s)|,  D^(s+1) = |x^(s+2) - x^(s+1)|
//   Delta   = |D^(s) - D^(s+1)|
//   r       = min(Delta / x-hat^(s+1), 1),  x-hat = C if x == 0 else |x| (or x)
//   v_t     = (sum Delta / n_t) * max Delta * (sum r / n_t)
// so that tLISI_t = 1 - v_t / M^2; M is one scalar for the stack and is
// reduced here too (max over every pixel, Eq. tLISI denominator).
//
// GB300 design (differs from the paper's one-block-per-tile kernel, which
// re-reads a materialised Delta image per unit):
//   * a CTA owns a box of TBX x TBY tiles and marches through time; each
//     snapshot box arrives by a 3-D TMA load into a ring of shared-memory
//     stages completed on mbarriers, so every stack pixel is read from HBM once;
//   * each thread owns one pixel column of R rows of a tile band and carries
//     x^(s+1) and D^(s) in registers from one snapshot to the next, so Delta and
//     r never touch memory;
//   * per-thread partial sums go to shared memory once per snapshot, and one
//     warp per tile combines them in a fixed order (deterministic).
// The one __syncthreads per snapshot also guards the reuse of ring stages, so
// no "empty" barriers are needed.
//
// Difference-coded half storage (FITRIG_CODING_DELTA): the stack holds an FP32
// key frame (snapshot 0, outside the TMA ring) and half-rounded differences
// q^(s); the thread-per-tile marches decode xt^(s) = fl32(xt^(s-1) + q^(s)) in
// the registers that already carry x^(s+1), so the rest of the arithmetic is
// the FP32 march on the decoded values.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "internal.cuh"

namespace fitrig {

constexpr int kStackMaxThreads = 512;
constexpr int kSmallMaxThreads = 256;   // thread-per-tile path: 32 x TBY tiles per CTA
constexpr int kSmallMaxW = 6;

// Approximate reciprocal (rcp.approx.ftz: relative error below 2^-23).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Maximum of v over the calling threads into *key.  Full warps reduce with
// shuffles first; the threads of a trailing partial warp (a block size that is
// not a multiple of 32) go straight to the atomic.
__device__ __forceinline__ void max_to(float v, unsigned* key, bool full_warp) {
  if (full_warp) {
    warp_max_to(v, key);
    return;
  }
  if (v > -INFINITY) atomicMax(key, f32_key(v));
}

template <typename T, int R, bool SIGNED>
__global__ void __launch_bounds__(kStackMaxThreads) k_stack_tile(const __grid_constant__ CUtensorMap tmap,
                                                     const StackArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const StackGeom& g = a.g;
  const int NS = g.stages;
  float4* part = reinterpret_cast<float4*>(smem + (size_t)NS * g.stage_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(part + 2 * g.threads);

  const int tid = threadIdx.x;
  const int c = tid % g.BW;
  const int rest = tid / g.BW;
  const int band = rest / g.nseg;
  const int seg = rest - band * g.nseg;
  const int rcount = min(R, g.w - seg * R);
  const int row0 = band * g.w + seg * R;
  const int x0 = blockIdx.x * g.BW;
  const int y0 = blockIdx.y * g.BH;
  const int xload = g.aligned ? x0 : (x0 & ~7);
  const int col = (x0 - xload) + c;
  const uint32_t bar0 = smem_u32(bars);
  const uint32_t stage0 = smem_u32(smem);
  const uint32_t box_bytes = (uint32_t)(g.boxW * g.BH * (int)sizeof(T));
  const int L = a.nsnap;

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int i = 0; i < NS; ++i) mbar_init(bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < NS && j < L; ++j) {
      mbar_expect_tx(bar0 + 8 * j, box_bytes);
      tma_load_3d(stage0 + j * (uint32_t)g.stage_bytes, &tmap, xload, y0, (a.zrot + j) % L, bar0 + 8 * j);
    }
  }

  float xp[R], dp[R];
#pragma unroll
  for (int i = 0; i < R; ++i) xp[i] = dp[i] = 0.f;
  float mx = -INFINITY;
  const uint64_t deadline = globaltimer_ns() + a.timeout_ns;

  int stg = 0;
  uint32_t phase = 0;
  for (int j = 0; j < L; ++j) {
    const bool ok = mbar_wait_bounded(bar0 + 8 * stg, phase, deadline);
    const T* st = reinterpret_cast<const T*>(smem + (size_t)stg * g.stage_bytes);
    float sm = -INFINITY;   // this snapshot's maximum over the thread's pixels
    if (ok) {
      if (j >= 2) {
        float s1 = 0.f, s2 = 0.f, s3 = 0.f;
        // ABS reading: when none of the column's x^(s+1) is zero (its smallest
        // |x| is not), r = sat(Delta * |1/x|) needs no guard (as in the
        // thread-per-tile march); otherwise every pixel takes the guarded form.
        float mn = INFINITY;
        if (!SIGNED) {
#pragma unroll
          for (int i = 0; i < R; ++i)
            if (i < rcount) mn = fminf(mn, fabsf(xp[i]));
        }
        const bool fast = !SIGNED && mn != 0.f;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (i < rcount) {
            const float xn = to_f32(st[(row0 + i) * g.boxW + col]);
            sm = fmaxf(sm, xn);
            const float dn = fabsf(xn - xp[i]);        // D^(s+1)
            const float d = fabsf(dn - dp[i]);         // Delta
            float r;
            if (fast) {
              r = __saturatef(d * fabsf(rcp_approx(xp[i])));
            } else {
              const float ref = SIGNED ? xp[i] : fabsf(xp[i]);
              const float xh = (xp[i] == 0.f) ? kGuardC : ref;   // Eq. 5
              r = fminf(__fdividef(d, xh), 1.f);                 // Eq. 4
            }
            s1 += d;
            s2 = fmaxf(s2, d);
            s3 += r;
            dp[i] = dn;
            xp[i] = xn;
          }
        }
        part[(j & 1) * g.threads + tid] = make_float4(s1, s2, s3, 0.f);
      } else {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (i < rcount) {
            const float xn = to_f32(st[(row0 + i) * g.boxW + col]);
            sm = fmaxf(sm, xn);
            dp[i] = fabsf(xn - xp[i]);   // D^(0) once j == 1
            xp[i] = xn;
          }
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      // A stage never completed: flag it, let in-flight copies land (bounded),
      // and leave.  No thread touches the ring after this point.
      if (tid == 0) {
        atomicOr(a.status, kErrTimeout);
        const uint64_t d2 = globaltimer_ns() + 1000000ull;
        for (int jj = j; jj < L && jj < j + NS; ++jj)
          mbar_wait_bounded(bar0 + 8 * (jj % NS), (uint32_t)((jj / NS) & 1), d2);
      }
      return;
    }
    mx = fmaxf(mx, sm);
    const bool full_warp = (tid >> 5) < (g.threads >> 5);
    if (a.smax) max_to(sm, a.smax + j, full_warp);
    if (tid == 0 && j + NS < L) {
      fence_proxy_async_smem();
      mbar_expect_tx(bar0 + 8 * stg, box_bytes);
      tma_load_3d(stage0 + stg * (uint32_t)g.stage_bytes, &tmap, xload, y0, (a.zrot + j + NS) % L,
                  bar0 + 8 * stg);
    }
    if (++stg == NS) {
      stg = 0;
      phase ^= 1u;
    }
    if (j >= 2) {
      // One full warp per tile combines the tile's nseg * w column partials:
      // lanes stride over them, then a fixed shuffle tree (deterministic).
      // Warps take tiles round-robin; a trailing partial warp takes none.
      const int warp = tid >> 5, lane = tid & 31, nwf = g.threads >> 5;
      const int NT = g.TBX * g.TBY, per = g.nseg * g.w;
      const float4* pp = part + (j & 1) * g.threads;
      for (int tt = warp; tt < NT && warp < nwf; tt += nwf) {
        const int tb = tt / g.TBX;
        const int tbx = tt - tb * g.TBX;
        float S1 = 0.f, S2 = 0.f, S3 = 0.f;
        for (int i = lane; i < per; i += 32) {
          const int sg = i / g.w, cc = i - sg * g.w;
          const float4 q = pp[(tb * g.nseg + sg) * g.BW + tbx * g.w + cc];
          S1 += q.x;
          S2 = fmaxf(S2, q.y);
          S3 += q.z;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          S1 += __shfl_xor_sync(0xffffffffu, S1, o);
          S2 = fmaxf(S2, __shfl_xor_sync(0xffffffffu, S2, o));
          S3 += __shfl_xor_sync(0xffffffffu, S3, o);
        }
        const int tx = blockIdx.x * g.TBX + tbx;
        const int ty = blockIdx.y * g.TBY + tb;
        if (lane == 0 && tx < a.Tx && ty < a.Ty) {
          const int hw = min(g.w, a.ny - ty * g.w);
          const int ww = min(g.w, a.nx - tx * g.w);
          const float n = (float)(hw * ww);
          float v = (S1 / n) * S2 * (S3 / n);
          if (!isfinite(S1) || !isfinite(v)) v = NAN;
          a.vp[(size_t)(j - 2) * (size_t)a.vstride + (size_t)ty * a.Tx + tx] = v;
        }
      }
    }
  }
  (void)stg;
  // Global maximum M (NaN ignored by fmaxf; +inf is resolved on the host).
  max_to(mx, a.gmax, (tid >> 5) < (g.threads >> 5));
}

// Small windows (W <= 6): one thread owns a whole W x W tile and keeps its
// W*W pixels' x^(s+1) and D^(s) in registers, so a tile's sums and maximum
// never leave the thread.  A warp covers 32 tiles side by side (lane t reads
// columns W*t .. W*t+W-1 of the stage, which spreads over all banks for odd W);
// the CTA covers 32 x TBY tiles (TBY and the ring depth are tunable).  One
// barrier per snapshot guards the ring.

// The TMA ring of one CTA.  Stage and phase advance with every snapshot
// consumed and carry over from one box to the next (persistent kernels).
struct Ring {
  uint32_t bar0, stage0;
  uint32_t box_bytes;
  int NS;
  uint32_t stage_bytes;
  int stg;          // next stage to consume
  uint32_t phase;   // its parity
};

// One field as the march sees it.
struct FieldView {
  int nx, ny, L, Tx, Ty;
  int zrot;
  const float* key = nullptr;   // FP32 key frame of a difference-coded stack
  int64_t kpitch = 0;
  int64_t vstride;
  float* vp;
  uint8_t* arg;
  unsigned* smax;
  unsigned* status;
};

__device__ __forceinline__ void ring_init(Ring& rg, unsigned char* smem, const StackGeom& g,
                                          int elem) {
  rg.NS = g.stages;
  rg.stage_bytes = (uint32_t)g.stage_bytes;
  rg.box_bytes = (uint32_t)(g.boxW * g.BH * elem);
  rg.stage0 = smem_u32(smem);
  rg.bar0 = smem_u32(smem + (size_t)g.stages * g.stage_bytes);
  rg.stg = 0;
  rg.phase = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < rg.NS; ++i) mbar_init(rg.bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncthreads();
}

// Running maximum over one tile row, two pixels per three-input max.
template <int W>
__device__ __forceinline__ float row_max(float m, const float* xn) {
#pragma unroll
  for (int q = 0; q + 1 < W; q += 2) m = max3f(m, xn[q], xn[q + 1]);
  if (W & 1) m = fmaxf(m, xn[W - 1]);
  return m;
}

// r of Eq. 4/5 from Delta (>= 0) and the reference intensity x^(s+1), with
// the guard x-hat = C where x == 0.  In the ABS reading x-hat = |x|, so the
// quotient is never negative and the multiply's saturation to [0, 1] is the
// clamp min(., 1).
template <bool SIGNED>
__device__ __forceinline__ float r_term(float d, float xref) {
  if (SIGNED) {
    const float xh = (xref == 0.f) ? kGuardC : xref;
    return fminf(__fdividef(d, xh), 1.f);
  }
  const float xh = (xref == 0.f) ? kGuardC : fabsf(xref);
  return __saturatef(__fdividef(d, xh));
}

// Waits for the ring's current stage (bounded); false when it never completed.
__device__ __forceinline__ bool ring_wait(const Ring& rg, uint64_t deadline) {
  return mbar_wait_bounded(rg.bar0 + 8 * rg.stg, rg.phase, deadline);
}

// After every thread has consumed the current stage (snapshot j of L): on a
// failed wait anywhere in the CTA, flag it, let copies in flight land
// (bounded) and return false; otherwise refill the stage with snapshot
// j + NS and advance the ring.
__device__ __forceinline__ bool ring_release(Ring& rg, bool ok, const CUtensorMap* tmap,
                                             unsigned* status, int j, int L, int x0, int y0,
                                             int zrot) {
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicOr(status, kErrTimeout);
      const uint64_t d2 = globaltimer_ns() + 1000000ull;
      int s = rg.stg;
      uint32_t ph = rg.phase;
      for (int jj = j; jj < L && jj < j + rg.NS; ++jj) {
        mbar_wait_bounded(rg.bar0 + 8 * s, ph, d2);
        if (++s == rg.NS) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    return false;
  }
  if (threadIdx.x == 0 && j + rg.NS < L) {
    fence_proxy_async_smem();
    mbar_expect_tx(rg.bar0 + 8 * rg.stg, rg.box_bytes);
    tma_load_3d(rg.stage0 + rg.stg * rg.stage_bytes, tmap, x0, y0, (zrot + j + rg.NS) % L,
                rg.bar0 + 8 * rg.stg);
  }
  if (++rg.stg == rg.NS) {
    rg.stg = 0;
    rg.phase ^= 1u;
  }
  return true;
}

// One tile row of W stage elements into FP32.  For W = 4 the row is one
// 16-byte (FP32) or 8-byte (half) shared-memory load: a lane's row starts at a
// multiple of 4 elements, and four scalar loads at a 4-word lane stride would
// meet 4-way bank conflicts.
template <typename T, int W>
__device__ __forceinline__ void load_row(const T* src, float* dst) {
  if constexpr (W == 4 && sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(src);
    dst[0] = v.x;
    dst[1] = v.y;
    dst[2] = v.z;
    dst[3] = v.w;
  } else if constexpr (W == 4 && sizeof(T) == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(src);
    const uint16_t h[4] = {(uint16_t)(v.x & 0xffffu), (uint16_t)(v.x >> 16),
                           (uint16_t)(v.y & 0xffffu), (uint16_t)(v.y >> 16)};
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = to_f32(T{h[q]});
  } else {
#pragma unroll
    for (int q = 0; q < W; ++q) dst[q] = to_f32(src[q]);
  }
}

// One unit of the thread's W x W tile: from x^(s+1) (xp) and D^(s) (dp) and
// the stage holding x^(s+2), writes x^(s+2) to xn and D^(s+1) to dn (separate
// arrays, so that the caller alternates them and no value is copied), and
// returns the tile sums.  Row partials first, then the rows in order: short
// dependency chains for the sums, the maximum with its first position in
// row-major order (strict >), and this snapshot's maximum sm.
//
// ABS reading: for x != 0, r = sat(Delta * |1/x|) needs no guard.  A row whose
// reference pixels multiply to a non-zero product has no zero among them and
// takes that form; any other row (a zero pixel, the zero fill outside the
// image, or a product that underflows) takes the guarded form of Eq. 5.  Both
// give the same r for a non-zero x.
// With DELTA the stage holds the differences q^(s+2) and the row is decoded
// first: x^(s+2) = fl32(x^(s+1) + q^(s+2)), the coder's own sum.
template <typename T, int W, bool SIGNED, bool DELTA = false>
__device__ __forceinline__ void tile_unit(const T* st, const float (&xp)[W * W],
                                          const float (&dp)[W * W], float (&xn)[W * W],
                                          float (&dn)[W * W], float& sm, float& s1, float& s2,
                                          float& s3, int& am) {
  s1 = 0.f;
  s2 = 0.f;
  s3 = 0.f;
  am = 0;
#pragma unroll
  for (int r = 0; r < W; ++r) {
    float r1 = 0.f, r3 = 0.f, rm = 0.f;
    int ri = 0;
    float dd[W];
    load_row<T, W>(st + r * (32 * W), &xn[r * W]);
    if (DELTA) {
#pragma unroll
      for (int q = 0; q < W; ++q) xn[r * W + q] = __fadd_rn(xp[r * W + q], xn[r * W + q]);
    }
    sm = row_max<W>(sm, &xn[r * W]);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const int i = r * W + q;
      dn[i] = fabsf(xn[i] - xp[i]);       // D^(s+1)
      dd[q] = fabsf(dn[i] - dp[i]);       // Delta
      r1 += dd[q];
      if (dd[q] > rm) {
        rm = dd[q];
        ri = q;
      }
    }
    float pz = xp[r * W];
#pragma unroll
    for (int q = 1; q < W; ++q) pz *= xp[r * W + q];
    if (SIGNED || pz == 0.f) {
#pragma unroll
      for (int q = 0; q < W; ++q) r3 += r_term<SIGNED>(dd[q], xp[r * W + q]);
    } else {
#pragma unroll
      for (int q = 0; q < W; ++q) r3 += __saturatef(dd[q] * fabsf(rcp_approx(xp[r * W + q])));
    }
    s1 += r1;
    s3 += r3;
    if (rm > s2) {
      s2 = rm;
      am = r * W + ri;
    }
  }
}

// Snapshots 0 and 1 of a tile: x^(j) into xn, and D^(0) once j == 1.  With
// DELTA (snapshot 1 only) the stage holds q^(1), decoded against x^(0) in xp.
template <typename T, int W, bool DELTA = false>
__device__ __forceinline__ void tile_load(const T* st, const float (&xp)[W * W],
                                          float (&xn)[W * W], float (&dn)[W * W], bool first,
                                          float& sm) {
#pragma unroll
  for (int r = 0; r < W; ++r) {
    load_row<T, W>(st + r * (32 * W), &xn[r * W]);
    if (DELTA) {
#pragma unroll
      for (int q = 0; q < W; ++q) xn[r * W + q] = __fadd_rn(xp[r * W + q], xn[r * W + q]);
    }
    sm = row_max<W>(sm, &xn[r * W]);
  }
  if (!first) {
#pragma unroll
    for (int i = 0; i < W * W; ++i) dn[i] = fabsf(xn[i] - xp[i]);
  }
}

// The FP32 key frame of an H x W pixel block at (px, py) (plain loads: a warp
// reads whole rows of adjacent tiles), zero outside the analysed nx x ny
// region like the TMA fill of the differences.
template <int H, int W>
__device__ __forceinline__ void key_load(const float* key, int64_t kpitch, int px, int py, int nx,
                                         int ny, float (&xn)[H * W], float& sm) {
#pragma unroll
  for (int r = 0; r < H; ++r) {
    const int y = py + r;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const int x = px + q;
      xn[r * W + q] = (y < ny && x < nx) ? __ldg(key + (int64_t)y * kpitch + x) : 0.f;
    }
    sm = row_max<W>(sm, &xn[r * W]);
  }
}

// Marches box (bx, by) of a field through its snapshots; mx collects the
// running maximum.  Returns false (after flagging and draining, bounded) if a
// stage never completed; the caller must then leave.
// With DELTA, snapshot 0 is the key frame (no ring stage) and the ring
// carries the differences of snapshots 1..L-1.
template <typename T, int W, bool SIGNED, bool DELTA = false>
__device__ __forceinline__ bool march_small(const CUtensorMap* tmap, const FieldView& f, int bx,
                                            int by, int tby, Ring& rg, unsigned char* smem,
                                            uint64_t deadline, float& mx) {
  constexpr int N = W * W;
  const int tid = threadIdx.x;
  const int tbx = tid & 31;
  const int tb = tid >> 5;
  const int tx = bx * 32 + tbx;
  const int ty = by * tby + tb;
  const int L = f.L;
  const int x0 = bx * 32 * W, y0 = by * tby * W;
  const bool live = tx < f.Tx && ty < f.Ty;
  // 1 / n_t^2 of this tile (edge tiles are clipped)
  const int hw = live ? min(W, f.ny - ty * W) : 1;
  const int ww = live ? min(W, f.nx - tx * W) : 1;
  const float inv_n2 = 1.f / ((float)(hw * ww) * (float)(hw * ww));
  const int off = (tb * W) * (32 * W) + tbx * W;
  const int j0 = DELTA ? 1 : 0;   // first snapshot that comes through the ring
  if (tid == 0) {
    int s = rg.stg;
    for (int j = j0; j < j0 + rg.NS && j < L; ++j) {
      mbar_expect_tx(rg.bar0 + 8 * s, rg.box_bytes);
      tma_load_3d(rg.stage0 + s * rg.stage_bytes, tmap, x0, y0, (f.zrot + j) % L, rg.bar0 + 8 * s);
      if (++s == rg.NS) s = 0;
    }
  }
  const size_t tile = (size_t)ty * f.Tx + tx;
  float* out = f.vp + tile;
  uint8_t* aout = f.arg ? f.arg + tile : nullptr;
  auto stage = [&]() {
    return reinterpret_cast<const T*>(smem + (size_t)rg.stg * rg.stage_bytes) + off;
  };
  // Two register sets alternate between x^(s+1), D^(s) and x^(s+2), D^(s+1).
  float xa[N], da[N], xb[N], db[N];
  if (DELTA) {
    float sm = -INFINITY;
    key_load<W, W>(f.key, f.kpitch, x0 + tbx * W, y0 + tb * W, f.nx, f.ny, xa, sm);
    mx = fmaxf(mx, sm);
    if (f.smax) warp_max_to(sm, f.smax);
  }
#pragma unroll
  for (int j = j0; j < 2; ++j) {
    if (j >= L) break;
    const bool ok = ring_wait(rg, deadline);
    float sm = -INFINITY;
    if (ok) {
      if (j == 0) tile_load<T, W>(stage(), xb, xa, da, true, sm);
      else tile_load<T, W, DELTA>(stage(), xa, xb, db, false, sm);
    }
    if (!ring_release(rg, ok, tmap, f.status, j, L, x0, y0, f.zrot)) return false;
    mx = fmaxf(mx, sm);
    if (f.smax) warp_max_to(sm, f.smax + j);
  }
  // After the prologue x^(1) and D^(0) are in (xb, db) when L > 1.
  auto unit = [&](int j, const float (&xp)[N], const float (&dp)[N], float (&xn)[N],
                  float (&dn)[N]) -> bool {
    const bool ok = ring_wait(rg, deadline);
    float sm = -INFINITY;
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int am = 0;
    if (ok) tile_unit<T, W, SIGNED, DELTA>(stage(), xp, dp, xn, dn, sm, s1, s2, s3, am);
    if (!ring_release(rg, ok, tmap, f.status, j, L, x0, y0, f.zrot)) return false;
    mx = fmaxf(mx, sm);
    if (f.smax) warp_max_to(sm, f.smax + j);
    if (live) {
      float v = s1 * s2 * s3 * inv_n2;
      if (!isfinite(s1) || !isfinite(v)) v = NAN;
      out[(size_t)(j - 2) * (size_t)f.vstride] = v;
      if (aout) aout[(size_t)(j - 2) * (size_t)f.vstride] = (uint8_t)am;
    }
    return true;
  };
  for (int j = 2; j < L; j += 2) {
    if (!unit(j, xb, db, xa, da)) return false;
    if (j + 1 < L && !unit(j + 1, xa, da, xb, db)) return false;
  }
  return true;
}

__device__ __forceinline__ void block_max_to(float mx, unsigned* gmax) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > -INFINITY) atomicMax(gmax, f32_key(mx));
}

template <typename T, int W, bool SIGNED, bool DELTA>
__global__ void __launch_bounds__(kSmallMaxThreads) k_stack_small(const __grid_constant__ CUtensorMap tmap,
                                                               const StackArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (threadIdx.x == 0) prefetch_tmap(&tmap);
  Ring rg;
  ring_init(rg, smem, a.g, (int)sizeof(T));
  FieldView f;
  f.nx = a.nx;
  f.ny = a.ny;
  f.L = a.nsnap;
  f.Tx = a.Tx;
  f.Ty = a.Ty;
  f.zrot = a.zrot;
  f.vstride = a.vstride;
  f.vp = a.vp;
  f.arg = a.arg;
  f.smax = a.smax;
  f.status = a.status;
  f.key = a.key;
  f.kpitch = a.kpitch;
  float mx = -INFINITY;
  const uint64_t deadline = globaltimer_ns() + a.timeout_ns;
  if (!march_small<T, W, SIGNED, DELTA>(&tmap, f, blockIdx.x, blockIdx.y, a.g.TBY, rg, smem,
                                        deadline, mx))
    return;
  block_max_to(mx, a.gmax);
}

// Windows that are multiples of 4 up to 64 (8, 16, 32, 64): the thread-per-tile
// march on 4 x 4 sub-tiles.  Each thread keeps its sub-tile's x^(s+1) and
// D^(s) in registers (tile_unit with W = 4); a warp covers 128 columns x 4
// rows.  A w x w tile spans w/4 lanes and w/4 warps: its lanes combine by a
// shuffle tree, each warp leaves one partial per tile in shared memory, and
// after the ring barrier of the snapshot one thread per tile adds the w/4
// warp partials in order (deterministic).  The partials are double-buffered by
// unit parity, so the next unit's partials never overwrite ones being read.
constexpr int kSubCols = 128;   // 32 lanes x 4 columns

// Partials after the ring stages and their barriers, 16-byte aligned.
__host__ __device__ __forceinline__ size_t sub_part_offset_host(int stages, size_t stage_bytes) {
  return ((size_t)stages * stage_bytes + 8 * (size_t)stages + 15) / 16 * 16;
}
__device__ __forceinline__ size_t sub_part_offset(const StackGeom& g) {
  return sub_part_offset_host(g.stages, g.stage_bytes);
}

template <typename T, bool SIGNED, bool DELTA>
__device__ __forceinline__ bool march_sub(const CUtensorMap* tmap, const StackArgs& a, Ring& rg,
                                          unsigned char* smem, uint64_t deadline, float& mx) {
  constexpr int N = 16;
  const StackGeom& g = a.g;
  const int w = g.w, gl = w / 4;             // lanes (and warps) per tile side
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = g.threads >> 5;
  const int L = a.nsnap;
  const int x0 = blockIdx.x * kSubCols, y0 = blockIdx.y * g.BH;
  float4* part = reinterpret_cast<float4*>(smem + sub_part_offset(g));   // [2][nw][TBX]
  const int off = (warp * 4) * kSubCols + lane * 4;
  const int j0 = DELTA ? 1 : 0;   // first snapshot that comes through the ring
  if (tid == 0) {
    int s = rg.stg;
    for (int j = j0; j < j0 + rg.NS && j < L; ++j) {
      mbar_expect_tx(rg.bar0 + 8 * s, rg.box_bytes);
      tma_load_3d(rg.stage0 + s * rg.stage_bytes, tmap, x0, y0, (a.zrot + j) % L, rg.bar0 + 8 * s);
      if (++s == rg.NS) s = 0;
    }
  }
  auto stage = [&]() {
    return reinterpret_cast<const T*>(smem + (size_t)rg.stg * rg.stage_bytes) + off;
  };
  // the tile this thread reduces after each barrier (one per tile of the CTA)
  const int NT = g.TBX * g.TBY;
  const int rtb = tid / g.TBX, rtc = tid - (tid / g.TBX) * g.TBX;
  const int rtx = blockIdx.x * g.TBX + rtc, rty = blockIdx.y * g.TBY + rtb;
  const bool rlive = tid < NT && rtx < a.Tx && rty < a.Ty;
  float inv_n = 0.f;
  if (rlive) {
    const int hw = min(w, a.ny - rty * w), ww = min(w, a.nx - rtx * w);
    inv_n = 1.f / (float)(hw * ww);
  }
  float* out = a.vp + (rlive ? (size_t)rty * a.Tx + rtx : 0);
  float xa[N], da[N], xb[N], db[N];
  if (DELTA) {
    float sm = -INFINITY;
    key_load<4, 4>(a.key, a.kpitch, x0 + lane * 4, y0 + warp * 4, a.nx, a.ny, xa, sm);
    mx = fmaxf(mx, sm);
    if (a.smax) warp_max_to(sm, a.smax);
  }
#pragma unroll
  for (int j = j0; j < 2; ++j) {
    if (j >= L) break;
    const bool ok = ring_wait(rg, deadline);
    float sm = -INFINITY;
    if (ok) {
      if (j == 0) tile_load<T, 4>(stage(), xb, xa, da, true, sm);
      else tile_load<T, 4, DELTA>(stage(), xa, xb, db, false, sm);
    }
    if (!ring_release(rg, ok, tmap, a.status, j, L, x0, y0, a.zrot)) return false;
    mx = fmaxf(mx, sm);
    if (a.smax) warp_max_to(sm, a.smax + j);
  }
  auto unit = [&](int j, const float (&xp)[N], const float (&dp)[N], float (&xn)[N],
                  float (&dn)[N]) -> bool {
    const bool ok = ring_wait(rg, deadline);
    float sm = -INFINITY;
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int am = 0;
    if (ok) tile_unit<T, 4, SIGNED, DELTA>(stage(), xp, dp, xn, dn, sm, s1, s2, s3, am);
    for (int o = gl >> 1; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 = fmaxf(s2, __shfl_xor_sync(0xffffffffu, s2, o));
      s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    float4* pp = part + (size_t)(j & 1) * nw * g.TBX;
    if (lane % gl == 0) pp[warp * g.TBX + lane / gl] = make_float4(s1, s2, s3, 0.f);
    if (!ring_release(rg, ok, tmap, a.status, j, L, x0, y0, a.zrot)) return false;
    mx = fmaxf(mx, sm);
    if (a.smax) warp_max_to(sm, a.smax + j);
    if (rlive) {
      float S1 = 0.f, S2 = 0.f, S3 = 0.f;
      for (int k = 0; k < gl; ++k) {
        const float4 q = pp[(rtb * gl + k) * g.TBX + rtc];
        S1 += q.x;
        S2 = fmaxf(S2, q.y);
        S3 += q.z;
      }
      float v = (S1 * inv_n) * S2 * (S3 * inv_n);
      if (!isfinite(S1) || !isfinite(v)) v = NAN;
      out[(size_t)(j - 2) * (size_t)a.vstride] = v;
    }
    return true;
  };
  for (int j = 2; j < L; j += 2) {
    if (!unit(j, xb, db, xa, da)) return false;
    if (j + 1 < L && !unit(j + 1, xa, da, xb, db)) return false;
  }
  return true;
}

// MAXT = 256 (w <= 32, eight warps) leaves room for three CTAs per SM;
// MAXT = 512 (w = 64, sixteen warps) for one.
template <typename T, bool SIGNED, int MAXT, bool DELTA>
__global__ void __launch_bounds__(MAXT, MAXT == 256 ? 3 : 1) k_stack_sub(const __grid_constant__ CUtensorMap tmap,
                                                                const StackArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (threadIdx.x == 0) prefetch_tmap(&tmap);
  Ring rg;
  ring_init(rg, smem, a.g, (int)sizeof(T));
  float mx = -INFINITY;
  const uint64_t deadline = globaltimer_ns() + a.timeout_ns;
  if (!march_sub<T, SIGNED, DELTA>(&tmap, a, rg, smem, deadline, mx)) return;
  block_max_to(mx, a.gmax);
}

// Persistent form over many fields (one launch for a whole batch): each CTA
// takes the next (field, box) item from a global counter until none is left;
// fields are ordered largest first.  Every field has its own TMA descriptor in
// global memory; the ring carries over between items.
template <typename T, int W, bool SIGNED>
__global__ void __launch_bounds__(kSmallMaxThreads) k_stack_multi(const FieldDesc* __restrict__ fields,
                                                               int nfields, int64_t nitems,
                                                               unsigned long long* counter,
                                                               const StackGeom g,
                                                               uint64_t timeout_ns) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ long long s_item;
  __shared__ int s_field;
  Ring rg;
  ring_init(rg, smem, g, (int)sizeof(T));
  const uint64_t deadline = globaltimer_ns() + timeout_ns;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = (long long)atomicAdd(counter, 1ull);
      int lo = 0, hi = nfields - 1;   // last field with item0 <= it
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fields[mid].item0 <= it) lo = mid; else hi = mid - 1;
      }
      s_item = it;
      s_field = lo;
    }
    __syncthreads();
    const long long it = s_item;
    const int fi = s_field;
    __syncthreads();   // everyone has read the item before thread 0 fetches the next
    if (it >= nitems) return;
    const FieldDesc& d = fields[fi];
    const long long b = it - d.item0;
    FieldView f;
    f.nx = d.nx;
    f.ny = d.ny;
    f.L = d.L;
    f.Tx = d.Tx;
    f.Ty = d.Ty;
    f.zrot = d.zrot;
    f.vstride = d.vstride;
    f.vp = d.vp;
    f.arg = d.arg;
    f.smax = d.smax;
    f.status = d.status;
    float mx = -INFINITY;
    if (!march_small<T, W, SIGNED>(&d.tmap, f, (int)(b % d.gridX), (int)(b / d.gridX), g.TBY, rg,
                                   smem, deadline, mx))
      return;
    block_max_to(mx, d.gmax);
  }
}

// Finite maximum over the stack; used only when the fused maximum saw +inf.
template <typename T>
__global__ void k_finite_max(const T* __restrict__ x, int L, int ny, int nx, int64_t pitch,
                             unsigned* gmax) {
  float m = -INFINITY;
  const int64_t total = (int64_t)L * ny * nx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / ((int64_t)ny * nx);
    const int64_t rem = i - s * ny * nx;
    const int64_t yy = rem / nx, xx = rem - yy * nx;
    const float v = to_f32(x[(s * ny + yy) * pitch + xx]);
    if (isfinite(v)) m = fmaxf(m, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > -INFINITY) atomicMax(gmax, f32_key(m));
}

// Finite maxima of a difference-coded stack, each pixel decoded in snapshot
// order (xt^(0) = key, xt^(s) = fl32(xt^(s-1) + q^(s)), as the march does);
// used only when a fused maximum saw +inf.  With smax, shared memory holds one
// flag (smax[k] was +inf) and one running key per snapshot.
template <typename T>
__global__ void k_delta_finite_max(const float* __restrict__ key, int64_t kpitch,
                                   const T* __restrict__ q, size_t slice, int L, int ny, int nx,
                                   int64_t pitch, unsigned* gmax, unsigned* smax) {
  extern __shared__ unsigned sk[];   // [L] flags, [L] keys (only with smax)
  const unsigned inf_key = f32_key(INFINITY);
  if (smax) {
    int any = 0;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
      sk[k] = smax[k] == inf_key ? 1u : 0u;
      sk[L + k] = 0u;
      any |= (int)sk[k];
    }
    // nothing to do unless a snapshot's fused maximum was +inf (the usual
    // case for the per-snapshot maxima of the running reading)
    if (!__syncthreads_or(any) && !gmax) return;
  }
  float m = -INFINITY;
  const int64_t total = (int64_t)ny * nx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t yy = i / nx, xx = i - yy * nx;
    float x = key[yy * kpitch + xx];
    for (int k = 0; k < L; ++k) {
      if (k > 0) x = __fadd_rn(x, to_f32(q[(size_t)k * slice + yy * pitch + xx]));
      if (isfinite(x)) {
        m = fmaxf(m, x);
        if (smax && sk[k]) atomicMax(&sk[L + k], f32_key(x));
      }
    }
  }
  if (gmax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > -INFINITY) atomicMax(gmax, f32_key(m));
  }
  if (smax) {
    __syncthreads();
    for (int k = threadIdx.x; k < L; k += blockDim.x)
      if (sk[k] && sk[L + k]) atomicMax(&smax[L + k], sk[L + k]);
  }
}

cudaError_t launch_delta_finite_max(const float* key, int64_t kpitch, const void* stack,
                                    int storage, int L, int ny, int nx, int64_t pitch,
                                    unsigned* gmax, unsigned* smax, cudaStream_t st) {
  if (smax && L > kDeltaMaxSnaps) return cudaErrorInvalidValue;
  const size_t slice = (size_t)pitch * ny;
  const size_t sm = smax ? sizeof(unsigned) * 2 * (size_t)L : 0;
  const int64_t total = (int64_t)ny * nx;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(152 * 4, (total + 255) / 256));
  if (storage == FITRIG_BF16) {
    auto kern = k_delta_finite_max<bf16_t>;
    if (sm > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
      if (e != cudaSuccess) return e;
    }
    kern<<<blocks, 256, sm, st>>>(key, kpitch, static_cast<const bf16_t*>(stack), slice, L, ny, nx,
                                  pitch, gmax, smax);
  } else if (storage == FITRIG_F16) {
    auto kern = k_delta_finite_max<f16_t>;
    if (sm > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
      if (e != cudaSuccess) return e;
    }
    kern<<<blocks, 256, sm, st>>>(key, kpitch, static_cast<const f16_t*>(stack), slice, L, ny, nx,
                                  pitch, gmax, smax);
  } else {
    return cudaErrorInvalidValue;
  }
  count_launches(1);
  return cudaGetLastError();
}

// One bounded wait on an mbarrier that nothing completes (fitrig_wait_probe):
// the same helper as the march's waits; reports whether it gave up.
__global__ void k_wait_probe(uint64_t timeout_ns, unsigned* gave_up) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  fence_mbar_init();
  const bool ok = mbar_wait_bounded(b, 0u, globaltimer_ns() + timeout_ns);
  *gave_up = ok ? 0u : 1u;
}

cudaError_t launch_wait_probe(uint64_t timeout_ns, unsigned* gave_up, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(timeout_ns, gave_up);
  count_launches(1);
  return cudaGetLastError();
}

bool small_geometry(int w, int elem_bytes, int tby, int stages, StackGeom* g) {
  // 32 tiles across (lane = tile), TBY tile rows per CTA
  if (w < 3 || w > kSmallMaxW || tby < 1 || 32 * tby > kSmallMaxThreads || stages < 2) return false;
  const int tbx = 32;
  const int BW = tbx * w, BH = tby * w;
  if (BW > 256 || BH > 256 || (BW * elem_bytes) % 16 != 0 || BW % 8 != 0) return false;
  size_t stage = (size_t)BW * BH * elem_bytes;
  stage = (stage + 127) / 128 * 128;
  const size_t smem = (size_t)stages * stage + 8 * 8;
  if (smem > 232448 - 1024) return false;
  g->w = w;
  g->R = 0;   // marks the thread-per-tile path
  g->nseg = 1;
  g->TBX = tbx;
  g->TBY = tby;
  g->BW = BW;
  g->BH = BH;
  g->boxW = BW;
  g->aligned = true;
  g->stages = stages;
  g->threads = 32 * tby;
  g->stage_bytes = stage;
  g->smem_bytes = smem;
  return true;
}

// Sub-tile march (w = 8, 16, 32, 64): a CTA covers 128 columns (128 / w tiles)
// and 32 rows (64 for w = 64) with one warp per 4 rows; about 64 KB of ring.
static bool sub_geometry(int w, int elem_bytes, StackGeom* g) {
  if (w != 8 && w != 16 && w != 32 && w != 64) return false;
  const int BH = w <= 32 ? 32 : 64;
  const int nw = BH / 4;
  size_t stage = (size_t)kSubCols * BH * elem_bytes;
  stage = (stage + 127) / 128 * 128;
  const int stages = std::max(3, std::min(8, (int)(65536 / stage)));
  g->w = w;
  g->R = -1;   // marks the sub-tile path
  g->nseg = 1;
  g->TBX = kSubCols / w;
  g->TBY = BH / w;
  g->BW = kSubCols;
  g->BH = BH;
  g->boxW = kSubCols;
  g->aligned = true;
  g->stages = stages;
  g->threads = 32 * nw;
  g->stage_bytes = stage;
  g->smem_bytes = sub_part_offset_host(stages, stage) + (size_t)2 * nw * g->TBX * sizeof(float4);
  return g->smem_bytes <= 232448 - 1024;
}

bool stack_geometry(int w, int elem_bytes, StackGeom* g) {
  if (w < 1 || w > 128) return false;
  if (w >= 3 && w <= kSmallMaxW && small_geometry(w, elem_bytes, 4, 4, g)) return true;
  if (sub_geometry(w, elem_bytes, g)) return true;
  // rows per thread R (a template value) and row segments per tile band
  int R, nseg;
  if (w <= 8) {
    R = w;
    nseg = 1;
  } else if (w <= 32) {
    nseg = (w + 7) / 8;
    R = (w + nseg - 1) / nseg;
  } else if (w <= 64) {
    R = 16;
    nseg = (w + 15) / 16;
  } else {
    R = 32;
    nseg = (w + 31) / 32;
  }
  // Tiles per CTA in x: about 160 pixel columns, preferring an origin that is
  // always a multiple of 8 elements (TMA needs 16-byte aligned x).
  const int max_cols = std::min(160, kStackMaxThreads / nseg);
  if (w > max_cols) return false;
  int tbx = 0;
  for (int t = max_cols / w; t >= 1; --t)
    if ((t * w) % 8 == 0) { tbx = t; break; }
  bool aligned = tbx > 0;
  if (!aligned) tbx = max_cols / w;
  const int BW = tbx * w;
  int tby = 320 / (BW * nseg);
  if (tby < 1) tby = 1;
  if (tby * w > 256) tby = 256 / w;
  if (tby < 1) return false;
  const int threads = BW * tby * nseg;
  if (threads > kStackMaxThreads) return false;
  const int boxW = aligned ? BW : ((BW + 7) / 8) * 8 + 8;
  if (boxW > 256) return false;
  const int BH = tby * w;
  size_t stage = (size_t)boxW * BH * elem_bytes;
  stage = (stage + 127) / 128 * 128;
  const size_t fixed = (size_t)2 * threads * sizeof(float4) + 8 * 8;
  const size_t limit = 232448 - 1024;
  int ns = 4;
  while (ns > 2 && fixed + ns * stage > limit) --ns;
  if (fixed + ns * stage > limit) return false;
  g->w = w;
  g->R = R;
  g->nseg = nseg;
  g->TBX = tbx;
  g->TBY = tby;
  g->BW = BW;
  g->BH = BH;
  g->boxW = boxW;
  g->aligned = aligned;
  g->stages = ns;
  g->threads = threads;
  g->stage_bytes = stage;
  g->smem_bytes = fixed + ns * stage;
  return true;
}

template <typename T, int R, bool SIGNED>
static cudaError_t launch_one(const CUtensorMap* tmap, const StackArgs& a, cudaStream_t st) {
  auto kern = k_stack_tile<T, R, SIGNED>;
  static size_t configured = 0;
  if (a.g.smem_bytes > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)a.g.smem_bytes);
    if (e != cudaSuccess) return e;
    configured = a.g.smem_bytes;
  }
  dim3 grid(a.g.gridX, a.g.gridY);
  kern<<<grid, a.g.threads, a.g.smem_bytes, st>>>(*tmap, a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, int W, bool SIGNED, bool DELTA>
static cudaError_t launch_small(const CUtensorMap* tmap, const StackArgs& a, cudaStream_t st) {
  auto kern = k_stack_small<T, W, SIGNED, DELTA>;
  static size_t configured = 0;
  if (a.g.smem_bytes > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)a.g.smem_bytes);
    if (e != cudaSuccess) return e;
    configured = a.g.smem_bytes;
  }
  dim3 grid(a.g.gridX, a.g.gridY);
  kern<<<grid, a.g.threads, a.g.smem_bytes, st>>>(*tmap, a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, bool SIGNED, bool DELTA>
static cudaError_t launch_sub(const CUtensorMap* tmap, const StackArgs& a, cudaStream_t st) {
  const bool big = a.g.threads > 256;
  auto kern = big ? k_stack_sub<T, SIGNED, 512, DELTA> : k_stack_sub<T, SIGNED, 256, DELTA>;
  static size_t configured[2] = {0, 0};
  if (a.g.smem_bytes > configured[big]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)a.g.smem_bytes);
    if (e != cudaSuccess) return e;
    configured[big] = a.g.smem_bytes;
  }
  dim3 grid(a.g.gridX, a.g.gridY);
  kern<<<grid, a.g.threads, a.g.smem_bytes, st>>>(*tmap, a);
  count_launches(1);
  return cudaGetLastError();
}

// Difference-coded half stacks (a.key set): the thread-per-tile and sub-tile
// marches only.
template <typename T, bool SIGNED>
static cudaError_t launch_delta(const CUtensorMap* tmap, const StackArgs& a, cudaStream_t st) {
  if constexpr (sizeof(T) == 2) {
    if (a.zrot != 0) return cudaErrorInvalidValue;
    if (a.g.R < 0) return launch_sub<T, SIGNED, true>(tmap, a, st);
    if (a.g.R == 0) {
      switch (a.g.w) {
        case 3: return launch_small<T, 3, SIGNED, true>(tmap, a, st);
        case 4: return launch_small<T, 4, SIGNED, true>(tmap, a, st);
        case 5: return launch_small<T, 5, SIGNED, true>(tmap, a, st);
        case 6: return launch_small<T, 6, SIGNED, true>(tmap, a, st);
        default: break;
      }
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T, bool SIGNED>
static cudaError_t launch_r(const CUtensorMap* tmap, const StackArgs& a, cudaStream_t st) {
  if (a.key) return launch_delta<T, SIGNED>(tmap, a, st);
  if (a.g.R < 0) return launch_sub<T, SIGNED, false>(tmap, a, st);
  if (a.g.R == 0) {
    switch (a.g.w) {
      case 3: return launch_small<T, 3, SIGNED, false>(tmap, a, st);
      case 4: return launch_small<T, 4, SIGNED, false>(tmap, a, st);
      case 5: return launch_small<T, 5, SIGNED, false>(tmap, a, st);
      case 6: return launch_small<T, 6, SIGNED, false>(tmap, a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.g.R) {
    case 1: return launch_one<T, 1, SIGNED>(tmap, a, st);
    case 2: return launch_one<T, 2, SIGNED>(tmap, a, st);
    case 3: return launch_one<T, 3, SIGNED>(tmap, a, st);
    case 4: return launch_one<T, 4, SIGNED>(tmap, a, st);
    case 5: return launch_one<T, 5, SIGNED>(tmap, a, st);
    case 6: return launch_one<T, 6, SIGNED>(tmap, a, st);
    case 7: return launch_one<T, 7, SIGNED>(tmap, a, st);
    case 8: return launch_one<T, 8, SIGNED>(tmap, a, st);
    case 16: return launch_one<T, 16, SIGNED>(tmap, a, st);
    case 32: return launch_one<T, 32, SIGNED>(tmap, a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stack(const CUtensorMap* tmap, const StackArgs& a, int storage, int rmode,
                         cudaStream_t st) {
  const bool sg = rmode == FITRIG_RMODE_SIGNED;
  switch (storage) {
    case FITRIG_F32: return sg ? launch_r<float, true>(tmap, a, st) : launch_r<float, false>(tmap, a, st);
    case FITRIG_BF16: return sg ? launch_r<bf16_t, true>(tmap, a, st) : launch_r<bf16_t, false>(tmap, a, st);
    case FITRIG_F16: return sg ? launch_r<f16_t, true>(tmap, a, st) : launch_r<f16_t, false>(tmap, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int W, bool SIGNED>
static cudaError_t launch_multi_t(const FieldDesc* fields, int nfields, int64_t nitems,
                                  unsigned long long* counter, const StackGeom& g, int grid,
                                  uint64_t timeout_ns, cudaStream_t st) {
  auto kern = k_stack_multi<T, W, SIGNED>;
  static size_t configured = 0;
  if (g.smem_bytes > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)g.smem_bytes);
    if (e != cudaSuccess) return e;
    configured = g.smem_bytes;
  }
  kern<<<grid, g.threads, g.smem_bytes, st>>>(fields, nfields, nitems, counter, g, timeout_ns);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, bool SIGNED>
static cudaError_t launch_multi_w(const FieldDesc* fields, int nfields, int64_t nitems,
                                  unsigned long long* counter, const StackGeom& g, int grid,
                                  uint64_t timeout_ns, cudaStream_t st) {
  switch (g.w) {
    case 3: return launch_multi_t<T, 3, SIGNED>(fields, nfields, nitems, counter, g, grid, timeout_ns, st);
    case 4: return launch_multi_t<T, 4, SIGNED>(fields, nfields, nitems, counter, g, grid, timeout_ns, st);
    case 5: return launch_multi_t<T, 5, SIGNED>(fields, nfields, nitems, counter, g, grid, timeout_ns, st);
    case 6: return launch_multi_t<T, 6, SIGNED>(fields, nfields, nitems, counter, g, grid, timeout_ns, st);
    default: return cudaErrorInvalidValue;
  }
}

int multi_blocks_per_sm(const StackGeom& g, int storage, int rmode) {
  int n = 0;
  const void* fn = nullptr;
  const bool sg = rmode == FITRIG_RMODE_SIGNED;
#define FITRIG_PICK(T)                                                                      \
  switch (g.w) {                                                                            \
    case 3: fn = sg ? (const void*)k_stack_multi<T, 3, true> : (const void*)k_stack_multi<T, 3, false>; break; \
    case 4: fn = sg ? (const void*)k_stack_multi<T, 4, true> : (const void*)k_stack_multi<T, 4, false>; break; \
    case 5: fn = sg ? (const void*)k_stack_multi<T, 5, true> : (const void*)k_stack_multi<T, 5, false>; break; \
    case 6: fn = sg ? (const void*)k_stack_multi<T, 6, true> : (const void*)k_stack_multi<T, 6, false>; break; \
  }
  if (storage == FITRIG_F32) { FITRIG_PICK(float) }
  else if (storage == FITRIG_BF16) { FITRIG_PICK(bf16_t) }
  else { FITRIG_PICK(f16_t) }
#undef FITRIG_PICK
  if (!fn) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, g.threads, g.smem_bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_stack_multi(const FieldDesc* fields, int nfields, int64_t nitems,
                               unsigned long long* counter, const StackGeom& g, int grid,
                               int storage, int rmode, uint64_t timeout_ns, cudaStream_t st) {
  const bool sg = rmode == FITRIG_RMODE_SIGNED;
  switch (storage) {
    case FITRIG_F32:
      return sg ? launch_multi_w<float, true>(fields, nfields, nitems, counter, g, grid, timeout_ns, st)
                : launch_multi_w<float, false>(fields, nfields, nitems, counter, g, grid, timeout_ns, st);
    case FITRIG_BF16:
      return sg ? launch_multi_w<bf16_t, true>(fields, nfields, nitems, counter, g, grid, timeout_ns, st)
                : launch_multi_w<bf16_t, false>(fields, nfields, nitems, counter, g, grid, timeout_ns, st);
    case FITRIG_F16:
      return sg ? launch_multi_w<f16_t, true>(fields, nfields, nitems, counter, g, grid, timeout_ns, st)
                : launch_multi_w<f16_t, false>(fields, nfields, nitems, counter, g, grid, timeout_ns, st);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_finite_max(const void* stack, int storage, int L, int ny, int nx,
                              int64_t pitch, unsigned* gmax, cudaStream_t st) {
  const int blocks = 152 * 8, threads = 256;
  switch (storage) {
    case FITRIG_F32:
      k_finite_max<float><<<blocks, threads, 0, st>>>((const float*)stack, L, ny, nx, pitch, gmax);
      break;
    case FITRIG_BF16:
      k_finite_max<bf16_t><<<blocks, threads, 0, st>>>((const bf16_t*)stack, L, ny, nx, pitch, gmax);
      break;
    case FITRIG_F16:
      k_finite_max<f16_t><<<blocks, threads, 0, st>>>((const f16_t*)stack, L, ny, nx, pitch, gmax);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace fitrig
