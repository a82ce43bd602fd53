// Sliding-window mode: the tile statistic of Eq. (tLISI) evaluated over the
// odd w x w window centred on every pixel (clipped at the image border, n_p =
// number of in-image pixels of the window), for every unit s:
//   v(p) = (sum_W Delta / n_p) * max_W Delta * (sum_W r / n_p).
// Delta and r are the per-pixel terms of Eq. 3-5, as in the tile mode.
//
// A CTA owns an OW x OH block of output pixels and marches through time over
// the block plus a halo of h = (w-1)/2 pixels: each snapshot box (with halo,
// x origin rounded down to a multiple of 8 elements for TMA) arrives by a 3-D
// TMA load into a ring of shared-memory stages; each thread carries x^(s+1)
// and D^(s) of its pixels in registers.  Per unit, Delta and r of the extended
// block go to shared memory, a horizontal pass forms the w-wide row sums and
// maxima, and a vertical pass finishes the windows and writes v (windows above
// 9; smaller ones take the shuffle kernel below, which keeps Delta and r in
// registers).  Halo pixels
// outside the image read as zero, which adds nothing to the sums or the
// maximum (Delta >= 0), so only n_p needs the clipping.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "internal.cuh"

namespace fitrig {

constexpr int kSlideMaxThreads = 512;
constexpr int kSlideR = 8;

template <typename T, bool SIGNED>
__global__ void __launch_bounds__(kSlideMaxThreads) k_slide(const __grid_constant__ CUtensorMap tmap,
                                                            const SlideArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SlideGeom& g = a.g;
  const int NS = g.stages;
  float* dS = reinterpret_cast<float*>(smem + (size_t)NS * g.stage_bytes);   // [EH][EW]
  float* rS = dS + g.EH * g.EW;                                              // [EH][EW]
  float* h1 = rS + g.EH * g.EW;                                              // [EH][OW]
  float* h2 = h1 + g.EH * g.OW;
  float* h3 = h2 + g.EH * g.OW;
  uint64_t* bars = reinterpret_cast<uint64_t*>(h3 + g.EH * g.OW);

  const int tid = threadIdx.x;
  const int c = tid % g.EW;
  const int seg = tid / g.EW;
  const int row0 = seg * kSlideR;
  const int rcount = min(kSlideR, g.EH - row0);
  const int x0 = blockIdx.x * g.OW;             // first output column
  const int y0 = blockIdx.y * g.OH;             // first output row
  const int xe = x0 - g.h;                      // first extended column
  const int xload = xe >= 0 ? (xe & ~7) : -(((-xe) + 7) & ~7);
  const int col = (xe - xload) + c;
  const uint32_t bar0 = smem_u32(bars);
  const uint32_t stage0 = smem_u32(smem);
  const uint32_t box_bytes = (uint32_t)(g.boxW * g.EH * (int)sizeof(T));
  const int L = a.nsnap;
  const bool active = tid < g.EW * g.nseg;

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int i = 0; i < NS; ++i) mbar_init(bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < NS && j < L; ++j) {
      mbar_expect_tx(bar0 + 8 * j, box_bytes);
      tma_load_3d(stage0 + j * (uint32_t)g.stage_bytes, &tmap, xload, y0 - g.h, (a.zrot + j) % L,
                  bar0 + 8 * j);
    }
  }
  float xp[kSlideR], dp[kSlideR];
#pragma unroll
  for (int i = 0; i < kSlideR; ++i) xp[i] = dp[i] = 0.f;
  float mx = -INFINITY;
  const uint64_t deadline = globaltimer_ns() + a.timeout_ns;

  for (int j = 0; j < L; ++j) {
    const int stg = j % NS;
    const bool ok = mbar_wait_bounded(bar0 + 8 * stg, (uint32_t)((j / NS) & 1), deadline);
    const T* st = reinterpret_cast<const T*>(smem + (size_t)stg * g.stage_bytes);
    float sm = -INFINITY;   // this snapshot's maximum over the thread's pixels
    if (ok && active) {
#pragma unroll
      for (int i = 0; i < kSlideR; ++i) {
        if (i < rcount) {
          const float xn = to_f32(st[(row0 + i) * g.boxW + col]);
          sm = fmaxf(sm, xn);
          const float dn = fabsf(xn - xp[i]);
          if (j >= 2) {
            const float d = fabsf(dn - dp[i]);
            const float ref = SIGNED ? xp[i] : fabsf(xp[i]);
            const float xh = (xp[i] == 0.f) ? kGuardC : ref;
            dS[(row0 + i) * g.EW + c] = d;
            rS[(row0 + i) * g.EW + c] = fminf(__fdividef(d, xh), 1.f);
          }
          dp[i] = dn;
          xp[i] = xn;
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(a.status, kErrTimeout);
        const uint64_t d2 = globaltimer_ns() + 1000000ull;
        for (int jj = j; jj < L && jj < j + NS; ++jj)
          mbar_wait_bounded(bar0 + 8 * (jj % NS), (uint32_t)((jj / NS) & 1), d2);
      }
      return;
    }
    mx = fmaxf(mx, sm);
    if (a.smax) warp_max_to(sm, a.smax + j);
    if (tid == 0 && j + NS < L) {
      fence_proxy_async_smem();
      mbar_expect_tx(bar0 + 8 * stg, box_bytes);
      tma_load_3d(stage0 + stg * (uint32_t)g.stage_bytes, &tmap, xload, y0 - g.h,
                  (a.zrot + j + NS) % L, bar0 + 8 * stg);
    }
    if (j < 2) continue;
    // horizontal pass: window rows over the extended block
    for (int idx = tid; idx < g.EH * g.OW; idx += blockDim.x) {
      const int row = idx / g.OW, ox = idx - (idx / g.OW) * g.OW;
      const float* dr = dS + row * g.EW + ox;
      const float* rr = rS + row * g.EW + ox;
      float s1 = 0.f, s2 = 0.f, s3 = 0.f;
      for (int k = 0; k < g.w; ++k) {
        s1 += dr[k];
        s2 = fmaxf(s2, dr[k]);
        s3 += rr[k];
      }
      h1[idx] = s1;
      h2[idx] = s2;
      h3[idx] = s3;
    }
    __syncthreads();
    // vertical pass: finish the windows and write v
    for (int idx = tid; idx < g.OH * g.OW; idx += blockDim.x) {
      const int oy = idx / g.OW, ox = idx - (idx / g.OW) * g.OW;
      const int y = y0 + oy, x = x0 + ox;
      if (y >= a.ny || x >= a.nx) continue;
      float S1 = 0.f, S2 = 0.f, S3 = 0.f;
      for (int k = 0; k < g.w; ++k) {
        const int q = (oy + k) * g.OW + ox;
        S1 += h1[q];
        S2 = fmaxf(S2, h2[q]);
        S3 += h3[q];
      }
      const int ny_ = min(y + g.h, a.ny - 1) - max(y - g.h, 0) + 1;
      const int nx_ = min(x + g.h, a.nx - 1) - max(x - g.h, 0) + 1;
      const float n = (float)(ny_ * nx_);
      float v = (S1 / n) * S2 * (S3 / n);
      if (!isfinite(S1) || !isfinite(v)) v = NAN;
      a.vp[(size_t)(j - 2) * (size_t)a.vstride + (size_t)y * a.nx + x] = v;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0 && mx > -INFINITY) atomicMax(a.gmax, f32_key(mx));
}

// ---------------------------------------------------------------- small windows
// Odd windows up to 9 (h <= 4): one thread per column of the extended block,
// 16 output rows per CTA.  Each thread carries x^(s+1) and D^(s) of its
// column's 16 + 2h rows in registers; per unit, each row's Delta and r go
// straight into the horizontal window by warp shuffles (a warp of 32 columns
// yields the 32 - 2h windows that lie inside it; neighbouring warps overlap by
// 2h columns), and the vertical window is summed over the last w rows of
// horizontal results, held in registers as the rows stream past.  No Delta or
// r image is written to shared memory, and the only barrier per snapshot is
// the ring's.
constexpr int kShfRows = 8;     // output rows per CTA
constexpr int kShfWarps = 4;    // warps (column groups) per CTA

// Sum and maximum over lanes l .. l + W - 1 of a warp (binary decomposition:
// windows of 1, 2, 4, 8 lanes by doubling, then the blocks of W's bits).
// Lanes whose window runs past lane 31 get values that are not used.
template <int W>
__device__ __forceinline__ void lane_window(float v, float q, float& s, float& m, float& sq) {
  float s1 = v, m1 = v, q1 = q;
  float s2 = s1 + __shfl_down_sync(0xffffffffu, s1, 1);
  float m2 = fmaxf(m1, __shfl_down_sync(0xffffffffu, m1, 1));
  float q2 = q1 + __shfl_down_sync(0xffffffffu, q1, 1);
  float s4 = 0.f, m4 = 0.f, q4 = 0.f, s8 = 0.f, m8 = 0.f, q8 = 0.f;
  if (W >= 4) {
    s4 = s2 + __shfl_down_sync(0xffffffffu, s2, 2);
    m4 = fmaxf(m2, __shfl_down_sync(0xffffffffu, m2, 2));
    q4 = q2 + __shfl_down_sync(0xffffffffu, q2, 2);
  }
  if (W >= 8) {
    s8 = s4 + __shfl_down_sync(0xffffffffu, s4, 4);
    m8 = fmaxf(m4, __shfl_down_sync(0xffffffffu, m4, 4));
    q8 = q4 + __shfl_down_sync(0xffffffffu, q4, 4);
  }
  // W = 3: 2 + 1; 5: 4 + 1; 7: 4 + 2 + 1; 9: 8 + 1
  if (W == 1) {
    s = s1; m = m1; sq = q1;
  } else if (W == 3) {
    s = s2 + __shfl_down_sync(0xffffffffu, s1, 2);
    m = fmaxf(m2, __shfl_down_sync(0xffffffffu, m1, 2));
    sq = q2 + __shfl_down_sync(0xffffffffu, q1, 2);
  } else if (W == 5) {
    s = s4 + __shfl_down_sync(0xffffffffu, s1, 4);
    m = fmaxf(m4, __shfl_down_sync(0xffffffffu, m1, 4));
    sq = q4 + __shfl_down_sync(0xffffffffu, q1, 4);
  } else if (W == 7) {
    s = s4 + __shfl_down_sync(0xffffffffu, s2, 4);
    m = fmaxf(m4, __shfl_down_sync(0xffffffffu, m2, 4));
    sq = q4 + __shfl_down_sync(0xffffffffu, q2, 4);
    s += __shfl_down_sync(0xffffffffu, s1, 6);
    m = fmaxf(m, __shfl_down_sync(0xffffffffu, m1, 6));
    sq += __shfl_down_sync(0xffffffffu, q1, 6);
  } else {   // W == 9
    s = s8 + __shfl_down_sync(0xffffffffu, s1, 8);
    m = fmaxf(m8, __shfl_down_sync(0xffffffffu, m1, 8));
    sq = q8 + __shfl_down_sync(0xffffffffu, q1, 8);
  }
}

template <typename T, int W, bool SIGNED>
__global__ void __launch_bounds__(kShfWarps * 32, 4) k_slide_shf(const __grid_constant__ CUtensorMap tmap,
                                                                 const SlideArgs a) {
  constexpr int H = W / 2, EH = kShfRows + 2 * H, OWW = 32 - 2 * H;   // OWW outputs per warp
  extern __shared__ __align__(128) unsigned char smem[];
  const SlideGeom& g = a.g;
  const int NS = g.stages;
  const uint32_t stage0 = smem_u32(smem);
  const uint32_t bar0 = smem_u32(smem + (size_t)NS * g.stage_bytes);
  const uint32_t box_bytes = (uint32_t)(g.boxW * EH * (int)sizeof(T));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = blockIdx.x * g.OW, y0 = blockIdx.y * kShfRows;
  const int xe = x0 - H;                        // first extended column
  const int xload = xe >= 0 ? (xe & ~7) : -(((-xe) + 7) & ~7);
  const int col = (xe - xload) + warp * OWW + lane;
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
      tma_load_3d(stage0 + j * (uint32_t)g.stage_bytes, &tmap, xload, y0 - H, (a.zrot + j) % L,
                  bar0 + 8 * j);
    }
  }
  // the output column of this lane (lanes below OWW) and its clipped width
  const int ox = x0 + warp * OWW + lane;
  const bool outcol = lane < OWW && ox < a.nx;
  const int nxw = min(ox + H, a.nx - 1) - max(ox - H, 0) + 1;
  float xp[EH], dp[EH];
#pragma unroll
  for (int i = 0; i < EH; ++i) xp[i] = dp[i] = 0.f;
  float mx = -INFINITY;
  const uint64_t deadline = globaltimer_ns() + a.timeout_ns;

  for (int j = 0; j < L; ++j) {
    const int stg = j % NS;
    // one decision per warp, so that every lane takes part in the shuffles
    const bool ok = __all_sync(0xffffffffu,
                               mbar_wait_bounded(bar0 + 8 * stg, (uint32_t)((j / NS) & 1), deadline));
    const T* st = reinterpret_cast<const T*>(smem + (size_t)stg * g.stage_bytes) + col;
    float sm = -INFINITY;
    if (ok) {
      float rs[W], rm[W], rq[W];   // horizontal windows of the last W rows (a ring)
#pragma unroll
      for (int i = 0; i < EH; ++i) {
        const float xn = to_f32(st[i * g.boxW]);
        sm = fmaxf(sm, xn);
        const float dn = fabsf(xn - xp[i]);   // D^(s+1)
        if (j >= 2) {
          const float d = fabsf(dn - dp[i]);   // Delta
          const float ref = SIGNED ? xp[i] : fabsf(xp[i]);
          const float xh = (xp[i] == 0.f) ? kGuardC : ref;   // Eq. 5
          const float r = fminf(__fdividef(d, xh), 1.f);     // Eq. 4
          lane_window<W>(d, r, rs[i % W], rm[i % W], rq[i % W]);
          if (i >= W - 1) {
            const int oy = i - (W - 1);        // output row, window rows oy .. i
            const int y = y0 + oy;
            float S1 = 0.f, S2 = 0.f, S3 = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
              S1 += rs[(oy + k) % W];
              S2 = fmaxf(S2, rm[(oy + k) % W]);
              S3 += rq[(oy + k) % W];
            }
            if (outcol && y < a.ny) {
              // 1 / n_p^2: a constant inside the image, one division at its
              // border (the tile march's form of the product)
              const int nyw = min(y + H, a.ny - 1) - max(y - H, 0) + 1;
              constexpr float kInvFull = 1.f / (float)(W * W * W * W);
              const float np = (float)(nyw * nxw);
              const float inv = (nyw == W && nxw == W) ? kInvFull : 1.f / (np * np);
              float v = S1 * S2 * S3 * inv;
              if (!isfinite(S1) || !isfinite(v)) v = NAN;
              a.vp[(size_t)(j - 2) * (size_t)a.vstride + (size_t)y * a.nx + ox] = v;
            }
          }
        }
        dp[i] = dn;
        xp[i] = xn;
      }
    }
    if (__syncthreads_or(!ok)) {
      // a stage never completed: flag it, let copies in flight land (bounded)
      if (tid == 0) {
        atomicOr(a.status, kErrTimeout);
        const uint64_t d2 = globaltimer_ns() + 1000000ull;
        for (int jj = j; jj < L && jj < j + NS; ++jj)
          mbar_wait_bounded(bar0 + 8 * (jj % NS), (uint32_t)((jj / NS) & 1), d2);
      }
      return;
    }
    mx = fmaxf(mx, sm);
    if (a.smax) warp_max_to(sm, a.smax + j);
    if (tid == 0 && j + NS < L) {
      fence_proxy_async_smem();
      mbar_expect_tx(bar0 + 8 * stg, box_bytes);
      tma_load_3d(stage0 + stg * (uint32_t)g.stage_bytes, &tmap, xload, y0 - H,
                  (a.zrot + j + NS) % L, bar0 + 8 * stg);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > -INFINITY) atomicMax(a.gmax, f32_key(mx));
}

bool slide_geometry(int w, int elem_bytes, SlideGeom* g) {
  if (w < 1 || (w & 1) == 0 || w > 31) return false;
  const int h = w / 2;
  if (w >= 3 && w <= 9) {   // the shuffle kernel (nseg = 0 marks it)
    const int OW = kShfWarps * (32 - 2 * h);
    const int EW = OW + 2 * h, EH = kShfRows + 2 * h;
    const int boxW = (EW + 7 + 7) / 8 * 8;
    size_t stage = (size_t)boxW * EH * elem_bytes;
    stage = (stage + 127) / 128 * 128;
    const int ns = 4;
    g->w = w;
    g->h = h;
    g->OW = OW;
    g->OH = kShfRows;
    g->EW = EW;
    g->EH = EH;
    g->nseg = 0;
    g->boxW = boxW;
    g->threads = kShfWarps * 32;
    g->stages = ns;
    g->stage_bytes = stage;
    g->smem_bytes = ns * stage + 8 * ns;
    return boxW <= 256;
  }
  int OW = 128, OH = 16, EW, EH, nseg, threads;
  for (;;) {
    EW = OW + 2 * h;
    EH = OH + 2 * h;
    nseg = (EH + kSlideR - 1) / kSlideR;
    threads = EW * nseg;
    if (threads <= kSlideMaxThreads) break;
    if (OH > 4) OH /= 2;
    else if (OW > 32) OW /= 2;
    else return false;
  }
  const int boxW = ((OW + 2 * h + 7) + 7) / 8 * 8;
  if (boxW > 256 || EH > 256) return false;
  size_t stage = (size_t)boxW * EH * elem_bytes;
  stage = (stage + 127) / 128 * 128;
  const size_t fixed = (size_t)(2 * EH * EW + 3 * EH * OW) * sizeof(float) + 8 * 8;
  const size_t limit = 232448 - 1024;
  int ns = 4;
  while (ns > 2 && fixed + ns * stage > limit) --ns;
  if (fixed + ns * stage > limit) return false;
  g->w = w;
  g->h = h;
  g->OW = OW;
  g->OH = OH;
  g->EW = EW;
  g->EH = EH;
  g->nseg = nseg;
  g->boxW = boxW;
  g->threads = ((threads + 31) / 32) * 32;
  g->stages = ns;
  g->stage_bytes = stage;
  g->smem_bytes = fixed + ns * stage;
  return true;
}

template <typename T, int W, bool SIGNED>
static cudaError_t launch_shf_t(const CUtensorMap* tmap, const SlideArgs& a, cudaStream_t st) {
  auto kern = k_slide_shf<T, W, SIGNED>;
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

template <typename T, bool SIGNED>
static cudaError_t launch_slide_t(const CUtensorMap* tmap, const SlideArgs& a, cudaStream_t st) {
  if (a.g.nseg == 0) {
    switch (a.g.w) {
      case 3: return launch_shf_t<T, 3, SIGNED>(tmap, a, st);
      case 5: return launch_shf_t<T, 5, SIGNED>(tmap, a, st);
      case 7: return launch_shf_t<T, 7, SIGNED>(tmap, a, st);
      case 9: return launch_shf_t<T, 9, SIGNED>(tmap, a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  auto kern = k_slide<T, SIGNED>;
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

cudaError_t launch_slide(const CUtensorMap* tmap, const SlideArgs& a, int storage, int rmode,
                         cudaStream_t st) {
  const bool sg = rmode == FITRIG_RMODE_SIGNED;
  switch (storage) {
    case FITRIG_F32: return sg ? launch_slide_t<float, true>(tmap, a, st) : launch_slide_t<float, false>(tmap, a, st);
    case FITRIG_BF16: return sg ? launch_slide_t<bf16_t, true>(tmap, a, st) : launch_slide_t<bf16_t, false>(tmap, a, st);
    case FITRIG_F16: return sg ? launch_slide_t<f16_t, true>(tmap, a, st) : launch_slide_t<f16_t, false>(tmap, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fitrig
