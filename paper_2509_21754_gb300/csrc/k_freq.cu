// Image-frequency branch (Sec. 2.4.2): per tile, the series of the tile
// statistic over the n = L - 2 units, its mean removed (the DC term of Eq.
// eta), an unnormalised DFT of exact length n, and
//   eta_t = max_{k=1..floor(n/2)} |X_k|   (h = maximum spectral magnitude)
// with the arg-max bin (smallest k on ties), or, with hmax > 1, h = the
// incoherent harmonic sum
//   eta_t = max_{m = 1, 2, 4, .., hmax} max_{k: m k <= floor(n/2)}
//           (|X_k| + |X_2k| + .. + |X_mk|) / sqrt(m)
// with the fundamental k (ties: smaller m, then smaller k).  Sec. 2.4.2 names
// harmonic summing as a choice of h without a formula; this is the classic
// incoherent form.
//
// The series used is v_t(s) = mean(Delta) max(Delta) mean(r), i.e. the tLISI
// complement times M^2 with one M for the stack, so |X_k| of tLISI is |X_k|/M^2
// and the z-score of eta is unchanged.
//
// One thread per tile; the series is staged in shared memory (coalesced over
// tiles).  Real input: pairs y_s, y_{n-s} are folded into e_s = y_s + y_{n-s}
// and o_s = y_s - y_{n-s}, so that Re X_k = y_0 + sum e_s cos + [n even]
// (-1)^k y_{n/2} and Im X_k = -sum o_s sin, halving the multiply-adds.  The
// twiddles cos/sin(2 pi k s / n) come from a table filled on the host in FP64.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace fitrig {

constexpr int kDftThreads = 128;

// The harmonic sum over one tile's magnitudes |X_k| = mag[(k - 1) * stride],
// k = 1..K, in the order (m ascending, k ascending) so that ties keep the
// smaller m, then the smaller k.
__device__ __forceinline__ void harmonic_best(const float* mag, int stride, int K, int hmax,
                                              float& best, int& bk) {
  best = -1.f;
  bk = 1;
  for (int m = 1; m <= hmax && m <= K; m <<= 1) {
    const float inv = 1.f / sqrtf((float)m);
    for (int k = 1; k * m <= K; ++k) {
      float acc = 0.f;
      for (int j = 1; j <= m; ++j) acc += mag[(j * k - 1) * stride];
      acc *= inv;
      if (acc > best) {
        best = acc;
        bk = k;
      }
    }
  }
}

__global__ void __launch_bounds__(kDftThreads) k_dft(const float* __restrict__ vp, int n,
                                                     int64_t T, int64_t vs,
                                                     const float2* __restrict__ tw,
                                                     const float* __restrict__ wts,
                                                     float* eta, int* bin) {
  extern __shared__ float ys[];   // [n][kDftThreads]
  const int tid = threadIdx.x;
  const int64_t t = (int64_t)blockIdx.x * kDftThreads + tid;
  const bool live = t < T;
  bool ok = live;
  float s = 0.f, comp = 0.f;
  for (int q = 0; q < n; ++q) {
    const float v = live ? (wts ? vp[(size_t)q * vs + t] * wts[q] : vp[(size_t)q * vs + t]) : 0.f;
    ok = ok && isfinite(v);
    ys[q * kDftThreads + tid] = v;
    const float y = v - comp;
    const float u = s + y;
    comp = (u - s) - y;
    s = u;
  }
  if (!live) return;
  if (!ok) {
    eta[t] = NAN;
    bin[t] = -1;
    return;
  }
  const float mean = s / (float)n;
  const int H = (n - 1) / 2;        // folded pairs s = 1..H
  const bool even = (n & 1) == 0;
  const float y0 = ys[tid] - mean;
  const float ymid = even ? ys[(n / 2) * kDftThreads + tid] - mean : 0.f;
  for (int q = 1; q <= H; ++q) {
    const float a = ys[q * kDftThreads + tid] - mean;
    const float b = ys[(n - q) * kDftThreads + tid] - mean;
    ys[q * kDftThreads + tid] = a + b;         // e_q
    ys[(n - q) * kDftThreads + tid] = a - b;   // o_q
  }
  const int K = n / 2;
  float best = -1.f;
  int bk = 1;
  for (int k = 1; k <= K; ++k) {
    float re = y0 + ((even && (k & 1)) ? -ymid : ymid);
    float im = 0.f;
    const float2* twk = tw + (size_t)(k - 1) * H;
    for (int q = 1; q <= H; ++q) {
      const float2 cs = twk[q - 1];
      re = fmaf(ys[q * kDftThreads + tid], cs.x, re);
      im = fmaf(ys[(n - q) * kDftThreads + tid], cs.y, im);
    }
    const float m2 = re * re + im * im;
    if (m2 > best) {
      best = m2;
      bk = k;
    }
  }
  eta[t] = sqrtf(best);
  bin[t] = bk;
}

// Short series (n <= 2*KMAX + 1): the pair loop runs outermost and the
// accumulators of every bin stay in registers; each twiddle is a shared-memory
// broadcast, so one load feeds two multiply-adds.
template <int KMAX, bool HARM>
__global__ void __launch_bounds__(kDftThreads) k_dft_short(const float* __restrict__ vp, int n,
                                                           int64_t T, int64_t vs,
                                                           const float2* __restrict__ tw,
                                                           const float* __restrict__ wts,
                                                           int hmax, float* eta, int* bin) {
  extern __shared__ float2 tws[];   // [H][K] twiddles, pair-major, then [n][threads] series
  const int H = (n - 1) / 2, K = n / 2;
  float* ys = reinterpret_cast<float*>(tws + H * K);
  for (int i = threadIdx.x; i < H * K; i += blockDim.x) {
    const int q = i / K, k = i - (i / K) * K;
    tws[i] = tw[(size_t)k * H + q];
  }
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * kDftThreads + threadIdx.x;
  if (t >= T) return;
  float s = 0.f, comp = 0.f;
  bool ok = true;
  float* my = ys + threadIdx.x;
  for (int q = 0; q < n; ++q) {
    const float v = wts ? vp[(size_t)q * vs + t] * wts[q] : vp[(size_t)q * vs + t];
    ok = ok && isfinite(v);
    my[q * kDftThreads] = v;
    const float y = v - comp;
    const float u = s + y;
    comp = (u - s) - y;
    s = u;
  }
  if (!ok) {
    eta[t] = NAN;
    bin[t] = -1;
    return;
  }
  const float mean = s / (float)n;
  const bool even = (n & 1) == 0;
  const float y0 = my[0] - mean;
  const float ymid = even ? my[(n / 2) * kDftThreads] - mean : 0.f;
  float re[KMAX], im[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    re[k] = y0 + ((even && ((k + 1) & 1)) ? -ymid : ymid);
    im[k] = 0.f;
  }
  for (int q = 1; q <= H; ++q) {
    const float a = my[q * kDftThreads] - mean;
    const float b = my[(n - q) * kDftThreads] - mean;
    const float e = a + b, o = a - b;
    const float2* row = tws + (q - 1) * K;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      if (k < K) {
        const float2 cs = row[k];
        re[k] = fmaf(e, cs.x, re[k]);
        im[k] = fmaf(o, cs.y, im[k]);
      }
    }
  }
  float best = -1.f;
  int bk = 1;
  if constexpr (HARM) {
    // the series is spent: its column holds the magnitudes for the harmonic sum
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      if (k < K) my[k * kDftThreads] = sqrtf(re[k] * re[k] + im[k] * im[k]);
    harmonic_best(my, kDftThreads, K, hmax, best, bk);
    eta[t] = best;
    bin[t] = bk;
  } else {
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      if (k < K) {
        const float m2 = re[k] * re[k] + im[k] * im[k];
        if (m2 > best) {
          best = m2;
          bk = k + 1;
        }
      }
    }
    eta[t] = sqrtf(best);
    bin[t] = bk;
  }
}

// Even n = 2m (n <= 66): the transform splits into the two length-m DFTs of
// the even- and odd-indexed samples, X_k = E_k + W^k O_k with W = e^(-2 pi i/n)
// (a radix-2 decimation in time).  E and O are DFTs of real series, so only
// their bins k = 0..floor(m/2) are formed (the others are complex conjugates,
// E_(m-k) = conj(E_k)), each from folded pairs of samples; one shared-memory
// twiddle then feeds four multiply-adds (both halves, real and imaginary
// parts), half the work of the direct form.  X_m = E_0 - O_0 (Nyquist).
// Twiddles come from the host's FP64 table of 2 pi q / n (its first row) by
// symmetry.
template <int KH, bool HARM>
__global__ void __launch_bounds__(kDftThreads) k_dft_even(const float* __restrict__ vp, int n,
                                                          int64_t T, int64_t vs,
                                                          const float2* __restrict__ tw,
                                                          const float* __restrict__ wts,
                                                          int hmax, float* eta, int* bin) {
  extern __shared__ float2 sm2[];
  const int m = n / 2, Hm = (m - 1) / 2, K = m / 2, H = (n - 1) / 2;
  float2* th = sm2;                                 // [Hm][K]: 2 pi j k / m, j,k >= 1
  float2* tk = th + (Hm > 0 ? Hm * K : 0);          // [m]: 2 pi k / n
  float* ys = reinterpret_cast<float*>(tk + m);     // [n][kDftThreads]
  // (cos, sin) of 2 pi a / n from the table row q = 1..H and symmetry
  auto ang = [&](int a) -> float2 {
    if (a == 0) return make_float2(1.f, 0.f);
    if (2 * a == n) return make_float2(-1.f, 0.f);
    if (a <= H) return tw[a - 1];
    const float2 c = tw[n - a - 1];
    return make_float2(c.x, -c.y);
  };
  for (int i = threadIdx.x; i < Hm * K; i += blockDim.x) {
    const int j = i / K + 1, k = i - (i / K) * K + 1;
    th[i] = ang((2 * j * k) % n);
  }
  for (int k = threadIdx.x; k < m; k += blockDim.x) tk[k] = ang(k);
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * kDftThreads + threadIdx.x;
  if (t >= T) return;
  float* my = ys + threadIdx.x;
  // the series arrives by asynchronous global -> shared copies, all n of a
  // thread in flight at once (coalesced over the CTA's tiles)
  for (int q = 0; q < n; ++q) {
    const uint32_t dst = smem_u32(my + q * kDftThreads);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst),
                 "l"(vp + (size_t)q * vs + t)
                 : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  float sum = 0.f;
  bool ok = true;
  for (int q = 0; q < n; ++q) {
    float v = my[q * kDftThreads];
    if (wts) {
      v *= wts[q];
      my[q * kDftThreads] = v;
    }
    ok = ok && isfinite(v);
    sum += v;
  }
  if (!ok) {
    eta[t] = NAN;
    bin[t] = -1;
    return;
  }
  const float mean = sum / (float)n;
  auto ye = [&](int j) { return my[(2 * j) * kDftThreads] - mean; };       // y_(2j)
  auto yo = [&](int j) { return my[(2 * j + 1) * kDftThreads] - mean; };   // y_(2j+1)
  const float ye0 = ye(0), yo0 = yo(0);
  const bool meven = (m & 1) == 0;
  const float yem = meven ? ye(m / 2) : 0.f, yom = meven ? yo(m / 2) : 0.f;
  float E0 = ye0 + yem, O0 = yo0 + yom;   // bin 0 of each half
  float er[KH], es[KH], orr[KH], os[KH];  // bins 1..K: real parts, and the sums of
                                          // the odd folds times sin (imag = -that)
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    const float sg = ((k + 1) & 1) ? -1.f : 1.f;   // (-1)^(k+1)
    er[k] = ye0 + sg * yem;
    orr[k] = yo0 + sg * yom;
    es[k] = 0.f;
    os[k] = 0.f;
  }
  for (int j = 1; j <= Hm; ++j) {
    const float a = ye(j), b = ye(m - j), c = yo(j), d = yo(m - j);
    const float ee = a + b, eo = a - b, oe = c + d, oo = c - d;
    E0 += ee;
    O0 += oe;
    const float2* row = th + (j - 1) * K;
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      if (k < K) {
        const float2 w = row[k];
        er[k] = fmaf(ee, w.x, er[k]);
        es[k] = fmaf(eo, w.y, es[k]);
        orr[k] = fmaf(oe, w.x, orr[k]);
        os[k] = fmaf(oo, w.y, os[k]);
      }
    }
  }
  // X_k = E_k + W^k O_k, W^k = (c, -s):  Re = Er + c Or + s Oi,  Im = Ei + c Oi - s Or
  float best = -1.f;
  int bk = 1;
  // with harmonic summing the spent series column collects |X_k| at row k - 1
  constexpr bool harm = HARM;
  auto take = [&](int k, float Er, float Ei, float Or, float Oi) {
    const float2 w = tk[k];
    const float re = Er + w.x * Or + w.y * Oi;
    const float im = Ei + w.x * Oi - w.y * Or;
    const float m2 = re * re + im * im;
    if constexpr (harm) my[(k - 1) * kDftThreads] = sqrtf(m2);
    if (m2 > best || (m2 == best && k < bk)) {
      best = m2;
      bk = k;
    }
  };
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    if (k < K) {
      take(k + 1, er[k], -es[k], orr[k], -os[k]);                    // bin k+1
      if (m - (k + 1) > K) take(m - (k + 1), er[k], es[k], orr[k], os[k]);   // its mirror
    }
  }
  {
    const float x = E0 - O0;   // bin m
    const float m2 = x * x;
    if constexpr (HARM) my[(m - 1) * kDftThreads] = fabsf(x);
    if (m2 > best || (m2 == best && m < bk)) {
      best = m2;
      bk = m;
    }
  }
  if constexpr (HARM) {
    harmonic_best(my, kDftThreads, m, hmax, best, bk);
    eta[t] = best;
    bin[t] = bk;
  } else {
    eta[t] = sqrtf(best);
    bin[t] = bk;
  }
}

// Long series (n up to kLongMaxN) and harmonic sums beyond the short kernels:
// one warp per tile, a CTA stages the series of kLongWarps consecutive tiles
// (each cube row a 32-byte segment) and transposes them into shared memory.
// Lane l forms bins k = l + 1 + 32 j, kLongB at a time, over the folded pairs
// (e_q, o_q) read as broadcasts; the phasor (cos, sin)(2 pi k q / n) advances by
// one complex multiply per step and is re-seeded from the host's FP64 table
// every kSeed steps, so its rounding error stays that of a few dozen
// multiplies.  The magnitudes go to shared memory for the maximum or the
// harmonic sum, which the warp then reduces.
constexpr int kLongWarps = 8;
constexpr int kLongMaxN = 4096;
constexpr int kLongB = 4;
constexpr int kSeed = 32;

// Warp reduction of one tile's squared magnitudes mk[k] = |X_k|^2, k = 1..K:
// the maximum magnitude (hmax = 1) or the largest harmonic sum, with its bin
// (ties: smaller m, then smaller k).  Lane 0 writes eta and the bin.
__device__ __forceinline__ void warp_spectrum_best(const float* mk, int K, int hmax, int lane,
                                                   float* eta, int* bin) {
  float best = -1.f;
  int bk = 1, bm = 1;
  if (hmax <= 1) {
    for (int k = 1 + lane; k <= K; k += 32) {
      const float v = mk[k];
      if (v > best) {
        best = v;
        bk = k;
      }
    }
  } else {
    for (int m = 1; m <= hmax && m <= K; m <<= 1) {
      const float inv = 1.f / sqrtf((float)m);
      for (int k = 1 + lane; k * m <= K; k += 32) {
        float acc = 0.f;
        for (int j = 1; j <= m; ++j) acc += sqrtf(mk[j * k]);
        acc *= inv;
        if (acc > best) {
          best = acc;
          bk = k;
          bm = m;
        }
      }
    }
  }
  // warp arg-max: larger value, then smaller m, then smaller k
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, off);
    const int okk = __shfl_xor_sync(0xffffffffu, bk, off);
    const int om = __shfl_xor_sync(0xffffffffu, bm, off);
    if (ov > best || (ov == best && (om < bm || (om == bm && okk < bk)))) {
      best = ov;
      bk = okk;
      bm = om;
    }
  }
  if (lane == 0) {
    *eta = hmax <= 1 ? sqrtf(best) : best;
    *bin = bk;
  }
}

__host__ __device__ constexpr int long_ldy(int n) { return (n + 27) / 32 * 32 + 4; }

__global__ void __launch_bounds__(kLongWarps * 32) k_dft_long(const float* __restrict__ vp, int n,
                                                              int64_t T, int64_t vs,
                                                              const float2* __restrict__ tw,
                                                              const float* __restrict__ wts,
                                                              int hmax, float* eta, int* bin) {
  extern __shared__ float lsm[];
  const int K = n / 2, H = (n - 1) / 2, ldy = long_ldy(n);
  float* ys = lsm;                                 // [kLongWarps][ldy]
  float* mg = lsm + kLongWarps * ldy;              // [kLongWarps][K + 1]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t0 = (int64_t)blockIdx.x * kLongWarps;
  for (int i = threadIdx.x; i < n * kLongWarps; i += blockDim.x) {
    const int q = i / kLongWarps, c = i - q * kLongWarps;
    const int64_t t = t0 + c;
    float v = t < T ? vp[(size_t)q * vs + t] : 0.f;
    if (wts) v *= wts[q];
    ys[c * ldy + q] = v;
  }
  __syncthreads();
  const int64_t t = t0 + warp;
  if (t >= T) return;
  float* y = ys + warp * ldy;
  float sum = 0.f;
  bool ok = true;
  for (int q = lane; q < n; q += 32) {
    const float v = y[q];
    ok = ok && isfinite(v);
    sum += v;
  }
  ok = __all_sync(0xffffffffu, ok);
#pragma unroll
  for (int off = 16; off; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if (!ok) {
    if (lane == 0) {
      eta[t] = NAN;
      bin[t] = -1;
    }
    return;
  }
  const float mean = sum / (float)n;
  __syncwarp();
  for (int q = 1 + lane; q <= H; q += 32) {
    const float a = y[q] - mean, b = y[n - q] - mean;
    y[q] = a + b;       // e_q
    y[n - q] = a - b;   // o_q
  }
  __syncwarp();
  const bool even = (n & 1) == 0;
  const float y0 = y[0] - mean;
  const float ymid = even ? y[n / 2] - mean : 0.f;
  // (cos, sin) of 2 pi a / n, 0 <= a < n, from the table's first row and symmetry
  auto ang = [&](int a) -> float2 {
    if (a == 0) return make_float2(1.f, 0.f);
    if (2 * a == n) return make_float2(-1.f, 0.f);
    if (a <= H) return tw[a - 1];
    const float2 c = tw[n - a - 1];
    return make_float2(c.x, -c.y);
  };
  float* mk = mg + warp * (K + 1);   // |X_k|^2 at mk[k]
  for (int kb = 1; kb <= K; kb += 32 * kLongB) {
    int kk[kLongB];
    float re[kLongB], im[kLongB], c[kLongB], sn[kLongB], wc[kLongB], ws[kLongB];
#pragma unroll
    for (int b = 0; b < kLongB; ++b) {
      kk[b] = min(kb + lane + 32 * b, K);
      re[b] = y0 + ((even && (kk[b] & 1)) ? -ymid : ymid);
      im[b] = 0.f;
      const float2 w = ang(kk[b]);
      wc[b] = w.x;
      ws[b] = w.y;
    }
    for (int q0 = 1; q0 <= H; q0 += kSeed) {
#pragma unroll
      for (int b = 0; b < kLongB; ++b) {
        const float2 e = ang((int)(((int64_t)kk[b] * q0) % n));
        c[b] = e.x;
        sn[b] = e.y;
      }
      const int qe = min(H, q0 + kSeed - 1);
      for (int q = q0; q <= qe; ++q) {
        const float e = y[q], o = y[n - q];
#pragma unroll
        for (int b = 0; b < kLongB; ++b) {
          re[b] = fmaf(e, c[b], re[b]);
          im[b] = fmaf(o, sn[b], im[b]);
          const float cn = fmaf(c[b], wc[b], -sn[b] * ws[b]);
          sn[b] = fmaf(sn[b], wc[b], c[b] * ws[b]);
          c[b] = cn;
        }
      }
    }
#pragma unroll
    for (int b = 0; b < kLongB; ++b)
      if (kb + lane + 32 * b <= K) mk[kk[b]] = re[b] * re[b] + im[b] * im[b];
  }
  __syncwarp();
  warp_spectrum_best(mk, K, hmax, lane, eta + t, bin + t);
}

// Powers of two, kFftMinN <= n <= kLongMaxN: a radix FFT per tile instead of
// the O(n^2) direct sum.  One warp per tile; a CTA stages the series of
// TILES consecutive tiles by asynchronous global -> shared copies (each cube
// row a TILES x 4-byte segment).  The real series y_0..y_(n-1), mean removed,
// is read as the complex series z_j = y_(2j) + i y_(2j+1) of N = n/2 points
// (the staging buffer already holds it in that order), transformed by a
// Stockham autosort FFT (radix-4 passes, one radix-2 pass when log2 N is odd)
// that alternates between the staging buffer and a second warp buffer, and
// the real spectrum is recovered as
//   X_k = (Z_k + conj Z_(N-k)) / 2 - (i/2) e^(-2 pi i k/n) (Z_k - conj Z_(N-k)),
//   X_(n/2) = Re Z_0 - Im Z_0,
// whose squared magnitudes feed the same maximum / harmonic-sum reduction as
// the direct kernels.  Every twiddle is an entry of the host's FP64 table of
// (cos, sin)(2 pi a / n), a = 0..n-1, rounded once to FP32.
constexpr int kFftMinN = 128;

__host__ __device__ constexpr bool fft_length(int n) {
  return n >= kFftMinN && n <= kLongMaxN && (n & (n - 1)) == 0;
}

__device__ __forceinline__ float2 cmul_conj(float2 a, float2 w) {   // a * conj(w)
  return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}

template <int TILES>
__global__ void __launch_bounds__(TILES * 32) k_fft_pow2(const float* __restrict__ vp, int n,
                                                         int logN, int64_t T, int64_t vs,
                                                         const float2* __restrict__ fw,
                                                         const float* __restrict__ wts, int hmax,
                                                         float* eta, int* bin) {
  extern __shared__ float2 fsm[];
  const int N = n >> 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t0 = (int64_t)blockIdx.x * TILES;
  for (int i = threadIdx.x; i < n * TILES; i += TILES * 32) {
    const int q = i / TILES, c = i - q * TILES;
    float* dst = reinterpret_cast<float*>(fsm + (size_t)c * 2 * N) + q;
    if (t0 + c < T) {
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)),
                   "l"(vp + (size_t)q * vs + t0 + c)
                   : "memory");
    } else {
      *dst = 0.f;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int64_t t = t0 + warp;
  if (t >= T) return;
  float2* src = fsm + (size_t)warp * 2 * N;   // z_j = (y_2j, y_2j+1)
  float2* dst = src + N;
  float* y = reinterpret_cast<float*>(src);
  float sum = 0.f;
  bool ok = true;
  for (int q = lane; q < n; q += 32) {
    float v = y[q];
    if (wts) {
      v *= wts[q];
      y[q] = v;
    }
    ok = ok && isfinite(v);
    sum += v;
  }
  ok = __all_sync(0xffffffffu, ok);
#pragma unroll
  for (int off = 16; off; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if (!ok) {
    if (lane == 0) {
      eta[t] = NAN;
      bin[t] = -1;
    }
    return;
  }
  const float mean = sum / (float)n;
  for (int q = lane; q < n; q += 32) y[q] -= mean;
  __syncwarp();
  int Ns = 1;
  for (int pass = 0; pass < (logN >> 1); ++pass) {
    const int Q = N >> 2, step = n / (4 * Ns);
    for (int j = lane; j < Q; j += 32) {
      const int k = j & (Ns - 1);
      const int e = k * step;   // W_(4 Ns)^(r k) = W_n^(r e), r e < 3n/4
      const float2 a0 = src[j];
      const float2 a1 = cmul_conj(src[j + Q], __ldg(fw + e));
      const float2 a2 = cmul_conj(src[j + 2 * Q], __ldg(fw + 2 * e));
      const float2 a3 = cmul_conj(src[j + 3 * Q], __ldg(fw + 3 * e));
      const float2 b0 = make_float2(a0.x + a2.x, a0.y + a2.y);
      const float2 b1 = make_float2(a0.x - a2.x, a0.y - a2.y);
      const float2 b2 = make_float2(a1.x + a3.x, a1.y + a3.y);
      const float2 b3 = make_float2(a1.y - a3.y, a3.x - a1.x);   // -i (a1 - a3)
      const int base = ((j - k) << 2) + k;
      dst[base] = make_float2(b0.x + b2.x, b0.y + b2.y);
      dst[base + Ns] = make_float2(b1.x + b3.x, b1.y + b3.y);
      dst[base + 2 * Ns] = make_float2(b0.x - b2.x, b0.y - b2.y);
      dst[base + 3 * Ns] = make_float2(b1.x - b3.x, b1.y - b3.y);
    }
    __syncwarp();
    float2* tmp = src;
    src = dst;
    dst = tmp;
    Ns <<= 2;
  }
  if (logN & 1) {   // last pass radix 2: Ns = N / 2, twiddle W_N^j = W_n^(2j)
    for (int j = lane; j < Ns; j += 32) {
      const float2 a0 = src[j];
      const float2 a1 = cmul_conj(src[j + Ns], __ldg(fw + 2 * j));
      dst[j] = make_float2(a0.x + a1.x, a0.y + a1.y);
      dst[j + Ns] = make_float2(a0.x - a1.x, a0.y - a1.y);
    }
    __syncwarp();
    float2* tmp = src;
    src = dst;
    dst = tmp;
  }
  float* mk = reinterpret_cast<float*>(dst);   // |X_k|^2 at mk[k], k = 1..N
  for (int k = 1 + lane; k <= N; k += 32) {
    float m2;
    if (k == N) {
      const float2 z0 = src[0];
      const float x = z0.x - z0.y;
      m2 = x * x;
    } else {
      const float2 zk = src[k], zc = src[N - k];
      const float er = 0.5f * (zk.x + zc.x), ei = 0.5f * (zk.y - zc.y);
      const float orr = 0.5f * (zk.y + zc.y), oi = 0.5f * (zc.x - zk.x);
      const float2 w = __ldg(fw + k);   // (cos, sin)(2 pi k / n); forward uses conj
      const float xr = er + fmaf(w.x, orr, w.y * oi);
      const float xi = ei + fmaf(w.x, oi, -w.y * orr);
      m2 = xr * xr + xi * xi;
    }
    mk[k] = m2;
  }
  __syncwarp();
  warp_spectrum_best(mk, N, hmax, lane, eta + t, bin + t);
}

static int fft_tiles(int n) { return n <= 1024 ? 8 : 4; }

std::vector<float2> spectrum_twiddles(int n) {
  std::vector<float2> tw;
  if (fft_length(n)) {   // the full circle: (cos, sin)(2 pi a / n), a = 0..n-1
    tw.resize((size_t)n);
    for (int a = 0; a < n; ++a) {
      const double ang = 2.0 * M_PI * (double)a / (double)n;
      tw[(size_t)a] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    return tw;
  }
  // (cos, sin)(2 pi ((k q) mod n) / n) for k = 1..K, q = 1..H: [K][H] for the
  // direct kernels of series up to 256 points; longer series take only the
  // first row (k = 1), which is all the warp-per-tile kernel reads.
  const int H = (n - 1) / 2, K = n > 256 ? 1 : n / 2;
  tw.resize((size_t)std::max(1, K * H));
  for (int k = 1; k <= K; ++k)
    for (int q = 1; q <= H; ++q) {
      const double ang = 2.0 * M_PI * (double)(((int64_t)k * q) % n) / (double)n;
      tw[(size_t)(k - 1) * H + (q - 1)] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  return tw;
}

int spectrum_max_n() { return kLongMaxN; }

static cudaError_t launch_long(const float* vp, int n, int64_t T, int64_t vs,
                               const float2* tw_row, const float* wts, int hmax, float* eta,
                               int* bin, cudaStream_t st) {
  const int K = n / 2;
  const size_t sm = (size_t)kLongWarps * (long_ldy(n) + K + 1) * sizeof(float);
  static size_t long_configured = 0;
  if (sm > 48 * 1024 && sm > long_configured) {
    cudaError_t e = cudaFuncSetAttribute(k_dft_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    long_configured = sm;
  }
  const int64_t lblocks = (T + kLongWarps - 1) / kLongWarps;
  k_dft_long<<<(unsigned)lblocks, kLongWarps * 32, sm, st>>>(vp, n, T, vs, tw_row, wts, hmax,
                                                             eta, bin);
  count_launches(1);
  return cudaGetLastError();
}

template <int TILES>
static cudaError_t launch_fft_t(const float* vp, int n, int64_t T, int64_t vs, const float2* fw,
                                const float* wts, int hmax, float* eta, int* bin,
                                cudaStream_t st) {
  const size_t sm = (size_t)TILES * n * sizeof(float2);   // two N-point buffers per tile
  static size_t configured = 0;
  if (sm > 48 * 1024 && sm > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_pow2<TILES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    configured = sm;
  }
  int logN = 0;
  while ((2 << logN) < n) ++logN;   // N = n / 2 = 2^logN
  const int64_t blocks = (T + TILES - 1) / TILES;
  k_fft_pow2<TILES><<<(unsigned)blocks, TILES * 32, sm, st>>>(vp, n, logN, T, vs, fw, wts, hmax,
                                                             eta, bin);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_spectrum_method(const float* vp, int n, int64_t T, int64_t vs,
                                   const float2* twiddle, const float* wts, int hmax, float* eta,
                                   int* bin, int method, cudaStream_t st) {
  if (n < 2 || n > kLongMaxN || hmax < 1) return cudaErrorInvalidValue;
  if (T == 0) return cudaSuccess;
  if (fft_length(n)) {
    if (method == kSpectrumDirect)   // the O(n^2) warp kernel on the same table
      return launch_long(vp, n, T, vs, twiddle + 1, wts, hmax, eta, bin, st);
    return fft_tiles(n) == 8 ? launch_fft_t<8>(vp, n, T, vs, twiddle, wts, hmax, eta, bin, st)
                             : launch_fft_t<4>(vp, n, T, vs, twiddle, wts, hmax, eta, bin, st);
  }
  if (method == kSpectrumRadix) return cudaErrorInvalidValue;
  return launch_spectrum(vp, n, T, vs, twiddle, wts, hmax, eta, bin, st);
}

cudaError_t launch_spectrum(const float* vp, int n, int64_t T, int64_t vs,
                            const float2* twiddle, const float* wts, int hmax, float* eta,
                            int* bin, cudaStream_t st) {
  const int64_t blocks = (T + kDftThreads - 1) / kDftThreads;
  const int H = (n - 1) / 2, K = n / 2;
  if (n < 2 || n > kLongMaxN || hmax < 1) return cudaErrorInvalidValue;
  if (T == 0) return cudaSuccess;
  if (fft_length(n))
    return launch_spectrum_method(vp, n, T, vs, twiddle, wts, hmax, eta, bin, kSpectrumAuto, st);
  const bool harm = hmax > 1;
  if ((n & 1) == 0 && n <= 66) {
    const int m = n / 2, Hm = (m - 1) / 2, Kh = m / 2;
    const size_t sm = (size_t)(Hm > 0 ? Hm * Kh : 0) * sizeof(float2) + (size_t)m * sizeof(float2) +
                      (size_t)n * kDftThreads * sizeof(float);
    auto kern = harm ? k_dft_even<16, true> : k_dft_even<16, false>;
    kern<<<(unsigned)blocks, kDftThreads, sm, st>>>(vp, n, T, vs, twiddle, wts, hmax, eta, bin);
    count_launches(1);
    return cudaGetLastError();
  }
  if (n <= 65 && H >= 1) {
    const size_t sm = (size_t)H * K * sizeof(float2) + (size_t)n * kDftThreads * sizeof(float);
    auto kern = K <= 16 ? (harm ? k_dft_short<16, true> : k_dft_short<16, false>)
                        : (harm ? k_dft_short<32, true> : k_dft_short<32, false>);
    kern<<<(unsigned)blocks, kDftThreads, sm, st>>>(vp, n, T, vs, twiddle, wts, hmax, eta, bin);
    count_launches(1);
    return cudaGetLastError();
  }
  if (n > 256 || hmax > 1) return launch_long(vp, n, T, vs, twiddle, wts, hmax, eta, bin, st);
  const size_t smem = (size_t)n * kDftThreads * sizeof(float);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_dft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  k_dft<<<(unsigned)blocks, kDftThreads, smem, st>>>(vp, n, T, vs, twiddle, wts, eta, bin);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- ingest conversion
__device__ __forceinline__ float load_any(const void* p, int type, int64_t i) {
  if (type == FITRIG_BF16) return to_f32(static_cast<const bf16_t*>(p)[i]);
  if (type == FITRIG_F16) return to_f32(static_cast<const f16_t*>(p)[i]);
  return static_cast<const float*>(p)[i];
}

// Stores v in `type` (half types: round to nearest even) and returns the
// stored value as FP32.
__device__ __forceinline__ float store_any(void* p, int type, int64_t i, float v) {
  if (type == FITRIG_BF16) {
    unsigned short h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(v));
    static_cast<uint16_t*>(p)[i] = h;
    return __uint_as_float((uint32_t)h << 16);
  }
  if (type == FITRIG_F16) {
    unsigned short h;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(v));
    static_cast<uint16_t*>(p)[i] = h;
    float r;
    asm("cvt.f32.f16 %0, %1;" : "=f"(r) : "h"(h));
    return r;
  }
  static_cast<float*>(p)[i] = v;
  return v;
}

// Rows over blockIdx.y, columns over the threads of blockIdx.x (no per-pixel
// division).
__global__ void k_convert(const void* src, int st, int64_t sp, void* dst, int dt, int64_t dp,
                          int ny, int nx) {
  for (int y = blockIdx.y; y < ny; y += gridDim.y)
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x)
      store_any(dst, dt, (int64_t)y * dp + x, load_any(src, st, (int64_t)y * sp + x));
}

static dim3 image_grid(int ny, int nx) {
  return dim3((unsigned)std::min(8, (nx + 255) / 256), (unsigned)std::min(ny, 4096));
}

// Difference coding, closed loop (FITRIG_CODING_DELTA): the first snapshot is
// kept in FP32 (key frame) and starts the coder's decoded snapshot `state`;
// each later one stores q = round-to-nearest-even half of the FP32 difference
// x - state, and state advances by the decoded difference, fl32(state + q),
// exactly as the stack march decodes it.  NaN and infinities propagate.
__global__ void k_delta_encode(const void* src, int st, int64_t sp, float* state, float* key,
                               int64_t kp, void* dst, int dt, int64_t dp, int first, int ny,
                               int nx) {
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    float* srow = state + (int64_t)y * nx;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
      const float v = load_any(src, st, (int64_t)y * sp + x);
      if (first) {
        key[(int64_t)y * kp + x] = v;
        srow[x] = v;
      } else {
        const float prev = srow[x];
        const float q = store_any(dst, dt, (int64_t)y * dp + x, __fsub_rn(v, prev));
        srow[x] = __fadd_rn(prev, q);   // the decoded difference
      }
    }
  }
}

cudaError_t launch_delta_encode(const void* src, int src_type, int64_t src_pitch, float* state,
                                float* key, int64_t key_pitch, void* dst, int dst_type,
                                int64_t dst_pitch, bool first, int ny, int nx, cudaStream_t st) {
  k_delta_encode<<<image_grid(ny, nx), 256, 0, st>>>(src, src_type, src_pitch, state, key,
                                                     key_pitch, dst, dst_type, dst_pitch,
                                                     first ? 1 : 0, ny, nx);
  count_launches(1);
  return cudaGetLastError();
}

// Snapshot accumulation (Sec. 3.3.2): acc = x (first raw snapshot of a
// block) or acc + x in FP32; the last raw snapshot of the block stores the
// sum, in the storage type, to the stack slot instead.
__global__ void k_accumulate(const void* src, int st, int64_t sp, float* acc, int first, int last,
                             void* dst, int dt, int64_t dp, int ny, int nx) {
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    float* arow = acc + (int64_t)y * nx;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
      const float v = load_any(src, st, (int64_t)y * sp + x);
      const float a = first ? v : arow[x] + v;
      if (last) store_any(dst, dt, (int64_t)y * dp + x, a);
      else arow[x] = a;
    }
  }
}

cudaError_t launch_accumulate(const void* src, int src_type, int64_t src_pitch, float* acc,
                              bool first, bool last, void* dst, int dst_type, int64_t dst_pitch,
                              int ny, int nx, cudaStream_t st) {
  k_accumulate<<<image_grid(ny, nx), 256, 0, st>>>(src, src_type, src_pitch, acc, first ? 1 : 0,
                                                   last ? 1 : 0, dst, dst_type, dst_pitch, ny, nx);
  count_launches(1);
  return cudaGetLastError();
}

// A serving unit's frequency-series weight 1 / M_s^2 (FP64, rounded to FP32),
// with M_s the running maximum over every snapshot seen so far (its ordered
// key, 0 before any finite pixel), floored at C (Eq. 5's constant).
__global__ void k_unit_weight(const unsigned* gmax_key, float* w) {
  const unsigned k = *gmax_key;
  double m = k ? (double)f32_from_key(k) : 0.0;
  if (!(m > (double)kGuardC)) m = (double)kGuardC;
  *w = (float)(1.0 / (m * m));
}

cudaError_t launch_unit_weight(const unsigned* gmax_key, float* w, cudaStream_t st) {
  k_unit_weight<<<1, 1, 0, st>>>(gmax_key, w);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int src_type, int64_t src_pitch, void* dst,
                           int dst_type, int64_t dst_pitch, int ny, int nx, cudaStream_t st) {
  k_convert<<<image_grid(ny, nx), 256, 0, st>>>(src, src_type, src_pitch, dst, dst_type, dst_pitch,
                                                ny, nx);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- timestamps
// The GPU's global nanosecond timer, written when the stream reaches this
// point (serving: per-stage device times of a unit, read by the host without
// a CUDA call).
__global__ void k_stamp(long long* dst) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *dst = (long long)t;
}

cudaError_t launch_stamp(long long* dst, cudaStream_t st) {
  k_stamp<<<1, 1, 0, st>>>(dst);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- autotuner probe data
// Deterministic pseudo-random values in [-4, 4) (an integer hash of the index),
// used only as timing input for the autotuner.
__global__ void k_fill_probe(void* dst, int type, int64_t n, uint32_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    store_any(dst, type, i, ((float)(h >> 8) * (1.0f / 16777216.0f)) * 8.f - 4.f);
  }
}

cudaError_t launch_fill_probe(void* dst, int type, int64_t n, uint32_t seed, cudaStream_t st) {
  k_fill_probe<<<152 * 8, 256, 0, st>>>(dst, type, n, seed);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tLISI report
// tLISI = 1 - v / M^2 in FP64 (Eq. tLISI), M = max(stack maximum, C).
__global__ void k_tlisi(const float* vp, int64_t n, const unsigned* gmax, const double* m_unit,
                        float* out) {
  double M;
  if (m_unit) {
    M = *m_unit;
  } else {
    const unsigned key = *gmax;
    M = key ? (double)f32_from_key(key) : 0.0;
    if (!(M > (double)kGuardC)) M = (double)kGuardC;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)(1.0 - (double)vp[i] / (M * M));
}

cudaError_t launch_tlisi_from_values(const float* vp, int64_t n, const unsigned* gmax,
                                     const double* m_unit, float* out, cudaStream_t st) {
  k_tlisi<<<152 * 2, 256, 0, st>>>(vp, n, gmax, m_unit, out);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- running M
// Real-time reading of M (Sec. 2.2.4): unit s is normalised by the maximum
// over snapshots 0..s+2.  The march leaves each snapshot's maximum key in
// smax[k] (+inf included); a snapshot whose maximum is +inf gets the maximum
// of its finite pixels instead (rare: only stacks with non-finite pixels).
template <typename T>
__global__ void k_snap_finite_max(const T* stack, int L, int ny, int nx, int64_t pitch,
                                  size_t slice, unsigned* smax) {
  const unsigned inf_key = f32_key(INFINITY);
  for (int k = 0; k < L; ++k) {
    if (smax[k] != inf_key) continue;   // uniform: every thread reads the same word
    const T* x = stack + (size_t)k * slice;
    float m = -INFINITY;
    const int64_t total = (int64_t)ny * nx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
      const float v = to_f32(x[(i / nx) * pitch + (i % nx)]);
      if (isfinite(v)) m = fmaxf(m, v);
    }
    // the words are replaced only after every block has read them: write the
    // finite maxima to the upper half and let k_running_norm prefer it
    warp_max_to(m, smax + L + k);
  }
}

// M_s = max(C, max over k <= s + 2 of the snapshot maxima) for s < U, in FP64,
// and the series weights (M_{U-1} / M_s)^2 of the frequency branch, whose
// spectrum is then the spectrum of the tLISI series scaled by M^2 like the
// global reading's.
__global__ void k_running_norm(const unsigned* smax, int L, double* m_unit, float* wts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned inf_key = f32_key(INFINITY);
  const int U = L - 2;
  double run = (double)kGuardC;
  for (int k = 0; k < L; ++k) {
    unsigned key = smax[k];
    if (key == inf_key) key = smax[L + k];
    if (key) {
      const double v = (double)f32_from_key(key);
      if (v > run) run = v;   // NaN never compares greater
    }
    if (k >= 2) m_unit[k - 2] = run;
  }
  const double last = m_unit[U - 1];
  for (int s = 0; s < U; ++s) {
    const double q = last / m_unit[s];
    wts[s] = (float)(q * q);
  }
}

cudaError_t launch_running_norm(const void* stack, int storage, int L, int ny, int nx,
                                int64_t pitch, unsigned* smax, double* m_unit, float* wts,
                                cudaStream_t st) {
  const size_t slice = (size_t)pitch * ny;
  int n = 1;
  if (!stack) {
    // a difference-coded stack: the caller ran launch_delta_finite_max
  } else if (storage == FITRIG_F32)
    k_snap_finite_max<float><<<152 * 2, 256, 0, st>>>(static_cast<const float*>(stack), L, ny, nx,
                                                       pitch, slice, smax);
  else if (storage == FITRIG_BF16)
    k_snap_finite_max<bf16_t><<<152 * 2, 256, 0, st>>>(static_cast<const bf16_t*>(stack), L, ny,
                                                        nx, pitch, slice, smax);
  else
    k_snap_finite_max<f16_t><<<152 * 2, 256, 0, st>>>(static_cast<const f16_t*>(stack), L, ny, nx,
                                                       pitch, slice, smax);
  if (stack) n = 2;
  k_running_norm<<<1, 32, 0, st>>>(smax, L, m_unit, wts);
  count_launches(n);
  return cudaGetLastError();
}

}  // namespace fitrig
