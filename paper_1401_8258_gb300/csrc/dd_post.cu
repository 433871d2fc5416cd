// dd_post.cu -- post-processing of dedispersed series on the GPU:
//   dd_median_filter   windowed median (Sec. 3.5, median filtering);
//   dd_detrend         least-squares line removal and normalisation
//                      (Sec. 3.5, detrending and normalisation);
//   dd_boxcar_detect   boxcar smoothing by successive adjacent sums and n-sigma
//                      thresholding of every width (Sec. 1.5.1).
// All three are bound by HBM: each reads its rows about once (the median's
// window halo and the boxcar's width halo come from L2) and the arithmetic
// per sample is a handful of integer or float operations.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "dd_post.h"

namespace {

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? DD_OK : DD_ERR_CUDA; }

inline bool overlap(const void *a, size_t na, const void *b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

inline size_t row_span(int32_t nrows, int64_t pitch, int64_t ncols, size_t esize) {
  return (static_cast<size_t>(nrows - 1) * static_cast<size_t>(pitch) + static_cast<size_t>(ncols)) *
         esize;
}

template <typename T> __device__ __forceinline__ T vmin(T a, T b);
template <typename T> __device__ __forceinline__ T vmax(T a, T b);
template <> __device__ __forceinline__ int32_t vmin<int32_t>(int32_t a, int32_t b) { return min(a, b); }
template <> __device__ __forceinline__ int32_t vmax<int32_t>(int32_t a, int32_t b) { return max(a, b); }
template <> __device__ __forceinline__ float vmin<float>(float a, float b) { return fminf(a, b); }
template <> __device__ __forceinline__ float vmax<float>(float a, float b) { return fmaxf(a, b); }

// ------------------------------------------------------------------ median
//
// CTA = one tile of kMedTile outputs of one row.  The tile's samples and a
// halo of H on each side (clamped to the row: the window repeats the end
// sample) are staged in shared memory.  A thread takes output pairs
// (t, t + 1): their windows share the 2H samples t-H+1 .. t+H, whose two
// middle order statistics lo <= hi come from one sorting network; the median
// of a window is then its remaining sample clamped to [lo, hi].

constexpr int kMedThreads = 256;
constexpr int kMedTile = 4096;

// Ascending sort of s[0..N) by odd-even transposition (N rounds).
template <typename T, int N>
__device__ __forceinline__ void sort_network(T (&s)[N]) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
#pragma unroll
    for (int i = r & 1; i + 1 < N; i += 2) {
      const T a = s[i], b = s[i + 1];
      s[i] = vmin(a, b);
      s[i + 1] = vmax(a, b);
    }
  }
}

template <typename T> struct Pair;
template <> struct Pair<int32_t> { using type = int2; };
template <> struct Pair<float> { using type = float2; };

template <typename T, int H>
__global__ void __launch_bounds__(kMedThreads)
dd_median(const T *__restrict__ in, int64_t in_pitch, int64_t ncols, int ntiles,
          T *__restrict__ out, int64_t out_pitch, int pair_store) {
  using P2 = typename Pair<T>::type;
  __shared__ __align__(16) T s[kMedTile + 2 * H];
  const int64_t row = blockIdx.x / ntiles;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x % ntiles) * kMedTile;
  const T *x = in + row * in_pitch;
  T *y = out + row * out_pitch;
  // s[i] = sample t0 - H + i, clamped to the row; several loads in flight
  // per thread before their stores
  constexpr int kLoads = (kMedTile + 2 * H + kMedThreads - 1) / kMedThreads;
  T v[kLoads];
#pragma unroll
  for (int r = 0; r < kLoads; ++r) {
    const int i = threadIdx.x + r * kMedThreads;
    int64_t g = t0 - H + i;
    g = g < 0 ? 0 : (g >= ncols ? ncols - 1 : g);
    v[r] = i < kMedTile + 2 * H ? x[g] : T(0);
  }
#pragma unroll
  for (int r = 0; r < kLoads; ++r) {
    const int i = threadIdx.x + r * kMedThreads;
    if (i < kMedTile + 2 * H) s[i] = v[r];
  }
  __syncthreads();
  const P2 *s2 = reinterpret_cast<const P2 *>(s);
  for (int p = threadIdx.x; p < kMedTile / 2; p += kMedThreads) {
    const int64_t t = t0 + 2 * p;
    if (t >= ncols) break;
    // v[k] = sample t - H + k, k = 0 .. 2H+1 (window of t: v[0..2H], of t+1: v[1..2H+1])
    T v[2 * H + 2];
#pragma unroll
    for (int k = 0; k < H + 1; ++k) {
      const P2 q = s2[p + k];
      v[2 * k] = q.x;
      v[2 * k + 1] = q.y;
    }
    T m0, m1;
    if constexpr (H == 0) {
      m0 = v[0];
      m1 = v[1];
    } else {
      T c[2 * H];
#pragma unroll
      for (int k = 0; k < 2 * H; ++k) c[k] = v[k + 1];
      sort_network(c);
      const T lo = c[H - 1], hi = c[H];
      m0 = vmin(vmax(v[0], lo), hi);
      m1 = vmin(vmax(v[2 * H + 1], lo), hi);
    }
    if (pair_store && t + 1 < ncols) {
      P2 q;
      q.x = m0;
      q.y = m1;
      *reinterpret_cast<P2 *>(y + t) = q;
    } else {
      y[t] = m0;
      if (t + 1 < ncols) y[t + 1] = m1;
    }
  }
}

template <typename T>
int launch_median(const T *in, int64_t in_pitch, int32_t nrows, int64_t ncols, int width, T *out,
                  int64_t out_pitch, cudaStream_t s) {
  const int64_t ntiles = (ncols + kMedTile - 1) / kMedTile;
  if (ntiles * nrows > INT32_MAX) return DD_ERR_SIZE;
  const int grid = static_cast<int>(ntiles * nrows);
  // 8-byte pair stores when every row start is 8-byte aligned (t is even)
  const int pair_store = (reinterpret_cast<uintptr_t>(out) % 8 == 0) && (out_pitch % 2 == 0);
  const int nt = static_cast<int>(ntiles);
  switch (width / 2) {
    case 0: dd_median<T, 0><<<grid, kMedThreads, 0, s>>>(in, in_pitch, ncols, nt, out, out_pitch, pair_store); break;
    case 1: dd_median<T, 1><<<grid, kMedThreads, 0, s>>>(in, in_pitch, ncols, nt, out, out_pitch, pair_store); break;
    case 2: dd_median<T, 2><<<grid, kMedThreads, 0, s>>>(in, in_pitch, ncols, nt, out, out_pitch, pair_store); break;
    case 3: dd_median<T, 3><<<grid, kMedThreads, 0, s>>>(in, in_pitch, ncols, nt, out, out_pitch, pair_store); break;
    case 4: dd_median<T, 4><<<grid, kMedThreads, 0, s>>>(in, in_pitch, ncols, nt, out, out_pitch, pair_store); break;
    case 5: dd_median<T, 5><<<grid, kMedThreads, 0, s>>>(in, in_pitch, ncols, nt, out, out_pitch, pair_store); break;
    case 6: dd_median<T, 6><<<grid, kMedThreads, 0, s>>>(in, in_pitch, ncols, nt, out, out_pitch, pair_store); break;
    case 7: dd_median<T, 7><<<grid, kMedThreads, 0, s>>>(in, in_pitch, ncols, nt, out, out_pitch, pair_store); break;
    default: return DD_ERR_ARG;
  }
  return cuda_status(cudaGetLastError());
}

// ----------------------------------------------------------------- detrend
//
// CTA = one row.  Pass 1 sums the row: exactly in 128-bit integers for int32
// rows (Sy = sum y, Sty = sum t y, Syy = sum y^2), in float chunks of 16
// consecutive samples about the row's first value, added in double, for
// float rows.  Thread 0 solves the least-squares line from the centred sums
//   Sxx = n St2 - St^2,  Sxy = n Sty - St Sy,  Syyc = n Syy - Sy^2
// (St, St2: sums of t and t^2, closed forms).  Int rows: the residual sum of
// squares is n RSS = Syyc - Sxy^2 / Sxx, exactly zero when Syyc Sxx == Sxy^2
// (tested in 256 bits).  Float rows take the thesis's second pass instead,
// summing the squared residual itself.  The last pass writes (y - a - b t)/s
// in float: a + b t is formed in double once per 16 samples and split into
// an integer part (subtracted exactly from int rows) and a small float part.

constexpr int kDtThreads = 256;
constexpr int kDtChunk = 16;

using i128 = __int128;
using u128 = unsigned __int128;

__device__ double u128_to_double(u128 v) {
  const unsigned long long hi = static_cast<unsigned long long>(v >> 64);
  const unsigned long long lo = static_cast<unsigned long long>(v);
  if (hi == 0) return __ull2double_rn(lo);
  // top 64 bits with a sticky bit for everything below: one rounding
  const int drop = 64 - __clzll(static_cast<long long>(hi));
  const u128 mask = (static_cast<u128>(1) << drop) - 1;
  const unsigned long long top =
      static_cast<unsigned long long>(v >> drop) | static_cast<unsigned long long>((v & mask) != 0);
  return scalbn(__ull2double_rn(top), drop);
}

__device__ double i128_to_double(i128 v) {
  return v < 0 ? -u128_to_double(static_cast<u128>(-v)) : u128_to_double(static_cast<u128>(v));
}

// 256-bit product of two unsigned 128-bit values as (hi, lo).
__device__ void mul_u128(u128 a, u128 b, u128 *hi, u128 *lo) {
  const unsigned long long a0 = static_cast<unsigned long long>(a), a1 = static_cast<unsigned long long>(a >> 64);
  const unsigned long long b0 = static_cast<unsigned long long>(b), b1 = static_cast<unsigned long long>(b >> 64);
  const u128 p00 = static_cast<u128>(a0) * b0, p01 = static_cast<u128>(a0) * b1;
  const u128 p10 = static_cast<u128>(a1) * b0, p11 = static_cast<u128>(a1) * b1;
  const u128 mid = (p00 >> 64) + static_cast<unsigned long long>(p01) + static_cast<unsigned long long>(p10);
  *lo = (p00 & ~static_cast<unsigned long long>(0)) | (mid << 64);
  *hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
}

__device__ __forceinline__ i128 shfl_down_i128(i128 v, int o) {
  long long lo = static_cast<long long>(static_cast<unsigned long long>(v));
  long long hi = static_cast<long long>(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, o);
  hi = __shfl_down_sync(0xffffffffu, hi, o);
  return (static_cast<i128>(hi) << 64) | static_cast<unsigned long long>(lo);
}

// Sum of v over the CTA, valid in thread 0.
template <typename V>
__device__ V block_sum(V v, V *scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if constexpr (sizeof(V) == 16) {
      v += shfl_down_i128(v, o);
    } else {
      v += __shfl_down_sync(0xffffffffu, v, o);
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  V total = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kDtThreads / 32; ++k) total += scratch[k];
  return total;
}

// v[k] = x[t + k] for t + k < lim, else 0; one 16-byte load per four
// samples when the chunk is whole (x + t is then 16-byte aligned).
template <typename X>
__device__ __forceinline__ void load16(const X *x, int64_t t, int64_t lim, X (&v)[kDtChunk]) {
  if (t + kDtChunk <= lim) {
    const int4 *p = reinterpret_cast<const int4 *>(x + t);
#pragma unroll
    for (int q = 0; q < kDtChunk / 4; ++q) {
      const int4 u = p[q];
      v[4 * q] = *reinterpret_cast<const X *>(&u.x);
      v[4 * q + 1] = *reinterpret_cast<const X *>(&u.y);
      v[4 * q + 2] = *reinterpret_cast<const X *>(&u.z);
      v[4 * q + 3] = *reinterpret_cast<const X *>(&u.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < kDtChunk; ++k) v[k] = t + k < lim ? x[t + k] : X(0);
  }
}

// Pairwise (tree) sum of 16 floats.
__device__ __forceinline__ float tree16(const float (&v)[kDtChunk]) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = v[2 * k] + v[2 * k + 1];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = a[2 * k] + a[2 * k + 1];
  a[0] = a[0] + a[1];
  a[2] = a[2] + a[3];
  return a[0] + a[2];
}

// Least-squares line and residual rms of an int32 row from its exact sums
// (thread 0 only; kept out of line so that the sweep loops keep their
// registers).  line[0..3) = a, b, s.
__device__ __noinline__ void line_i32(i128 sy, i128 sty, i128 syy, int64_t n, double *line) {
  const i128 N = n, St = N * (N - 1) / 2, St2 = (N - 1) * N * (2 * N - 1) / 6;
  const i128 Sxx = N * St2 - St * St;  // 0 only for n == 1
  double a, b, s;
  if (Sxx == 0) {
    a = i128_to_double(sy);  // n == 1: the line is the sample
    b = 0.0;
    s = 0.0;
  } else {
    const i128 Sxy = N * sty - St * sy;
    const i128 Syyc = N * syy - sy * sy;  // >= 0
    const i128 An = sy * St2 - St * sty;  // a Sxx, exact
    const double dSxx = i128_to_double(Sxx);
    b = i128_to_double(Sxy) / dSxx;
    a = i128_to_double(An) / dSxx;
    u128 l_hi, l_lo, r_hi, r_lo;
    const u128 aSxy = static_cast<u128>(Sxy < 0 ? -Sxy : Sxy);
    mul_u128(static_cast<u128>(Syyc), static_cast<u128>(Sxx), &l_hi, &l_lo);
    mul_u128(aSxy, aSxy, &r_hi, &r_lo);
    if (l_hi == r_hi && l_lo == r_lo) {
      s = 0.0;
    } else {
      const double dSxy = i128_to_double(Sxy);
      const double rss_n = i128_to_double(Syyc) - dSxy * (dSxy / dSxx);
      s = rss_n > 0 ? sqrt(rss_n) / static_cast<double>(n) : 0.0;
    }
  }
  line[0] = a;
  line[1] = b;
  line[2] = s;
}

// Least-squares line of a float row from double sums of d = y - y0 and t d
// (thread 0 only).  line[0] = a, line[1] = b.
__device__ __noinline__ void line_f32(double sy, double sty, float y0, int64_t n, double *line) {
  const i128 N = n, St = N * (N - 1) / 2, St2 = (N - 1) * N * (2 * N - 1) / 6;
  const i128 Sxx = N * St2 - St * St;
  double a, b;
  if (Sxx == 0) {
    a = y0;
    b = 0.0;
  } else {
    const double dN = static_cast<double>(n), dSt = i128_to_double(St);
    const double dSt2 = i128_to_double(St2), dSxx = i128_to_double(Sxx);
    b = (dN * sty - dSt * sy) / dSxx;
    a = (sy * dSt2 - dSt * sty) / dSxx + static_cast<double>(y0);
  }
  line[0] = a;
  line[1] = b;
}

// One 16-sample chunk of an int32 row starting at sample t: its exact sums of
// y, t y and y^2 added to sy, sty, syy.
__device__ __forceinline__ void chunk_sums_i32(const int32_t (&v)[kDtChunk], int64_t t, i128 &sy,
                                               i128 &sty, i128 &syy) {
  long long c1 = 0, c2 = 0;  // chunk sums of y and of k y, k = 0..15
  u128 c3 = 0;
#pragma unroll
  for (int k = 0; k < kDtChunk; ++k) {
    const long long y = v[k];
    c1 += y;
    c2 += static_cast<long long>(k) * y;
    c3 += static_cast<u128>(static_cast<unsigned long long>(y * y));
  }
  sy += c1;
  sty += static_cast<i128>(t) * c1 + c2;
  syy += static_cast<i128>(c3);
}

// The chunk's detrended, normalised samples z[t + k] = (v[k] - (a + b (t+k))) / s
// for t + k < lim (the line evaluated as in the thesis: base = a + b t in
// double, split into integer and fraction, then per sample in float).
template <typename X>
__device__ __forceinline__ void chunk_out(const X (&v)[kDtChunk], int64_t t, int64_t lim,
                                          double a, double b, float bf, float inv, float *z,
                                          bool zvec) {
  const double base = fma(b, static_cast<double>(t), a);
  const double hi = floor(base);
  const float lo = static_cast<float>(base - hi);
  float r[kDtChunk];
#pragma unroll
  for (int k = 0; k < kDtChunk; ++k) {
    const float line = fmaf(bf, static_cast<float>(k), lo);
    if constexpr (std::is_integral<X>::value) {
      r[k] = static_cast<float>(static_cast<long long>(v[k]) - static_cast<long long>(hi)) - line;
    } else {
      r[k] = (v[k] - static_cast<float>(hi)) - line;
    }
    r[k] *= inv;
  }
  if (zvec && t + kDtChunk <= lim) {
    float4 *p = reinterpret_cast<float4 *>(z + t);
#pragma unroll
    for (int q = 0; q < kDtChunk / 4; ++q)
      p[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < kDtChunk; ++k)
      if (t + k < lim) z[t + k] = r[k];
  }
}

// Chunks of a row: the head [0, head) up to the first 16-byte boundary of the
// row (thread 0), then whole 16-sample chunks from `head`, one per thread
// in turn; `head` < 4.
template <typename F>
__device__ __forceinline__ void for_chunks(int64_t n, int head, F &&f) {
  if (threadIdx.x == 0 && head > 0) f(static_cast<int64_t>(0), static_cast<int64_t>(head));
  const int64_t step = static_cast<int64_t>(kDtThreads) * kDtChunk;
  for (int64_t t = head + static_cast<int64_t>(threadIdx.x) * kDtChunk; t < n; t += step)
    f(t, n);
}

template <typename X>
__global__ void __launch_bounds__(kDtThreads, 4)  // four rows in flight per SM
dd_detrend_rows(const X *in, int64_t in_pitch, int64_t n, float *out, int64_t out_pitch,
                double *coef) {  // no __restrict__: out may be in (float rows, in place)
  __shared__ i128 s_i[kDtThreads / 32];
  __shared__ double s_d[kDtThreads / 32];
  __shared__ double s_line[3];  // a, b, s
  const int64_t row = blockIdx.x;
  const X *x = in + row * in_pitch;
  float *z = out + row * out_pitch;
  const int head = static_cast<int>(
      min(n, static_cast<int64_t>(((16 - reinterpret_cast<uintptr_t>(x) % 16) % 16) / 4)));
  // 16-byte stores when the output row has the input row's alignment phase
  const bool zvec = (reinterpret_cast<uintptr_t>(z + head) % 16) == 0;

  if constexpr (std::is_integral<X>::value) {  // int32 rows: exact sums
    i128 sy = 0, sty = 0, syy = 0;
    for_chunks(n, head, [&](int64_t t, int64_t lim) {
      X v[kDtChunk];
      load16<X>(x, t, lim, v);
      chunk_sums_i32(v, t, sy, sty, syy);
    });
    sy = block_sum(sy, s_i);
    sty = block_sum(sty, s_i);
    syy = block_sum(syy, s_i);
    if (threadIdx.x == 0) line_i32(sy, sty, syy, n, s_line);
  } else {  // float rows: three passes in the thesis's order
    const float y0 = x[0];
    double sy = 0, sty = 0;
    for_chunks(n, head, [&](int64_t t, int64_t lim) {
      X v[kDtChunk];
      load16<X>(x, t, lim, v);
      float d[kDtChunk], kd[kDtChunk];
#pragma unroll
      for (int k = 0; k < kDtChunk; ++k) {
        d[k] = t + k < lim ? v[k] - y0 : 0.0f;
        kd[k] = static_cast<float>(k) * d[k];
      }
      const double c1 = tree16(d), c2 = tree16(kd);
      sy += c1;
      sty += static_cast<double>(t) * c1 + c2;
    });
    sy = block_sum(sy, s_d);
    sty = block_sum(sty, s_d);
    if (threadIdx.x == 0) line_f32(sy, sty, y0, n, s_line);
    __syncthreads();
    const double a = s_line[0], b = s_line[1];
    const float bf = static_cast<float>(b);
    double rss = 0;
    for_chunks(n, head, [&](int64_t t, int64_t lim) {
      X v[kDtChunk];
      load16<X>(x, t, lim, v);
      const double base = fma(b, static_cast<double>(t), a);
      const double hi = floor(base);
      const float lo = static_cast<float>(base - hi), hf = static_cast<float>(hi);
      float r2[kDtChunk];
#pragma unroll
      for (int k = 0; k < kDtChunk; ++k) {
        const float r = (v[k] - hf) - fmaf(bf, static_cast<float>(k), lo);
        r2[k] = t + k < lim ? r * r : 0.0f;
      }
      rss += tree16(r2);
    });
    rss = block_sum(rss, s_d);
    if (threadIdx.x == 0) s_line[2] = rss > 0 ? sqrt(rss / static_cast<double>(n)) : 0.0;
  }
  __syncthreads();
  const double a = s_line[0], b = s_line[1], s = s_line[2];
  if (coef && threadIdx.x == 0) {
    coef[3 * row] = a;
    coef[3 * row + 1] = b;
    coef[3 * row + 2] = s;
  }
  const float inv = s > 0 ? static_cast<float>(1.0 / s) : 0.0f;
  const float bf = static_cast<float>(b);
  for_chunks(n, head, [&](int64_t t, int64_t lim) {
    X v[kDtChunk];
    load16<X>(x, t, lim, v);
    chunk_out(v, t, lim, a, b, bf, inv, z, zvec);
  });
}

// ------------------------------------------------------------------ boxcar
//
// Thresholds: for each (row, width) the smallest sum that passes the double
// S/N test (a bisection over int64 sums or over floats in order; the test is
// monotone in the sum), so the sweep compares sums only.
// Sweep (count pass, then write pass for tiles with pulses): CTA = one tile
// of kBoxTile start samples of one row; the tile plus a halo of
// 2^(nwidths-1) - 1 samples sits in shared memory and is replaced, width by
// width, by S_2w[i] = S_w[i] + S_w[i + w]; thread k owns elements
// k + 256 m in registers.  Pulses of a tile are ranked by start sample
// through a bitmap, after an exclusive scan of the per-tile counts in
// (row, tile) order, so the list is ordered by (row, t).

constexpr int kBoxThreads = 256;
constexpr int kBoxTile = 4096;
constexpr int kBoxOwn = kBoxTile / kBoxThreads;  // 16 outputs per thread
constexpr int kMaxWidths = 12;
constexpr int kBoxPer = (kBoxTile + (1 << (kMaxWidths - 1)) - 1 + kBoxThreads - 1) / kBoxThreads;
constexpr int kSmallWidths = 8;  // up to 128 samples: fewer registers per thread
constexpr int kBoxPerSmall =
    (kBoxTile + (1 << (kSmallWidths - 1)) - 1 + kBoxThreads - 1) / kBoxThreads;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ double boxcar_snr(double sum, int w, double mean, double sigma) {
  const double dw = static_cast<double>(w);
  return __ddiv_rn(__dsub_rn(sum, __dmul_rn(dw, mean)), __dmul_rn(sigma, __dsqrt_rn(dw)));
}

__device__ __forceinline__ uint32_t float_key(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// thr[row][j]: int rows -> smallest passing int64 sum (INT64_MAX: none);
// float rows -> bits of the smallest passing float (a NaN: none).
__global__ void dd_boxcar_thresholds(int32_t rows_type, int32_t nrows, int nwidths,
                                     const double *mean, const double *sigma, double nsigma,
                                     int64_t *thr) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<int64_t>(nrows) * kMaxWidths) return;
  const int64_t row = idx / kMaxWidths;
  const int j = static_cast<int>(idx % kMaxWidths);
  const double mu = mean ? mean[row] : 0.0, sg = sigma ? sigma[row] : 1.0;
  const bool ok = j < nwidths && isfinite(mu) && isfinite(sg) && sg > 0.0;
  const int w = 1 << j;
  if (rows_type == DD_ROWS_I32) {
    int64_t res = INT64_MAX;
    if (ok) {
      // |sums| < 2^43, so [-2^53, 2^53] brackets every decision
      int64_t lo = -(static_cast<int64_t>(1) << 53), hi = static_cast<int64_t>(1) << 53;
      if (boxcar_snr(static_cast<double>(lo), w, mu, sg) > nsigma) {
        res = lo;
      } else if (boxcar_snr(static_cast<double>(hi), w, mu, sg) > nsigma) {
        while (hi - lo > 1) {  // pass(lo) false, pass(hi) true
          const int64_t mid = lo + (hi - lo) / 2;
          if (boxcar_snr(static_cast<double>(mid), w, mu, sg) > nsigma) hi = mid; else lo = mid;
        }
        res = hi;
      }
    }
    thr[idx] = res;
  } else {
    uint32_t bits = 0x7fc00000u;  // NaN: no sum passes
    if (ok) {
      uint32_t lo = float_key(-INFINITY), hi = float_key(INFINITY);
      if (boxcar_snr(-static_cast<double>(INFINITY), w, mu, sg) > nsigma) {
        bits = __float_as_uint(-INFINITY);
      } else if (boxcar_snr(static_cast<double>(INFINITY), w, mu, sg) > nsigma) {
        while (hi - lo > 1) {
          const uint32_t mid = lo + (hi - lo) / 2;
          if (boxcar_snr(static_cast<double>(key_float(mid)), w, mu, sg) > nsigma) hi = mid; else lo = mid;
        }
        bits = __float_as_uint(key_float(hi));
      }
    }
    thr[idx] = static_cast<int64_t>(bits);
  }
}

template <typename V>
__device__ __forceinline__ bool passes(V s, int64_t thr);
template <> __device__ __forceinline__ bool passes<long long>(long long s, int64_t thr) { return s >= thr; }
template <> __device__ __forceinline__ bool passes<float>(float s, int64_t thr) {
  return s >= __uint_as_float(static_cast<uint32_t>(thr));
}

template <typename X, typename V, bool WRITE, int PER>
__global__ void __launch_bounds__(kBoxThreads)
dd_boxcar_sweep(const X *__restrict__ rows, int64_t pitch, int64_t ncols, int ntiles, int nwidths,
                const int64_t *__restrict__ thr_all, const double *mean, const double *sigma,
                int64_t *__restrict__ counts, const int64_t *__restrict__ offsets,
                dd_pulse *__restrict__ pulses, int64_t capacity) {
  // two buffers of E sums: width w reads buffer (j-1)&1 and writes j&1, so
  // one barrier per width separates every read from the next overwrite
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_thr[kMaxWidths];
  __shared__ double s_wmu[kMaxWidths], s_den[kMaxWidths], s_rden[kMaxWidths];
  __shared__ uint32_t s_bits[kBoxTile / 32];
  __shared__ int s_pre[kBoxTile / 32];
  __shared__ int s_cnt[kBoxThreads / 32];
  if (WRITE && counts[blockIdx.x] == 0) return;
  const int64_t row = blockIdx.x / ntiles;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x % ntiles) * kBoxTile;
  const X *x = rows + row * pitch;
  const int E = kBoxTile + (1 << (nwidths - 1)) - 1;
  V *buf0 = reinterpret_cast<V *>(smem_raw);
  V *buf1 = buf0 + E;
  if (threadIdx.x < kMaxWidths) {
    const int j = threadIdx.x;
    s_thr[j] = thr_all[row * kMaxWidths + j];
    if (WRITE) {
      // the S/N's constant parts, rounded exactly as in the S/N itself
      const double mu = mean ? mean[row] : 0.0, sg = sigma ? sigma[row] : 1.0;
      const double dw = static_cast<double>(1 << j);
      s_wmu[j] = __dmul_rn(dw, mu);
      s_den[j] = __dmul_rn(sg, __dsqrt_rn(dw));
      s_rden[j] = 1.0 / s_den[j];
    }
  }
  V reg[PER];
#pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int i = threadIdx.x + kBoxThreads * m;
    const int64_t g = t0 + i;
    reg[m] = (i < E && g < ncols) ? static_cast<V>(x[g]) : V(0);
    if (i < E) buf0[i] = reg[m];
  }
  __syncthreads();
  uint32_t mask = 0;  // bit m: element threadIdx.x + 256 m is a pulse start
  // write pass: per owned element the best width so far, its sum and an
  // approximate S/N (num / den through a rounded reciprocal: within a few
  // units in the last place of the exact quotient)
  double ba[WRITE ? kBoxOwn : 1];
  int bj[WRITE ? kBoxOwn : 1];
  V bval[WRITE ? kBoxOwn : 1];
  if constexpr (WRITE) {
#pragma unroll
    for (int m = 0; m < kBoxOwn; ++m) {
      ba[m] = -INFINITY;
      bj[m] = -1;
      bval[m] = V(0);
    }
  }
  for (int j = 0; j < nwidths; ++j) {
    const int w = 1 << j;
    if (j > 0) {
      const int half = w >> 1, lim = E - w + 1;
      const V *src = (j & 1) ? buf0 : buf1;
      V *dst = (j & 1) ? buf1 : buf0;
#pragma unroll
      for (int m = 0; m < PER; ++m) {
        const int i = threadIdx.x + kBoxThreads * m;
        if (i < lim) {
          reg[m] = reg[m] + src[i + half];
          dst[i] = reg[m];
        }
      }
    }
    const int64_t thr = s_thr[j];
#pragma unroll
    for (int m = 0; m < kBoxOwn; ++m) {
      const int64_t t = t0 + threadIdx.x + kBoxThreads * m;
      if (t + w <= ncols && passes<V>(reg[m], thr)) {
        mask |= 1u << m;
        if constexpr (WRITE) {
          // the oracle keeps the first width with the largest exact S/N;
          // the approximation decides unless two widths are within 2^-40
          const double num = __dsub_rn(static_cast<double>(reg[m]), s_wmu[j]);
          const double a = num * s_rden[j];
          bool take;
          if (bj[m] < 0) {
            take = true;
          } else if (fabs(a - ba[m]) > 0x1p-40 * fmax(fabs(a), fabs(ba[m]))) {
            take = a > ba[m];
          } else {
            const int k = bj[m];
            const double e_old =
                __ddiv_rn(__dsub_rn(static_cast<double>(bval[m]), s_wmu[k]), s_den[k]);
            take = __ddiv_rn(num, s_den[j]) > e_old;
          }
          if (take) {
            ba[m] = a;
            bj[m] = j;
            bval[m] = reg[m];
          }
        }
      }
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if constexpr (!WRITE) {
    int c = __popc(mask);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) s_cnt[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int total = 0;
      for (int k = 0; k < kBoxThreads / 32; ++k) total += s_cnt[k];
      counts[blockIdx.x] = total;
    }
  } else {
    // element i = threadIdx.x + 256 m lies in word (i >> 5) = warp + 8 m, bit lane
#pragma unroll
    for (int m = 0; m < kBoxOwn; ++m) {
      const uint32_t b = __ballot_sync(0xffffffffu, (mask >> m) & 1u);
      if (lane == 0) s_bits[warp + (kBoxThreads / 32) * m] = b;
    }
    __syncthreads();
    if (threadIdx.x < kBoxTile / 32) {  // exclusive prefix of the word counts (4 warps)
      const int c = __popc(s_bits[threadIdx.x]);
      int inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      if (lane == 31) s_cnt[warp] = inc;
      s_pre[threadIdx.x] = inc - c;
    }
    __syncthreads();
    if (threadIdx.x < kBoxTile / 32) {
      int add = 0;
      for (int k = 0; k < warp; ++k) add += s_cnt[k];
      s_pre[threadIdx.x] += add;
    }
    __syncthreads();
    const int64_t base = offsets[blockIdx.x];
#pragma unroll
    for (int m = 0; m < kBoxOwn; ++m) {
      if (!((mask >> m) & 1u)) continue;
      const int i = threadIdx.x + kBoxThreads * m;
      const int word = i >> 5;
      const int64_t pos =
          base + s_pre[word] + __popc(s_bits[word] & ((1u << (i & 31)) - 1u));
      if (pos < capacity) {
        dd_pulse p;
        p.dm_idx = static_cast<int32_t>(row);
        p.t = static_cast<int32_t>(t0 + i);
        const int k = bj[m];
        p.width = 1 << k;
        p.snr = __double2float_rn(
            __ddiv_rn(__dsub_rn(static_cast<double>(bval[m]), s_wmu[k]), s_den[k]));
        p.value = static_cast<double>(bval[m]);
        pulses[pos] = p;
      }
    }
  }
}

// Count and write passes for up to kSmallWidths widths, in registers: CTA =
// the same 4096-sample tile as dd_boxcar_sweep, split between its warps.
// Lane l of a warp holds K consecutive samples of the warp's window (32 K >=
// the warp's start samples + 127, the largest width's reach), staged through
// shared memory so that the global loads are coalesced; each width's sums
// S_2w[k] = S_w[k] + S_w[k + w] take the partner from the lane's own
// registers or, past its K samples, from the next lanes by shuffle (fetched
// before the in-place update, so every partner is still a width-w sum).
// Lanes past the warp's start samples only feed others; a start sample's sums
// never reach past the window, so values shuffled in from beyond the warp
// never reach a counted sum.
// Two shapes: the count pass keeps 36 samples per lane (1024 start samples
// per warp, 4 warps: the fewest halo samples); the write pass keeps 20 per
// lane (512 per warp, 8 warps: twice the warps per SM for the same shared
// memory, which its per-sample state fills).
template <bool WRITE> struct RegShape;
template <> struct RegShape<false> { static constexpr int K = 36, OWN = 1024; };
template <> struct RegShape<true> { static constexpr int K = 20, OWN = 512; };

// Per start sample of a warp, the best width so far (write pass), and a
// queue of the samples that pass at the current width: their S/N work runs
// on all 32 lanes instead of on the few lanes a pulse lights up.
template <typename V, int OWN>
struct BestState {
  float a[OWN];          // S/N through the rounded reciprocal (float)
  V val[OWN];            // its sum
  V qval[OWN];           // queue: sums
  short qpos[OWN];       // queue: positions in the warp's range
  unsigned char j[OWN];  // its width index (0xff: none yet)
};

// Dynamic shared memory of dd_boxcar_regs: the staging area, which the
// write pass then reuses for the best-width state.
template <typename V, bool WRITE>
constexpr size_t reg_smem_bytes() {
  constexpr int K = RegShape<WRITE>::K, OWN = RegShape<WRITE>::OWN, W = kBoxTile / OWN;
  constexpr size_t stage = sizeof(V) * W * 32 * (K + 1);
  constexpr size_t best = sizeof(BestState<V, OWN>) * W;
  return (!WRITE || stage > best) ? stage : best;
}

template <typename X, typename V, bool WRITE>
__global__ void __launch_bounds__(kBoxTile / RegShape<WRITE>::OWN * 32)
dd_boxcar_regs(const X *__restrict__ rows, int64_t pitch, int64_t ncols, int ntiles, int nwidths,
               const int64_t *__restrict__ thr_all, const double *mean, const double *sigma,
               int64_t *__restrict__ counts, const int64_t *__restrict__ offsets,
               dd_pulse *__restrict__ pulses, int64_t capacity) {
  // the staging area is reused for the write pass's best-width state
  constexpr int kLaneK = RegShape<WRITE>::K, kWarpOwn = RegShape<WRITE>::OWN;
  constexpr int kRegWarps = kBoxTile / kWarpOwn;
  static_assert(32 * kLaneK >= kWarpOwn + (1 << (kSmallWidths - 1)) - 1, "window too short");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_thr[kMaxWidths];
  __shared__ double s_wmu[kMaxWidths], s_den[kMaxWidths], s_rden[kMaxWidths];
  __shared__ int s_cnt[kRegWarps];
  if (WRITE && counts[blockIdx.x] == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row = blockIdx.x / ntiles;
  const int64_t seg = static_cast<int64_t>(blockIdx.x % ntiles) * kBoxTile +
                      static_cast<int64_t>(warp) * kWarpOwn;
  const X *x = rows + row * pitch;
  if (threadIdx.x < kMaxWidths) {
    const int j = threadIdx.x;
    s_thr[j] = thr_all[row * kMaxWidths + j];
    if (WRITE) {
      const double mu = mean ? mean[row] : 0.0, sg = sigma ? sigma[row] : 1.0;
      const double dw = static_cast<double>(1 << j);
      s_wmu[j] = __dmul_rn(dw, mu);
      s_den[j] = __dmul_rn(sg, __dsqrt_rn(dw));
      s_rden[j] = 1.0 / s_den[j];
    }
  }
  V *st = reinterpret_cast<V *>(smem_raw) + warp * 32 * (kLaneK + 1);
#pragma unroll 4
  for (int q = 0; q < kLaneK; ++q) {
    const int p = lane + 32 * q;  // position in the warp's window
    const int64_t g = seg + p;
    st[(p / kLaneK) * (kLaneK + 1) + p % kLaneK] = g < ncols ? static_cast<V>(x[g]) : V(0);
  }
  __syncthreads();
  V v[kLaneK];
#pragma unroll
  for (int k = 0; k < kLaneK; ++k) v[k] = st[lane * (kLaneK + 1) + k];
  if (WRITE) __syncthreads();  // staging read: the area now holds the best-width state
  BestState<V, kWarpOwn> *bs = reinterpret_cast<BestState<V, kWarpOwn> *>(smem_raw) + warp;
  const int base = lane * kLaneK;        // first position of this lane
  const int64_t t_lane = seg + base;
  if (WRITE) {
    for (int k = lane; k < kWarpOwn; k += 32) bs->j[k] = 0xff;
    __syncwarp();
  }
  // a warp whose every counted sum ends inside the row needs no per-sample
  // length test; lane ownership (positions below 1024) is applied at the end
  const bool interior = seg + kWarpOwn - 1 + (1 << (nwidths - 1)) <= ncols;
  uint64_t mask = 0;
#pragma unroll
  for (int j = 0; j < kSmallWidths; ++j) {
    if (j >= nwidths) break;
    if (j > 0) {
      const int h = 1 << (j - 1);
      V part[kLaneK];
#pragma unroll
      for (int k = 0; k < kLaneK; ++k) {
        if (k + h >= kLaneK) {
          const int idx = k + h;
          part[k] = __shfl_down_sync(0xffffffffu, v[idx % kLaneK], idx / kLaneK);
        }
      }
#pragma unroll
      for (int k = 0; k < kLaneK; ++k) v[k] = v[k] + (k + h < kLaneK ? v[k + h] : part[k]);
    }
    const int w = 1 << j;
    const int64_t thr = s_thr[j];
    uint64_t hit = 0;
    if (interior) {
#pragma unroll
      for (int k = 0; k < kLaneK; ++k)
        if (passes<V>(v[k], thr)) hit |= 1ull << k;
    } else {
#pragma unroll
      for (int k = 0; k < kLaneK; ++k)
        if (t_lane + k + w <= ncols && passes<V>(v[k], thr)) hit |= 1ull << k;
    }
    if constexpr (WRITE) {
      // queue this width's passing owned samples in position order
      const int own_k = kWarpOwn - base;
      const uint64_t q = own_k <= 0 ? 0 : (own_k >= kLaneK ? hit : hit & ((1ull << own_k) - 1));
      const int nq = __popcll(q);
      int inc = nq;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      const int total = __shfl_sync(0xffffffffu, inc, 31);
      if (total > 0) {
        int e = inc - nq;
#pragma unroll
        for (int k = 0; k < kLaneK; ++k) {
          if ((q >> k) & 1) {
            bs->qpos[e] = static_cast<short>(base + k);
            bs->qval[e] = v[k];
            ++e;
          }
        }
        __syncwarp();
        // the oracle keeps the first width with the largest exact S/N; the
        // float approximation decides unless two widths are within 2^-20
        for (int e2 = lane; e2 < total; e2 += 32) {
          const int i = bs->qpos[e2];
          const V val = bs->qval[e2];
          const double num = __dsub_rn(static_cast<double>(val), s_wmu[j]);
          const float a = static_cast<float>(num * s_rden[j]);
          const int oj = bs->j[i];
          bool take;
          if (oj == 0xff) {
            take = true;
          } else if (fabsf(a - bs->a[i]) > 0x1p-20f * fmaxf(fabsf(a), fabsf(bs->a[i]))) {
            take = a > bs->a[i];
          } else {
            const double e_old =
                __ddiv_rn(__dsub_rn(static_cast<double>(bs->val[i]), s_wmu[oj]), s_den[oj]);
            take = __ddiv_rn(num, s_den[j]) > e_old;
          }
          if (take) {
            bs->a[i] = a;
            bs->j[i] = static_cast<unsigned char>(j);
            bs->val[i] = val;
          }
        }
        __syncwarp();
      }
    }
    mask |= hit;
  }
  // positions at or past the warp's 1024 belong to the next warp
  const int own = kWarpOwn - base;  // <= 0: none, >= kLaneK: all
  if (own <= 0) mask = 0;
  else if (own < kLaneK) mask &= (1ull << own) - 1;
  const int mine = __popcll(mask);
  if constexpr (!WRITE) {
    int c = mine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) s_cnt[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int total = 0;
      for (int k = 0; k < kRegWarps; ++k) total += s_cnt[k];
      counts[blockIdx.x] = total;
    }
  } else {
    // lanes' segments are in time order: rank = pulses of earlier warps and
    // lanes + earlier pulses of this lane
    int inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) s_cnt[warp] = inc;
    __syncthreads();
    int warp_before = 0;
    for (int k = 0; k < warp; ++k) warp_before += s_cnt[k];
    const int total = s_cnt[warp];
    // the warp's pulses in position order, then written by all lanes
    int e = inc - mine;
#pragma unroll
    for (int k = 0; k < kLaneK; ++k) {
      if ((mask >> k) & 1) {
        bs->qpos[e] = static_cast<short>(base + k);
        ++e;
      }
    }
    __syncwarp();
    const int64_t pos0 = offsets[blockIdx.x] + warp_before;
    for (int e2 = lane; e2 < total; e2 += 32) {
      const int64_t pos = pos0 + e2;
      if (pos >= capacity) break;
      const int i = bs->qpos[e2];
      const int bj = bs->j[i];
      dd_pulse p;
      p.dm_idx = static_cast<int32_t>(row);
      p.t = static_cast<int32_t>(seg + i);
      p.width = 1 << bj;
      p.snr = __double2float_rn(
          __ddiv_rn(__dsub_rn(static_cast<double>(bs->val[i]), s_wmu[bj]), s_den[bj]));
      p.value = static_cast<double>(bs->val[i]);
      pulses[pos] = p;
    }
  }
}

// Single-CTA exclusive scan of m counts; *total gets their sum.
__global__ void __launch_bounds__(kScanThreads)
dd_boxcar_scan(const int64_t *__restrict__ counts, int64_t m, int64_t *__restrict__ offsets,
               int64_t *__restrict__ total) {
  __shared__ int64_t s_part[kScanThreads];
  const int64_t per = (m + kScanThreads - 1) / kScanThreads;
  const int64_t lo = threadIdx.x * per;
  const int64_t hi = lo + per < m ? lo + per : m;
  int64_t sum = 0;
  for (int64_t i = lo; i < hi; ++i) sum += counts[i];
  s_part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const int64_t add = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0;
    __syncthreads();
    s_part[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t run = s_part[threadIdx.x] - sum;
  for (int64_t i = lo; i < hi; ++i) {
    offsets[i] = run;
    run += counts[i];
  }
  if (threadIdx.x == kScanThreads - 1) *total = s_part[kScanThreads - 1];
}

inline int64_t box_tiles(int64_t ncols) { return (ncols + kBoxTile - 1) / kBoxTile; }

inline int64_t box_workspace(int32_t nrows, int64_t ncols) {
  const int64_t m = static_cast<int64_t>(nrows) * box_tiles(ncols);
  return 8 * (static_cast<int64_t>(nrows) * kMaxWidths + 2 * m + 2);
}

template <typename X, typename V, int PER>
cudaError_t sweep_launches(const X *rows, int64_t pitch, int64_t ncols, int ntiles, int nwidths,
                           const int64_t *thr, const double *mean, const double *sigma,
                           int64_t *counts, int64_t *offsets, int64_t *total, int64_t m,
                           dd_pulse *pulses, int64_t capacity, unsigned grid, size_t smem,
                           cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(dd_boxcar_sweep<X, V, false, PER>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dd_boxcar_sweep<X, V, true, PER>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (PER == kBoxPerSmall) {  // up to kSmallWidths widths: the register passes
    const size_t rc = reg_smem_bytes<V, false>(), rw = reg_smem_bytes<V, true>();
    e = cudaFuncSetAttribute(dd_boxcar_regs<X, V, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(rc));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dd_boxcar_regs<X, V, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(rw));
    if (e != cudaSuccess) return e;
    dd_boxcar_regs<X, V, false><<<grid, kBoxTile / RegShape<false>::OWN * 32, rc, s>>>(
        rows, pitch, ncols, ntiles, nwidths, thr, mean, sigma, counts, offsets, pulses, capacity);
    dd_boxcar_scan<<<1, kScanThreads, 0, s>>>(counts, m, offsets, total);
    if (capacity > 0)
      dd_boxcar_regs<X, V, true><<<grid, kBoxTile / RegShape<true>::OWN * 32, rw, s>>>(
          rows, pitch, ncols, ntiles, nwidths, thr, mean, sigma, counts, offsets, pulses,
          capacity);
    return cudaGetLastError();
  }
  dd_boxcar_sweep<X, V, false, PER><<<grid, kBoxThreads, smem, s>>>(
      rows, pitch, ncols, ntiles, nwidths, thr, mean, sigma, counts, offsets, pulses, capacity);
  dd_boxcar_scan<<<1, kScanThreads, 0, s>>>(counts, m, offsets, total);
  if (capacity > 0)
    dd_boxcar_sweep<X, V, true, PER><<<grid, kBoxThreads, smem, s>>>(
        rows, pitch, ncols, ntiles, nwidths, thr, mean, sigma, counts, offsets, pulses, capacity);
  return cudaGetLastError();
}

template <typename X, typename V>
int launch_boxcar(const X *rows, int64_t pitch, int32_t nrows, int64_t ncols, const double *mean,
                  const double *sigma, int nwidths, float nsigma, unsigned char *ws, dd_pulse *pulses,
                  int64_t capacity, int64_t *count, cudaStream_t s) {
  const int64_t ntiles = box_tiles(ncols);
  const int64_t m = ntiles * nrows;
  int64_t *thr = reinterpret_cast<int64_t *>(ws);
  int64_t *counts = thr + static_cast<int64_t>(nrows) * kMaxWidths;
  int64_t *offsets = counts + m;
  int64_t *total = offsets + m;
  const int rows_type = sizeof(V) == 8 ? DD_ROWS_I32 : DD_ROWS_F32;
  const int64_t nthr = static_cast<int64_t>(nrows) * kMaxWidths;
  dd_boxcar_thresholds<<<static_cast<unsigned>((nthr + 255) / 256), 256, 0, s>>>(
      rows_type, nrows, nwidths, mean, sigma, static_cast<double>(nsigma), thr);
  const int E = kBoxTile + (1 << (nwidths - 1)) - 1;
  const size_t smem = 2 * static_cast<size_t>(E) * sizeof(V);
  const unsigned grid = static_cast<unsigned>(m);
  const int nt = static_cast<int>(ntiles);
  cudaError_t e;
  if (nwidths <= kSmallWidths)
    e = sweep_launches<X, V, kBoxPerSmall>(rows, pitch, ncols, nt, nwidths, thr, mean, sigma,
                                           counts, offsets, total, m, pulses, capacity, grid,
                                           smem, s);
  else
    e = sweep_launches<X, V, kBoxPer>(rows, pitch, ncols, nt, nwidths, thr, mean, sigma, counts,
                                      offsets, total, m, pulses, capacity, grid, smem, s);
  if (e != cudaSuccess) return DD_ERR_CUDA;
  e = cudaGetLastError();
  if (e != cudaSuccess) return DD_ERR_CUDA;
  int64_t found = 0;
  e = cudaMemcpyAsync(&found, total, sizeof(found), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return DD_ERR_CUDA;
  *count = found;
  return found > capacity ? DD_ERR_OVERFLOW : DD_OK;
}

}  // namespace

extern "C" int dd_median_filter(const void *in, int64_t in_pitch, int32_t rows_type, int32_t nrows,
                                int64_t ncols, int32_t width, void *out, int64_t out_pitch,
                                void *stream) {
  if (rows_type != DD_ROWS_I32 && rows_type != DD_ROWS_F32) return DD_ERR_DTYPE;
  if (!in || !out) return DD_ERR_ARG;
  if (nrows < 1 || ncols < 1 || ncols > INT32_MAX) return DD_ERR_SIZE;
  if (width < 1 || width > 15 || width % 2 == 0) return DD_ERR_ARG;
  if (in_pitch < ncols || out_pitch < ncols) return DD_ERR_ARG;
  if (overlap(in, row_span(nrows, in_pitch, ncols, 4), out, row_span(nrows, out_pitch, ncols, 4)))
    return DD_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (rows_type == DD_ROWS_I32)
    return launch_median(static_cast<const int32_t *>(in), in_pitch, nrows, ncols, width,
                         static_cast<int32_t *>(out), out_pitch, s);
  return launch_median(static_cast<const float *>(in), in_pitch, nrows, ncols, width,
                       static_cast<float *>(out), out_pitch, s);
}

extern "C" int dd_detrend(const void *in, int64_t in_pitch, int32_t rows_type, int32_t nrows,
                          int64_t ncols, float *out, int64_t out_pitch, double *coef, void *stream) {
  if (rows_type != DD_ROWS_I32 && rows_type != DD_ROWS_F32) return DD_ERR_DTYPE;
  if (!in || !out) return DD_ERR_ARG;
  if (nrows < 1 || ncols < 1 || ncols > (static_cast<int64_t>(1) << 24)) return DD_ERR_SIZE;
  if (in_pitch < ncols || out_pitch < ncols) return DD_ERR_ARG;
  const bool same = static_cast<const void *>(out) == in && out_pitch == in_pitch;
  if (!(same && rows_type == DD_ROWS_F32) &&
      overlap(in, row_span(nrows, in_pitch, ncols, 4), out, row_span(nrows, out_pitch, ncols, 4)))
    return DD_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (reinterpret_cast<uintptr_t>(in) % 4 != 0 || reinterpret_cast<uintptr_t>(out) % 4 != 0)
    return DD_ERR_ARG;
  if (rows_type == DD_ROWS_I32)
    dd_detrend_rows<int32_t><<<nrows, kDtThreads, 0, s>>>(static_cast<const int32_t *>(in),
                                                          in_pitch, ncols, out, out_pitch, coef);
  else
    dd_detrend_rows<float><<<nrows, kDtThreads, 0, s>>>(static_cast<const float *>(in), in_pitch,
                                                        ncols, out, out_pitch, coef);
  return cuda_status(cudaGetLastError());
}

extern "C" int dd_boxcar_workspace_bytes(int32_t nrows, int64_t ncols, int64_t *bytes) {
  if (!bytes) return DD_ERR_ARG;
  if (nrows < 1 || ncols < 1 || ncols > INT32_MAX) return DD_ERR_SIZE;
  *bytes = box_workspace(nrows, ncols);
  return DD_OK;
}

extern "C" int dd_boxcar_detect(const void *rows, int64_t pitch, int32_t rows_type, int32_t nrows,
                                int64_t ncols, const double *mean, const double *sigma,
                                int32_t nwidths, float nsigma, void *workspace,
                                int64_t workspace_bytes, dd_pulse *pulses, int64_t capacity,
                                int64_t *count, void *stream) {
  if (rows_type != DD_ROWS_I32 && rows_type != DD_ROWS_F32) return DD_ERR_DTYPE;
  if (!rows || !count || !workspace || capacity < 0 || (capacity > 0 && !pulses)) return DD_ERR_ARG;
  if (nrows < 1 || ncols < 1 || ncols > INT32_MAX) return DD_ERR_SIZE;
  if (nwidths < 1 || nwidths > kMaxWidths || !std::isfinite(nsigma) || pitch < ncols)
    return DD_ERR_ARG;
  if (box_tiles(ncols) * nrows > INT32_MAX) return DD_ERR_SIZE;
  if (workspace_bytes < box_workspace(nrows, ncols) ||
      reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
    return DD_ERR_ARG;
  *count = 0;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (rows_type == DD_ROWS_I32)
    return launch_boxcar<int32_t, long long>(static_cast<const int32_t *>(rows), pitch, nrows, ncols,
                                             mean, sigma, nwidths, nsigma, ws, pulses, capacity,
                                             count, s);
  return launch_boxcar<float, float>(static_cast<const float *>(rows), pitch, nrows, ncols, mean,
                                     sigma, nwidths, nsigma, ws, pulses, capacity, count, s);
}
