// dd_peak.cu -- throughput probes of the SM's 32-bit add pipes, used as the
// denominator of the dedispersion kernel's roofline (dd_peak.h).
//
// Each probe runs, in every thread, eight independent dependency chains of
// one instruction form, so that issue rate rather than latency bounds it.
// Cycles are read with clock64() inside the kernel (a per-SM counter), and
// each SM's busy span runs from the earliest start to the latest end of the
// blocks it ran, so the result in operations per clock per SM does not depend
// on the clock the GPU ran at nor on blocks starting at different times.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_peak.h"

namespace {

constexpr int kThreads = 256;
constexpr int kIters = 2048;
constexpr int kChains = 8;

template <int KIND>
__device__ __forceinline__ void step(uint32_t (&a)[kChains], uint32_t b, uint32_t c) {
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    if constexpr (KIND == DD_PEAK_FADD) {
      asm volatile("add.rn.f32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
    } else if constexpr (KIND == DD_PEAK_IADD) {
      asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
    } else if constexpr (KIND == DD_PEAK_IADD3) {
      asm volatile("{\n\t.reg .u32 t;\n\tadd.u32 t, %0, %1;\n\tadd.u32 %0, t, %2;\n\t}"
                   : "+r"(a[i]) : "r"(b), "r"(c));
    } else if constexpr (KIND == DD_PEAK_IMAD) {
      asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
    } else if constexpr (KIND == DD_PEAK_LOP3) {
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[i]) : "r"(b), "r"(c));
    } else if constexpr (KIND == DD_PEAK_PRMT) {
      asm volatile("prmt.b32 %0, %0, %1, 0x4321;" : "+r"(a[i]) : "r"(b));
    } else if constexpr (KIND == DD_PEAK_HADD2) {
      asm volatile("add.rn.f16x2 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
    } else if constexpr (KIND == DD_PEAK_FADD_F16) {
      asm volatile("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %1;\n\t"
                   "add.rn.f32.f16 %0, lo, %0;\n\t}"
                   : "+r"(a[i]) : "r"(b));
    } else if constexpr (KIND == DD_PEAK_PRMT_IADD) {
      asm volatile("{\n\t.reg .u32 t;\n\tprmt.b32 t, %1, 0, 0x4140;\n\tadd.u32 %0, %0, t;\n\t}"
                   : "+r"(a[i]) : "r"(b ^ a[(i + 1) % kChains]));
    } else if constexpr (KIND == DD_PEAK_LOP3_IADD) {
      asm volatile("{\n\t.reg .u32 t;\n\tand.b32 t, %1, 0x00FF00FF;\n\tadd.u32 %0, %0, t;\n\t}"
                   : "+r"(a[i]) : "r"(b ^ a[(i + 1) % kChains]));
    }
  }
}

// Operations per step() call per chain (adds counted as one each; the
// three-operand add counts two; the mixed prmt/and + add counts one add).
template <int KIND>
constexpr int ops_per_chain() {
  return (KIND == DD_PEAK_IADD3) ? 2 : (KIND == DD_PEAK_FADD2 ? 2 : 1);
}

__device__ __forceinline__ uint32_t sm_id() {
  uint32_t id;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
  return id;
}

// cycles[3 * block .. +3) = {SM id, start, end}
template <int KIND>
__global__ void __launch_bounds__(kThreads) peak_kernel(uint32_t *sink, long long *cycles) {
  uint32_t a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 7 + i;
  const uint32_t b = blockIdx.x | 1u, c = threadIdx.x | 3u;
  __syncthreads();
  const long long t0 = clock64();
  if constexpr (KIND == DD_PEAK_FADD2) {
    unsigned long long v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = (static_cast<unsigned long long>(a[i]) << 32) | a[i];
    const unsigned long long w = (static_cast<unsigned long long>(b) << 32) | c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(v[i]) : "l"(w));
    }
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = static_cast<uint32_t>(v[i] ^ (v[i] >> 32));
  } else {
    for (int it = 0; it < kIters; ++it) step<KIND>(a, b, c);
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) x ^= a[i];
  if (x == 0x9e3779b9u) sink[blockIdx.x] = x;  // keeps the chains live
  if (threadIdx.x == 0) {
    cycles[3 * blockIdx.x] = sm_id();
    cycles[3 * blockIdx.x + 1] = t0;
    cycles[3 * blockIdx.x + 2] = t1;
  }
}

template <int KIND>
int run(int device, double *ops_per_s, double *ops_per_clk_sm) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return DD_PEAK_ERR;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, peak_kernel<KIND>, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int blocks = sms * per_sm;
  uint32_t *sink = nullptr;
  long long *cyc = nullptr;
  if (cudaMalloc(&sink, blocks * sizeof(uint32_t)) != cudaSuccess) return DD_PEAK_ERR;
  if (cudaMalloc(&cyc, 3 * blocks * sizeof(long long)) != cudaSuccess) {
    cudaFree(sink);
    return DD_PEAK_ERR;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  peak_kernel<KIND><<<blocks, kThreads>>>(sink, cyc);  // warm-up
  cudaEventRecord(e0);
  constexpr int kReps = 5;
  for (int r = 0; r < kReps; ++r) peak_kernel<KIND><<<blocks, kThreads>>>(sink, cyc);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  // busy span of each SM over the last launch: earliest start to latest end
  long long *h = new long long[3 * blocks];
  cudaMemcpy(h, cyc, 3 * blocks * sizeof(long long), cudaMemcpyDeviceToHost);
  long long *lo = new long long[sms], *hi = new long long[sms];
  for (int i = 0; i < sms; ++i) lo[i] = -1, hi[i] = -1;
  for (int b = 0; b < blocks; ++b) {
    const long long id = h[3 * b], t0 = h[3 * b + 1], t1 = h[3 * b + 2];
    if (id < 0 || id >= sms) continue;
    if (lo[id] < 0 || t0 < lo[id]) lo[id] = t0;
    if (hi[id] < 0 || t1 > hi[id]) hi[id] = t1;
  }
  long long mx = 0;
  for (int i = 0; i < sms; ++i)
    if (lo[i] >= 0 && hi[i] - lo[i] > mx) mx = hi[i] - lo[i];
  delete[] h;
  delete[] lo;
  delete[] hi;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(cyc);
  if (err != cudaSuccess || ms <= 0.f || mx <= 0) return DD_PEAK_ERR;
  const double ops = static_cast<double>(blocks) * kThreads * kIters * kChains * ops_per_chain<KIND>();
  *ops_per_s = ops * kReps / (ms * 1e-3);
  *ops_per_clk_sm = ops / sms / static_cast<double>(mx);
  return 0;
}

}  // namespace

extern "C" int dd_measure_add_peak(int32_t kind, int32_t device, double *ops_per_s,
                                   double *ops_per_clk_per_sm) {
  if (!ops_per_s || !ops_per_clk_per_sm) return DD_PEAK_ERR;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return DD_PEAK_ERR;
  int st = DD_PEAK_ERR;
  switch (kind) {
    case DD_PEAK_FADD: st = run<DD_PEAK_FADD>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_FADD2: st = run<DD_PEAK_FADD2>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_IADD: st = run<DD_PEAK_IADD>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_IADD3: st = run<DD_PEAK_IADD3>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_IMAD: st = run<DD_PEAK_IMAD>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_LOP3: st = run<DD_PEAK_LOP3>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_PRMT: st = run<DD_PEAK_PRMT>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_HADD2: st = run<DD_PEAK_HADD2>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_FADD_F16: st = run<DD_PEAK_FADD_F16>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_PRMT_IADD: st = run<DD_PEAK_PRMT_IADD>(device, ops_per_s, ops_per_clk_per_sm); break;
    case DD_PEAK_LOP3_IADD: st = run<DD_PEAK_LOP3_IADD>(device, ops_per_s, ops_per_clk_per_sm); break;
    default: break;
  }
  cudaSetDevice(prev);
  return st;
}
