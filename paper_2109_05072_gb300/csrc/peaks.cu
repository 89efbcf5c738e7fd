// Arithmetic-throughput measurement (no counterpart in the paper): the rate at which this GPU
// retires FP64 FMAs, FP32 FMAs and packed two-lane FP32 FMAs (fma.rn.f32x2), so that the roofline
// of each operator is stated against a peak measured on the same GPU, in the same process, at the
// clock it runs at; and the rate of the packed compensated sums of the double-float operator.
//
// Every thread runs 8 independent FMA chains x <- x * b + c (b slightly below 1, so each chain
// converges to c / (1 - b) and stays finite); the grid fills every SM with 64 warps.  Thread 0 of
// block 0 reads clock64 and the global timer around its loop, which gives the SM clock during
// the measurement.  The result is written only under a condition the compiler cannot decide (a
// NaN compare), so the chains are not removed.
#include <algorithm>

#include "internal.h"

namespace ceedgb {

__device__ double g_peak_sink;  // external linkage: the conditional store below cannot be dropped
static __device__ unsigned long long g_peak_clock[2];  // SM cycles and nanoseconds of block 0's loop

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(long long iters, T b, T c, double never) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  unsigned long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    t0 = global_ns();
    c0 = clock64();
  }
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = x[k] * b + c;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long c1 = clock64(), t1 = global_ns();
    g_peak_clock[0] = c1 - c0;
    g_peak_clock[1] = t1 - t0;
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += (double)x[k];
  if (s == never) g_peak_sink = s;
}

// The same chains with two FP32 lanes per instruction (PTX fma.rn.f32x2 on sm_100 and later).
__global__ void __launch_bounds__(256) fma_chain_f32x2_kernel(long long iters, float b, float c, double never) {
  unsigned long long x[8], bb, cc;
  asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
  asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float lo = (float)(threadIdx.x + k), hi = (float)(threadIdx.x + k + 8);
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(lo), "f"(hi));
  }
  unsigned long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    t0 = global_ns();
    c0 = clock64();
  }
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(bb), "l"(cc));
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long c1 = clock64(), t1 = global_ns();
    g_peak_clock[0] = c1 - c0;
    g_peak_clock[1] = t1 - t0;
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
    s += (double)lo + (double)hi;
  }
  if (s == never) g_peak_sink = s;
}

// Compensated (Dot2) sums in packed two-lane form, as the double-float operator runs them: every
// thread advances 4 independent accumulators, each step one acc2_mac (a TwoProduct with its cross
// terms and a TwoSum: 12 packed instructions, 24 FP32 lane operations) that depends on the step
// before.  Launched at the double-float operator's occupancy (16 warps per SM) or at the maximum
// (64), it measures how fast the dependent compensated arithmetic itself can retire.
__global__ void __launch_bounds__(256) dot2_chain_kernel(long long iters, float mh, float ml, float vh, float vl,
                                                         double never) {
  const float2 MH = make_float2(mh, -mh), ML = make_float2(ml, -ml), VH = make_float2(vh, vh * 0.5f);
  const float2 VL = make_float2(vl, vl * 0.5f);
  DFAcc2 A[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    A[k].s = make_float2((float)(threadIdx.x + k), (float)(k + 1));
    A[k].c = make_float2(0.f, 0.f);
  }
  unsigned long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    t0 = global_ns();
    c0 = clock64();
  }
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc2_mac(A[k], MH, ML, VH, VL);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long c1 = clock64(), t1 = global_ns();
    g_peak_clock[0] = c1 - c0;
    g_peak_clock[1] = t1 - t0;
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += (double)A[k].s.x + (double)A[k].s.y + (double)A[k].c.x + (double)A[k].c.y;
  if (s == never) g_peak_sink = s;
}

}  // namespace ceedgb

using namespace ceedgb;

extern "C" int ceed_fma_throughput(int kind, double *tflops, double *fma_per_clk_sm, double *sm_mhz, void *stream) {
  if (kind < 0 || kind > 4 || !tflops)
    return fail(CEED_ERR_INVALID, "kind must be 0 (FP64), 1 (FP32), 2 (FP32x2), 3 or 4 (Dot2 chains)");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  CEED_CUDA_CHECK(cudaGetDevice(&dev));
  CEED_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // 8 blocks x 256 threads = 64 warps per SM (the maximum); kind 3: 2 blocks = 16 warps per SM
  const unsigned grid = (unsigned)nsm * (kind == 3 ? 2 : 8);
  const int threads = 256;
  // about 40-80 ms per run at GB300 rates: FP64 ~2 FMA/clk/SM, FP32 128 lanes/clk/SM
  const long long iters = kind == 0 ? 2000 : kind >= 3 ? 8000 : 80000;
  // operations per thread: FMAs for the FMA chains (two lanes for kind 2), FP32 lane operations for
  // the Dot2 chains (32 steps of 24 per iteration)
  const double fma_per_thread = kind >= 3 ? (double)iters * 32.0 * 24.0 : (double)iters * 64.0 * (kind == 2 ? 2.0 : 1.0);
  const double never = __builtin_nan("");
  cudaEvent_t e0, e1;
  CEED_CUDA_CHECK(cudaEventCreate(&e0));
  CEED_CUDA_CHECK(cudaEventCreate(&e1));
  auto launch = [&]() {
    if (kind == 0) fma_chain_kernel<double><<<grid, threads, 0, s>>>(iters, 0.9999999, 1e-7, never);
    else if (kind == 1) fma_chain_kernel<float><<<grid, threads, 0, s>>>(iters, 0.99999f, 1e-5f, never);
    else if (kind == 2) fma_chain_f32x2_kernel<<<grid, threads, 0, s>>>(iters, 0.99999f, 1e-5f, never);
    else dot2_chain_kernel<<<grid, threads, 0, s>>>(iters, 0.7071068f, 1.2e-8f, 1.0e-3f, 3.1e-11f, never);
  };
  launch();  // warm-up (clocks ramp, code loaded)
  float best = 1e30f;
  unsigned long long clk[2] = {0, 0};
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    CEED_CUDA_CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      CEED_CUDA_CHECK(cudaMemcpyFromSymbol(clk, g_peak_clock, sizeof(clk)));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CEED_CUDA_CHECK(cudaGetLastError());
  const double fmas = fma_per_thread * threads * (double)grid;
  *tflops = (kind >= 3 ? 1.0 : 2.0) * fmas / (best * 1e-3) / 1e12;
  const double mhz = clk[1] > 0 ? (double)clk[0] / (double)clk[1] * 1e3 : 0.0;
  if (sm_mhz) *sm_mhz = mhz;
  if (fma_per_clk_sm) *fma_per_clk_sm = mhz > 0 ? fmas / (best * 1e-3) / (mhz * 1e6) / nsm : 0.0;
  return CEED_OK;
}
