// Pipe-throughput microbenchmarks: results per SM per clock, for the roofline
// denominators of the pair kernels (FP32 FMA, packed FP32 FMA, SFU functions,
// FP64 FMA, FP32<->FP64 conversions).
//
// Each kernel runs CH independent dependency chains per thread for ITER
// iterations on a grid that is fully co-resident (SMs x occupancy CTAs), and
// every CTA times itself with clock64(), so the rate does not depend on the
// clock frequency.  Results are written to a device array and read on the host.
#include <cuda_runtime.h>
#include <stdint.h>

#include "md_peaks.h"

namespace {

constexpr int NT = 256;
constexpr int CH = 8;

__device__ __forceinline__ float sfu_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sfu_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sfu_sin(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sfu_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sfu_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float cvt_roundtrip(float x) {
  double d;
  float r;
  asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(x));
  asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(r) : "d"(d));
  return r;
}

// OP_MIX: half the chains packed FFMA2, half scalar FFMA (does the second FMA
// pipe add throughput next to packed instructions?)
enum Op { OP_FFMA = 0, OP_FFMA2, OP_RSQ, OP_RCP, OP_SIN, OP_LG2EX2, OP_DFMA, OP_CVT, OP_MIX, OP_COUNT };

template <int OP>
__global__ void __launch_bounds__(NT) pipe_kernel(const float *in, float *out, long long *cycles, int iters) {
  const float x = in[0], y = in[1];
  float a[CH];
  float2 b[CH];
  double d[CH];
#pragma unroll
  for (int c = 0; c < CH; c++) {
    a[c] = in[2] + c * 1e-3f + threadIdx.x * 1e-6f;
    b[c] = make_float2(a[c], a[c] + 0.5f);
    d[c] = (double)a[c];
  }
  const double xd = (double)x, yd = (double)y;
  const float2 x2 = make_float2(x, x), y2 = make_float2(y, y);
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < CH; c++) {
      if (OP == OP_FFMA) a[c] = fmaf(a[c], x, y);
      if (OP == OP_FFMA2) b[c] = __ffma2_rn(b[c], x2, y2);
      if (OP == OP_RSQ) a[c] = sfu_rsqrt(a[c]);
      if (OP == OP_RCP) a[c] = sfu_rcp(a[c] + y);  // the add keeps rcp(rcp(x)) from folding
      if (OP == OP_SIN) a[c] = sfu_sin(a[c]);
      if (OP == OP_LG2EX2) a[c] = sfu_ex2(sfu_lg2(a[c]));
      if (OP == OP_DFMA) d[c] = fma(d[c], xd, yd);
      if (OP == OP_CVT) a[c] = cvt_roundtrip(a[c]);
      if (OP == OP_MIX) {
        if (c < CH / 2) b[c] = __ffma2_rn(b[c], x2, y2);
        else a[c] = fmaf(a[c], x, y);
      }
    }
  }
  __syncthreads();
  long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CH; c++) s += a[c] + b[c].x + b[c].y + (float)d[c];
  out[blockIdx.x * NT + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// SFU / FMA operations counted per chain-iteration (the rcp chain's add is not counted)
const double kOpsPerIter[OP_COUNT] = {1, 2, 1, 1, 1, 2, 1, 2, 1.5};

template <int OP>
int run(int nsm, const float *din, float *dout, long long *dcyc, long long *hcyc, int iters, double *rate,
        double *mhz) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pipe_kernel<OP>, NT, 0);
  if (occ < 1) return 1;
  if (occ > 8) occ = 8;
  const int grid = nsm * occ;
  pipe_kernel<OP><<<grid, NT>>>(din, dout, dcyc, 16);  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  pipe_kernel<OP><<<grid, NT>>>(din, dout, dcyc, iters);
  cudaEventRecord(e1);
  if (cudaEventSynchronize(e1) != cudaSuccess) return 2;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaMemcpy(hcyc, dcyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  double mean = 0.0, mx = 0.0;
  for (int i = 0; i < grid; i++) {
    mean += (double)hcyc[i];
    if ((double)hcyc[i] > mx) mx = (double)hcyc[i];
  }
  mean /= grid;
  const double ops_per_cta = (double)NT * CH * iters * kOpsPerIter[OP];
  *rate = ops_per_cta * occ / mx;  // per SM per clock (slowest CTA bounds the SM)
  *mhz = mx / (ms * 1e-3) / 1e6;
  return 0;
}

}  // namespace

extern "C" int mdp_pipe_rates(double *out, int nout) {
  if (!out || nout < 2 * OP_COUNT + 1) return 1;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  float hin[3] = {0.999f, 1e-4f, 0.5f};
  float *din = nullptr, *dout = nullptr;
  long long *dcyc = nullptr;
  const int maxgrid = nsm * 8;
  long long *hcyc = new long long[maxgrid];
  int rc = 0;
  if (cudaMalloc(&din, sizeof hin) != cudaSuccess || cudaMalloc(&dout, sizeof(float) * NT * maxgrid) != cudaSuccess ||
      cudaMalloc(&dcyc, sizeof(long long) * maxgrid) != cudaSuccess)
    rc = 3;
  if (!rc) cudaMemcpy(din, hin, sizeof hin, cudaMemcpyHostToDevice);
  out[0] = nsm;
  for (int op = 0; op < OP_COUNT && !rc; op++) {
    double r = 0.0, mhz = 0.0;
    const int iters = (op == OP_DFMA || op == OP_CVT) ? 256 : 4096;
    switch (op) {
    case OP_FFMA: rc = run<OP_FFMA>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    case OP_FFMA2: rc = run<OP_FFMA2>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    case OP_RSQ: rc = run<OP_RSQ>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    case OP_RCP: rc = run<OP_RCP>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    case OP_SIN: rc = run<OP_SIN>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    case OP_LG2EX2: rc = run<OP_LG2EX2>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    case OP_DFMA: rc = run<OP_DFMA>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    case OP_CVT: rc = run<OP_CVT>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    case OP_MIX: rc = run<OP_MIX>(nsm, din, dout, dcyc, hcyc, iters, &r, &mhz); break;
    }
    out[1 + 2 * op] = r;
    out[2 + 2 * op] = mhz;
  }
  cudaFree(din);
  cudaFree(dout);
  cudaFree(dcyc);
  delete[] hcyc;
  return rc;
}
