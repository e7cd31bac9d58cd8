// Throughput probes of the two units the phasor sums run on (Section 5.1:
// the paper measures its hardware's FP32 peak and bounds each kernel by it).
//
// fma_probe_kernel: every thread runs kChains independent chains of packed
// f32x2 fused multiply-adds, so the FMA pipe, not a dependency, sets the
// rate.  sincos_probe_kernel: every thread evaluates __sincosf on kChains
// independent arguments per iteration; each evaluation is two MUFU
// operations (sine, cosine) plus a few FP32 adds, so the sine unit sets the
// rate.  Each kernel writes one value per thread that depends on every
// operation, so nothing is optimised away.
#include "kernels_common.cuh"

namespace idg {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float* out, int iters, float m, float c) {
  float2 acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = make_float2(float(threadIdx.x + k), float(blockIdx.x - k));
  const float2 M = make_float2(m, m), Cc = make_float2(c, c);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) acc[k] = ffma2(acc[k], M, Cc);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k].x + acc[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) sincos_probe_kernel(float* out, int iters, float step) {
  float x[kChains], acc = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * float(threadIdx.x + 37 * k);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float s, c;
      __sincosf(x[k], &s, &c);
      acc += s * c;
      x[k] += step;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

// Runs both probes on `stream` with every SM filled and returns, from CUDA
// events around each launch, FMA operations per second (one f32x2 FMA counts
// as two) and __sincosf evaluations per second.
int run_peak_probes(void* stream, double* fma_per_s, double* sincos_per_s, float* scratch, int n_blocks) {
  cudaStream_t st = cudaStream_t(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int fma_iters = 4096, sin_iters = 2048;
  float ms_fma = 0.f, ms_sin = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first pass warms up
    cudaEventRecord(e0, st);
    fma_probe_kernel<<<n_blocks, kProbeThreads, 0, st>>>(scratch, fma_iters, 0.999f, 1e-4f);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_fma, e0, e1);
    if (e != cudaSuccess) break;
    cudaEventRecord(e0, st);
    sincos_probe_kernel<<<n_blocks, kProbeThreads, 0, st>>>(scratch, sin_iters, 1.1e-3f);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_sin, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return int(e);
  const double threads = double(n_blocks) * kProbeThreads;
  *fma_per_s = threads * fma_iters * 8.0 * kChains * 2.0 / (double(ms_fma) * 1e-3);
  *sincos_per_s = threads * sin_iters * double(kChains) / (double(ms_sin) * 1e-3);
  return 0;
}

}  // namespace idg

using namespace idg;

extern "C" idg_status idg_peak_rates(void* cuda_stream, double* fma_per_s, double* sincos_per_s) {
  if (!fma_per_s || !sincos_per_s) return plan_set_error(nullptr, IDG_ERR_INVALID_ARG, "idg_peak_rates: NULL output");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_blocks = 8 * sms;  // 8 blocks of 256 threads per SM: 64 warps, a full SM
  float* scratch = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), sizeof(float) * n_blocks * kProbeThreads,
                                            cudaStream_t(cuda_stream));
  int r = int(e);
  if (r == 0) r = run_peak_probes(cuda_stream, fma_per_s, sincos_per_s, scratch, n_blocks);
  if (scratch) {
    cudaFreeAsync(scratch, cudaStream_t(cuda_stream));
    cudaStreamSynchronize(cudaStream_t(cuda_stream));
  }
  if (r) {
    const std::string msg = std::string("idg_peak_rates: ") + cudaGetErrorString(cudaError_t(r));
    return plan_set_error(nullptr, r == int(cudaErrorMemoryAllocation) ? IDG_ERR_OOM : IDG_ERR_CUDA, msg.c_str());
  }
  return IDG_OK;
}
