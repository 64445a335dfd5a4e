// Arithmetic-throughput probe: the measured FP64 / FP32 fused multiply-add
// rates that serve as the ALU roofline of the stencils (the Brillouin matvec
// runs on CUDA cores, not tensor cores, because SU(3) x spinor is not a dense
// contraction).  Every thread advances eight independent FMA chains so that
// the FMA latency is hidden; the grid is a multiple of the SM count; the
// result is folded into one value that is stored only under a condition the
// compiler cannot decide, so no chain is optimised away.
#include "internal.cuh"

#include <algorithm>

namespace bri {
namespace {

constexpr int CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T b, T c) {
  T a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  if (s == (T)-1.25) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the paired FP32 pipe (fma.rn.f32x2): two FMAs per instruction
__global__ void __launch_bounds__(256) k_fma2_probe(float* out, int iters, float b, float c) {
  float2 a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = make_float2((threadIdx.x + k) * 1e-3f, (threadIdx.x - k) * 1e-3f);
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k].x + a[k].y;
  if (s == -1.25f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace bri

using namespace bri;

extern "C" int bri_fma_probe(int kind, void* stream, double* tflops, double* ms) {
  if (!tflops || !ms || kind < 0 || kind > 2) {
    set_error("bri_fma_probe: kind must be 0 (FP64), 1 (FP32) or 2 (paired FP32) and outputs non-null");
    return BRI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  BRI_CUDA(cudaGetDevice(&dev));
  BRI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;
  const int iters = kind == 0 ? 4096 : 65536;
  void* out = nullptr;
  BRI_CUDA(cudaMallocAsync(&out, sizeof(double) * blocks * threads, s));
  note_device_alloc();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, s);
    if (kind == 0) k_fma_probe<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.999, 1e-4);
    else if (kind == 1) k_fma_probe<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.999f, 1e-4f);
    else k_fma2_probe<<<blocks, threads, 0, s>>>((float*)out, iters / 2, 0.999f, 1e-4f);
    note_launch();
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaFreeAsync(out, s);
      return cuda_fail(e, "bri_fma_probe");
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) best = std::min(best, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  BRI_LAUNCH_CHECK("bri_fma_probe");
  // FMAs: blocks * threads * CHAINS * iters (paired: iters/2 instructions of two FMAs)
  const double fmas = (double)blocks * threads * CHAINS * iters;
  *ms = best;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return BRI_OK;
}
