// Measured FMA throughput of the device: the denominator of the assembly kernels' roofline.
//
// The assembly is bound by the FP64 pipe, whose rate the measured peaks do not give.  This
// kernel keeps every FP64 (or FP32) FMA unit busy: each thread runs 8 independent FMA chains
// (x <- x * a + b, |a| < 1 so nothing overflows) for a fixed number of iterations, the grid is a
// multiple of the SM count with enough warps per SM to hide the FMA latency, and the chains' sum is
// stored so that nothing can be removed.  Flops = 2 per FMA.
#include <algorithm>

#include "bp_internal.cuh"

namespace {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_rate(int iters, T a, T b, T* __restrict__ out) {
  T x[PEAK_CHAINS];
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) s += x[k];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

template <class T>
int fma_rate(int device, double* tflops, cudaStream_t s) {
  int nsm = 0;
  BP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
  const int blocks = nsm * 8;  // 64 warps per SM
  const int iters = std::is_same<T, double>::value ? 4096 : 65536;
  T* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * PEAK_THREADS * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return BP_ENOMEM;
  }
  struct Free {
    T* p;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Free() {
      cudaFree(p);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } guard{out};
  BP_CUDA_TRY(cudaEventCreate(&guard.e0));
  BP_CUDA_TRY(cudaEventCreate(&guard.e1));
  const T a = (T)0.999999, b = (T)1e-6;
  k_fma_rate<T><<<blocks, PEAK_THREADS, 0, s>>>(iters, a, b, out);  // warm-up (clocks up, code loaded)
  BP_CUDA_TRY(cudaGetLastError());
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    BP_CUDA_TRY(cudaEventRecord(guard.e0, s));
    k_fma_rate<T><<<blocks, PEAK_THREADS, 0, s>>>(iters, a, b, out);
    BP_CUDA_TRY(cudaEventRecord(guard.e1, s));
    BP_CUDA_TRY(cudaEventSynchronize(guard.e1));
    float ms = 0.f;
    BP_CUDA_TRY(cudaEventElapsedTime(&ms, guard.e0, guard.e1));
    best = std::min(best, ms);
  }
  const double flops = 2.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return BP_OK;
}

}  // namespace

extern "C" int bp_measure_fma_peak(int precision, double* tflops, void* stream) {
  if (!tflops || (precision != BP_F64 && precision != BP_F32)) return BP_EINVAL;
  int device = 0;
  BP_CUDA_TRY(cudaGetDevice(&device));
  cudaStream_t s = (cudaStream_t)stream;
  return precision == BP_F64 ? fma_rate<double>(device, tflops, s) : fma_rate<float>(device, tflops, s);
}
