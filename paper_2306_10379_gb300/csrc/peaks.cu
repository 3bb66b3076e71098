// Arithmetic throughput of the float64 and float32 FMA pipes, the two
// denominators of the df64 design (the n x p x p work is placed on the
// float32 pipes and the tensor cores because the float64 pipe of this GPU is
// narrow). Each thread runs 8 independent multiply-add chains, so the pipes,
// not the dependency latency, bound the rate; every thread writes one sum so
// that no chain is dead code. 2 flops per multiply-add.
#include <cuda_runtime.h>

#include "common.cuh"

namespace gsi {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) fma_chains_kernel(T* out, int iters, T a, T b) {
  T x[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = fma(x[k], a, b);
  T s = 0;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += x[k];
  out[(size_t)blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

template <typename T>
static gsi_status time_chains(int blocks, int iters, T* out, cudaStream_t st, double* tflops) {
  cudaEvent_t e0, e1;
  GSI_CUDA_TRY(cudaEventCreate(&e0));
  GSI_CUDA_TRY(cudaEventCreate(&e1));
  const T a = (T)0.999999, b = (T)1e-7;  // x stays bounded: x -> b / (1 - a)
  fma_chains_kernel<T><<<blocks, PK_THREADS, 0, st>>>(out, iters / 8, a, b);  // warm-up
  GSI_LAUNCH_CHECK();
  float best = 0.f;
  for (int rep = 0; rep < 3; ++rep) {
    GSI_CUDA_TRY(cudaEventRecord(e0, st));
    fma_chains_kernel<T><<<blocks, PK_THREADS, 0, st>>>(out, iters, a, b);
    GSI_LAUNCH_CHECK();
    GSI_CUDA_TRY(cudaEventRecord(e1, st));
    GSI_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    GSI_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (rep == 0 || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * PK_CHAINS * (double)iters * blocks * PK_THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return GSI_OK;
}

}  // namespace gsi

using namespace gsi;

extern "C" gsi_status gsi_measure_fma_peaks(double* out, void* stream) {
  if (!out) return GSI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = sm_count() * 8;
  void* buf = nullptr;
  GSI_CUDA_TRY(cudaMallocAsync(&buf, (size_t)blocks * PK_THREADS * sizeof(double), st));
  // about 50 ms per timed launch at the expected rates
  gsi_status s = time_chains<double>(blocks, 8192, (double*)buf, st, &out[0]);
  if (s == GSI_OK) s = time_chains<float>(blocks, 393216, (float*)buf, st, &out[1]);
  cudaFreeAsync(buf, st);
  cudaStreamSynchronize(st);
  return s;
}
