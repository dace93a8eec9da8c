// Arithmetic-throughput probe: FP64 and FP32 FMA / add instruction rates of
// the device, from long dependent-chain loops (8 independent chains per
// thread, 8 blocks of 256 threads per SM), timed with CUDA events after two
// warm-up launches.  Prints one line per precision; used to bound the FP64
// stencil, whose roofline is min(HBM, FP64 ALU).
#include <cuda_runtime.h>

#include <cstdio>

template <typename T>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
__global__ void add_loop(T* out, int iters, T a) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 += a; x1 -= a; x2 += a; x3 -= a; x4 += a; x5 -= a; x6 += a; x7 -= a;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

#define CHECK(x)                                                              \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));           \
      return -1.0;                                                            \
    }                                                                         \
  } while (0)

// instructions per second of one kind
template <typename T, bool FMA>
double rate(int sms, int iters) {
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  CHECK(cudaMalloc(&out, sizeof(T) * blocks * threads));
  cudaEvent_t e0, e1;
  CHECK(cudaEventCreate(&e0));
  CHECK(cudaEventCreate(&e1));
  for (int rep = 0; rep < 3; ++rep) {
    if (rep == 2) CHECK(cudaEventRecord(e0));
    if (FMA)
      fma_loop<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-4);
    else
      add_loop<T><<<blocks, threads>>>(out, iters, (T)1e-4);
    CHECK(cudaGetLastError());
  }
  CHECK(cudaEventRecord(e1));
  CHECK(cudaEventSynchronize(e1));
  float ms = 0.0f;
  CHECK(cudaEventElapsedTime(&ms, e0, e1));
  CHECK(cudaFree(out));
  return (double)blocks * threads * iters * 16 * 8 / (ms * 1e-3);
}

int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) return 1;
  int clk = 0;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  std::printf("device %s sms %d cc %d.%d max_sm_clock_mhz %d\n", p.name, p.multiProcessorCount, p.major, p.minor,
              clk / 1000);
  const int sms = p.multiProcessorCount;
  const double d_fma = rate<double, true>(sms, 64), d_add = rate<double, false>(sms, 64);
  const double f_fma = rate<float, true>(sms, 1024), f_add = rate<float, false>(sms, 1024);
  if (d_fma <= 0 || d_add <= 0 || f_fma <= 0 || f_add <= 0) return 1;
  std::printf("fp64 fma_tinstr_s %.4f tflop_s %.4f add_tinstr_s %.4f\n", d_fma * 1e-12, 2 * d_fma * 1e-12,
              d_add * 1e-12);
  std::printf("fp32 fma_tinstr_s %.4f tflop_s %.4f add_tinstr_s %.4f\n", f_fma * 1e-12, 2 * f_fma * 1e-12,
              f_add * 1e-12);
  return 0;
}
