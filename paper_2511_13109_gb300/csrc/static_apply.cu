// Allocation-free Stokes operator apply for small grids.
//
// Some callers cannot allocate device memory themselves: code embedded in a
// host application whose device memory is owned by another allocator (a
// caching allocator or a fixed pool they must not bypass), or code in a loop
// where an allocation's latency or possible failure is not acceptable.  For
// them agca_stokes_apply_static computes y = K x on the finest grid without a
// context, a workspace or any allocation: the two fine-grid scratch fields the
// operator needs (the prolongated pressure P p and the divergence B_f u) live
// in a fixed file-scope device array that every GPU loading this library
// holds until the process exits.
//
// Limit: N <= kStaticMaxN pressure cubes per axis (the scratch holds
// 2 * (2N+1)^3 doubles, 4.4 MB at the limit).
#include <mutex>

#include "agca_internal.cuh"

namespace {

constexpr int kStaticMaxN = 32;
constexpr int64_t kStaticMaxV = (int64_t)(2 * kStaticMaxN + 1) * (2 * kStaticMaxN + 1) * (2 * kStaticMaxN + 1);

// [0, V): fine-grid pressure P p; [kStaticMaxV, kStaticMaxV + V): B_f u
static __device__ __align__(256) double g_stokes_scratch[2 * kStaticMaxV];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_stokes_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" agca_status agca_stokes_apply_static(int N, const double* eta_dev, const double* x_dev, double* y_dev,
                                                void* cuda_stream) {
  using namespace agca;
  if (N < 1 || N > kStaticMaxN) return AGCA_EINVAL;
  if (!eta_dev || !x_dev || !y_dev) return AGCA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return AGCA_ECUDA;
  const int n = 2 * N;
  const int64_t V = nverts(n);
  double* qfine = scratch;
  double* sfine = scratch + kStaticMaxV;
  // the same three launches as agca_stokes_apply, with the scratch above;
  // every scratch entry used is written before it is read
  if (launch_prolong<double>(n, 1, false, false, x_dev + 3 * V, qfine, s) != cudaSuccess) return AGCA_ECUDA;
  LevelOp<double> op{};
  op.n = n;
  op.h6 = 1.0 / (6.0 * n);
  op.hq = 1.0 / (6.0 * (double)n * n);
  op.coef = eta_dev;
  StencilArgs<double> a{};
  a.x = x_dev;
  a.q = qfine;
  a.out = y_dev;
  a.out2 = sfine;
  if (launch_stencil<double, double>(ST_STOKES, op, a, s) != cudaSuccess) return AGCA_ECUDA;
  if (launch_restrict<double>(n, 1, false, -1.0, sfine, y_dev + 3 * V, s) != cudaSuccess) return AGCA_ECUDA;
  return AGCA_OK;
}
