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
#include <cuda.h>  // driver types only: the two driver calls are resolved at run time

#include <mutex>

#include "agca_internal.cuh"

namespace {

constexpr int kStaticMaxN = 32;
constexpr int64_t kStaticMaxV = (int64_t)(2 * kStaticMaxN + 1) * (2 * kStaticMaxN + 1) * (2 * kStaticMaxN + 1);

// [0, V): fine-grid pressure P p; [kStaticMaxV, kStaticMaxV + V): B_f u
static __device__ __align__(256) double g_stokes_scratch[2 * kStaticMaxV];

// The scratch array's device address belongs to a CUDA context (a module is
// loaded per context), so it is cached per context, keyed by the context's
// process-unique ID: a caller that later works under another context (one it
// created with the driver API, or the primary context re-created after
// cudaDeviceReset) gets a fresh lookup, never a stale address.
constexpr int kMaxContexts = 64;
std::mutex g_mutex;
unsigned long long g_ctx_id[kMaxContexts] = {};
double* g_ctx_scratch[kMaxContexts] = {};
int g_n_ctx = 0;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

cudaError_t resolve_driver_calls() {
  if (g_get_current && g_get_id) return cudaSuccess;
  void* f0 = nullptr;
  void* f1 = nullptr;
  cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = cudaDriverEntryPointSymbolNotFound;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
  if (e != cudaSuccess) return e;
  e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
  if (e != cudaSuccess) return e;
  if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
    return cudaErrorNotSupported;
  g_get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
  g_get_id = reinterpret_cast<CtxGetIdFn>(f1);
  return cudaSuccess;
}

// Device address of the scratch array in the current context (the host-side
// symbol is only a stand-in, not a device address), looked up once per context.
cudaError_t scratch_address(double** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  cudaError_t e = resolve_driver_calls();
  if (e != cudaSuccess) return e;
  CUcontext ctx = nullptr;
  if (g_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
  if (!ctx) {
    // no context current yet: the runtime's lookup makes the device's
    // primary context current, which is the context the address belongs to
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_stokes_scratch);
    if (e != cudaSuccess) return e;
    if (g_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorUnknown;
  }
  unsigned long long id = 0;
  if (g_get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorUnknown;
  for (int i = 0; i < g_n_ctx; ++i) {
    if (g_ctx_id[i] == id) {
      *out = g_ctx_scratch[i];
      return cudaSuccess;
    }
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_stokes_scratch);
  if (e != cudaSuccess) return e;
  // a full table is recycled from its first slot (a lookup is never wrong,
  // only repeated)
  const int slot = g_n_ctx < kMaxContexts ? g_n_ctx++ : (int)(id % kMaxContexts);
  g_ctx_id[slot] = id;
  g_ctx_scratch[slot] = static_cast<double*>(p);
  *out = g_ctx_scratch[slot];
  return cudaSuccess;
}

// true when p is device (or managed) memory that the current device can use
bool on_current_device(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" agca_status agca_stokes_apply_static(int N, const double* eta_dev, const double* x_dev, double* y_dev,
                                                void* cuda_stream) {
  using namespace agca;
  if (N < 1 || N > kStaticMaxN) return AGCA_EINVAL;
  if (!eta_dev || !x_dev || !y_dev) return AGCA_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AGCA_ECUDA;
  if (!on_current_device(eta_dev, dev) || !on_current_device(x_dev, dev) || !on_current_device(y_dev, dev))
    return AGCA_EINVAL;
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
