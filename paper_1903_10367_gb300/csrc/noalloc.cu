// adafac_residual_norm_static: the residual norm sqrt(h^D sum_i r_i^2) of
// r = b - A u for a uniform d-linear operator, computed without allocating
// device memory.
//
// Callers that cannot allocate: a solver service whose device memory is fully
// committed to resident workspaces (any allocation may fail or evict), and
// code that must not pay the device-wide synchronisation cudaFree implies.
// Such callers get a residual check on caller-owned u and b only: the kernels
// keep their per-block partial sums in a file-scope device array instead of a
// workspace.
//
// The scratch array exists once per CUDA context that loads this library.
// Calls that overlap in time in one context -- on different streams or from
// different host threads without ordering -- race on it and may return wrong
// norms; order them on one stream.  Its device address is looked up once per
// context (keyed by the context's id, which a context re-created after
// cudaDeviceReset does not share), so the first call in each context must
// come before any stream capture; under capture a context without a cached
// address is refused.
#include <cuda.h>

#include <mutex>

#include "adafac.h"
#include "common.cuh"

namespace adafac {

namespace {

// partial sums: one per block of kVertsPerBlock vertices
constexpr int kMaxPartials = 4096;
constexpr int kThreads = 256;
constexpr long long kVertsPerBlock = 64LL * kThreads;  // 16384
constexpr int kMaxContexts = 64;

static __device__ __align__(256) double g_partials[kMaxPartials];

// cached device addresses of the scratch array, by context id
struct Cached {
  unsigned long long ctx = 0;
  double* addr = nullptr;
};
std::mutex g_lock;
Cached g_cache[kMaxContexts];
int g_next = 0;

// Partial sums of h^D r^2 over the interior vertices of one block's range,
// r = b - A u with A the assembled uniform stencil of -div(eps grad) on the
// d-linear finite element: the neighbour at offset o with k non-zero
// components shares 2^(D-k) cells with the centre, each contributing
// eps h^(D-2) K_ref(k).  Every partial is written, none accumulated.
template <int D>
__global__ void __launch_bounds__(kThreads)
    k_residual_partials(int n, double eps_hfac, const double* __restrict__ u,
                        const double* __restrict__ b, double hD, double* __restrict__ partials) {
  constexpr int NS = ipow_c(3, D);
  __shared__ double st[NS];
  __shared__ double red[kThreads / 32];
  if (threadIdx.x < NS) {
    int t = threadIdx.x, k = 0;
    for (int j = 0; j < D; ++j) {
      k += (t % 3) != 1;
      t /= 3;
    }
    st[threadIdx.x] = eps_hfac * (double)(1 << (D - k)) * kref<D, double>(k);
  }
  __syncthreads();
  const int np1 = n + 1;
  long long V = 1;
  for (int j = 0; j < D; ++j) V *= np1;
  const long long v0 = blockIdx.x * kVertsPerBlock;
  const long long v1 = v0 + kVertsPerBlock < V ? v0 + kVertsPerBlock : V;
  double acc = 0.0;
  for (long long v = v0 + threadIdx.x; v < v1; v += kThreads) {
    int c[D];
    decode<D>(v, np1, c);
    if (!is_interior<D>(c, n)) continue;
    double Au = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) Au += st[s] * u[v + stencil_offset<D>(s, np1)];
    const double r = b[v] - Au;
    acc += r * r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    partials[blockIdx.x] = t * hD;
  }
}

__global__ void __launch_bounds__(kThreads)
    k_norm_from_partials(const double* __restrict__ partials, int nblocks, double* out) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kThreads) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(red[0]);
}

// Id of the current CUDA context (unique for the life of the process), or 0
// when it cannot be read.  The driver entry points are taken through the
// runtime, so the library needs no link against the driver library.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(fn);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context: looked up
// (cudaGetSymbolAddress, with the context current) the first time a context is
// seen, and refused (nullptr) when that first time falls inside a stream
// capture on `s`.
double* scratch_address(cudaStream_t s) {
  const unsigned long long ctx = current_context_id();
  if (!ctx) return nullptr;
  std::lock_guard<std::mutex> g(g_lock);
  for (const Cached& c : g_cache)
    if (c.ctx == ctx) return c.addr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return nullptr;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
    cudaGetLastError();
    return nullptr;
  }
  Cached& slot = g_cache[g_next];
  g_next = (g_next + 1) % kMaxContexts;
  slot.ctx = ctx;
  slot.addr = static_cast<double*>(p);
  return slot.addr;
}

}  // namespace

}  // namespace adafac

extern "C" adafac_status adafac_residual_norm_static(int dim, int depth, double eps,
                                                     const double* u, const double* b,
                                                     double* norm, void* stream) {
  using namespace adafac;
  if ((dim != 2 && dim != 3) || depth < 1 || !(eps > 0.0) || eps > 1e300 || !u || !b ||
      !norm)
    return ADAFAC_ERR_INVALID_ARG;
  long long n = 1;
  for (int i = 0; i < depth; ++i) {
    n *= 3;
    if (n > (1 << 20)) return ADAFAC_ERR_INVALID_ARG;
  }
  long long V = 1;
  for (int j = 0; j < dim; ++j) V *= n + 1;
  const long long nblocks = (V + kVertsPerBlock - 1) / kVertsPerBlock;
  if (nblocks > kMaxPartials) return ADAFAC_ERR_INVALID_ARG;  // beyond the scratch
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* partials = scratch_address(s);
  if (!partials) return ADAFAC_ERR_CUDA;
  const double h = 1.0 / (double)n;
  const double hfac = dim == 2 ? 1.0 : h;
  const double hD = dim == 2 ? h * h : h * h * h;
  if (dim == 2)
    k_residual_partials<2><<<(int)nblocks, kThreads, 0, s>>>((int)n, eps * hfac, u, b, hD,
                                                              partials);
  else
    k_residual_partials<3><<<(int)nblocks, kThreads, 0, s>>>((int)n, eps * hfac, u, b, hD,
                                                              partials);
  k_norm_from_partials<<<1, kThreads, 0, s>>>(partials, (int)nblocks, norm);
  return cudaGetLastError() == cudaSuccess ? ADAFAC_OK : ADAFAC_ERR_CUDA;
}
