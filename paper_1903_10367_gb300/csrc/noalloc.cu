// adafac_residual_norm_static: the Eq. 10 norm of b - A u for a uniform
// d-linear operator, computed without allocating device memory.
//
// Callers that cannot allocate: a solver service whose device memory is fully
// committed to resident workspaces (any allocation may fail or evict), and
// code that must not pay the device-wide synchronisation cudaFree implies.
// Such callers get a residual check on caller-owned u and b only: the kernels
// keep their per-block partial sums in a file-scope device array instead of a
// workspace.
//
// The scratch array is one per device (one per CUDA context that loads this
// library).  Calls that overlap in time on one device -- on different streams
// or from different host threads without ordering -- race on it and may
// return wrong norms; order them on one stream.
#include <mutex>

#include "adafac.h"
#include "common.cuh"

namespace adafac {

namespace {

// partial sums: one per block of kVertsPerBlock vertices
constexpr int kMaxPartials = 4096;
constexpr int kThreads = 256;
constexpr long long kVertsPerBlock = 64LL * kThreads;  // 16384
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxPartials];

std::mutex g_lock;
double* g_addr[kMaxDevices] = {};

// Partial sums of h^D r^2 over the interior vertices of one block's range,
// r = b - A u with A the assembled uniform stencil of -div(eps grad) on the
// d-linear element (Sec. 2.1): the neighbour at offset o with k non-zero
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

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).
double* scratch_address(int dev) {
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess) return nullptr;
    g_addr[dev] = static_cast<double*>(p);
  }
  return g_addr[dev];
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
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return ADAFAC_ERR_CUDA;
  double* partials = scratch_address(dev);
  if (!partials) return ADAFAC_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
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
