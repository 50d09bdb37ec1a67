// Brick engine of the adaptive-tree cycles: see adaptive_brick.h for the
// formulation.  A cycle is three kernels per level and one norm kernel:
//   residual  (l = L .. 1)     rho_l = W_l + P^T rho_{l+1}, with the Eq. 10
//                              partials of the level's nodal-space vertices
//   correct   (l = lmin .. L)  g_l = c_l - c~_l (Jac), c_l (additive / exp),
//                              c_l - I c_{l+1} (PI), zero at inactive vertices
//   prolong   (l = lmin .. L)  T_l = g_l + P T_{l-1};  U_l += T_l
// each over the vertex tiles that meet an existing cell of the level.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "adaptive_brick.h"

namespace adafac {

void smoothed_restriction_stencil(int D, double* out);  // api.cu

namespace brick {
namespace {

constexpr int kT = kTX * kTY;  // threads per tile block

// the truncated smoothed-restriction stencil in the cycle's arithmetic type
template <typename T>
struct Stencil5 {
  T w[125];
};

// the level's vertex (x, y, z) of this thread in a tile (x: tile column |
// tile row << 16, y: plane); false outside the grid
template <int D>
__device__ __forceinline__ bool tile_vertex(int n, int2 tile, int* c) {
  const int np1 = n + 1;
  c[0] = (tile.x & 0xffff) * kTX + (int)(threadIdx.x % kTX);
  c[1] = (tile.x >> 16) * kTY + (int)(threadIdx.x / kTX);
  c[2] = D == 3 ? tile.y : 0;
  return c[0] < np1 && c[1] < np1;
}

template <int D>
__device__ __forceinline__ long long vidx(const int* c, int np1) {
  return D == 2 ? (long long)c[1] * np1 + c[0] : ((long long)c[2] * np1 + c[1]) * np1 + c[0];
}

template <int D>
__device__ __forceinline__ bool inner(const int* c, int n) {
  bool in = c[0] >= 1 && c[0] <= n - 1 && c[1] >= 1 && c[1] <= n - 1;
  if (D == 3) in = in && c[2] >= 1 && c[2] <= n - 1;
  return in;
}

__device__ __forceinline__ bool halted(const Ctl* c) { return c->done || c->diverged; }

// Sum of one value per thread in a fixed order (warp trees, then the warps
// in order); valid in thread 0.
__device__ __forceinline__ double block_sum(double a) {
  __shared__ double red[kT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kT / 32; ++w) s += red[w];
  return s;
}

// The arrays of one level a cycle works on, in its arithmetic type: the FP64
// iterate U_l and its chains, or in a mixed solve the FP32 correction E_l
// with the FP32 right-hand sides of the level's leaf cells.
template <typename T>
struct View {
  int n = 0;
  T* U = nullptr;         // iterate (or correction) on the level's grid
  T* R = nullptr;         // rho_l (mixed: the chain of -K e, added to R0)
  const T* R0 = nullptr;  // mixed: the step's FP64 rho_l rounded to FP32
  T* G = nullptr;         // g_l
  T* Tc = nullptr;        // T_l (null on the finest level)
  const T* IM = nullptr;  // 1 / M_l at active vertices, else 0
  const T* B = nullptr;   // load of the level's leaf cells (null: zero)
  T* BT = nullptr;        // b~_l (optional)
  const T* EL = nullptr;  // eps of the level's leaf cells, else 0
  const uint8_t* nodal = nullptr;
  const int2* tiles = nullptr;
  int part_off = 0;
};

// W_l at an interior vertex: the load of the level's leaf cells minus their
// element matrices applied to U_l (eps of a non-leaf cell is 0 there).
// d-linear element by the Hamming distance of two corners (Sec. 2.1):
// 2-D 2/3, -1/6, -1/3; 3-D 1/3, 0, -1/12, -1/12, times h^(D-2).
template <int D, typename T>
__device__ __forceinline__ T leaf_residual(const View<T>& lv, const int* c, long long v) {
  const int n = lv.n, np1 = n + 1;
  const T* __restrict__ U = lv.U;
  const T* __restrict__ e = lv.EL;
  if (D == 2) {
    T E[9];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) E[(dy + 1) * 3 + dx + 1] = U[v + dy * np1 + dx];
    const long long c0 = (long long)(c[1] - 1) * n + c[0] - 1;
    T Ax = T(0);
#pragma unroll
    for (int sy = 0; sy < 2; ++sy)
#pragma unroll
      for (int sx = 0; sx < 2; ++sx) {
        const T ec = e[c0 + sy * n + sx];
        const T near = E[3 + 2 * sx] + E[6 * sy + 1];
        Ax += ec * (T(2.0 / 3.0) * E[4] + T(-1.0 / 6.0) * near + T(-1.0 / 3.0) * E[6 * sy + 2 * sx]);
      }
    return (lv.B ? lv.B[v] : T(0)) - Ax;
  } else {
    const long long P = (long long)np1 * np1;
    T E[3][9];
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx)
          E[dz + 1][(dy + 1) * 3 + dx + 1] = U[v + dz * P + dy * np1 + dx];
    T esum = T(0), far = T(0);
#pragma unroll
    for (int sz = 0; sz < 2; ++sz) {
      const T* S = E[2 * sz];
      const long long cz = (long long)(c[2] - 1 + sz) * n;
#pragma unroll
      for (int sy = 0; sy < 2; ++sy)
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
          const T ec = e[(cz + c[1] - 1 + sy) * n + c[0] - 1 + sx];
          const T f = (E[1][6 * sy + 2 * sx] + S[3 + 2 * sx]) + (S[6 * sy + 1] + S[6 * sy + 2 * sx]);
          esum += ec;
          far += ec * f;
        }
    }
    const T h = T(1.0 / (double)n);
    return (lv.B ? lv.B[v] : T(0)) - h * (T(1.0 / 3.0) * E[1][4] * esum + T(-1.0 / 12.0) * far);
  }
}

// d-linear weight of offset o in [-2, 2] of the 3:1 restriction
template <typename T>
__device__ __forceinline__ T wrest(int o) {
  return o == 0 ? T(1) : (o == 1 || o == -1 ? T(2.0 / 3.0) : T(1.0 / 3.0));
}

template <int D>
__device__ __forceinline__ long long fine_of(const int* c, int nf1) {
  return D == 2 ? (long long)(3 * c[1]) * nf1 + 3 * c[0]
                : ((long long)(3 * c[2]) * nf1 + 3 * c[1]) * nf1 + 3 * c[0];
}

// rho_l = W_l + P^T rho_{l+1} at the tile's vertices, zero on the boundary.
// With part: partial of h^D rho^2 over the nodal-space vertices of the
// block's tile.
template <int D, typename T>
__global__ void __launch_bounds__(kT)
    k_br_residual(const View<T> lv, const View<T> fine, double hD, double* __restrict__ part,
                  const Ctl* ctl, int query) {
  if (!query && halted(ctl)) return;
  int c[3];
  const bool in = tile_vertex<D>(lv.n, lv.tiles[blockIdx.x], c);
  double acc = 0.0;
  if (in) {
    const int n = lv.n, np1 = n + 1;
    const long long v = vidx<D>(c, np1);
    T rho = T(0);
    if (inner<D>(c, n)) {
      rho = leaf_residual<D, T>(lv, c, v);
      if (fine.n) {
        const int nf1 = fine.n + 1;
        const long long f0 = fine_of<D>(c, nf1);
        T rs = T(0);
        constexpr int OZ = D == 3 ? 2 : 0;
        for (int oz = -OZ; oz <= OZ; ++oz) {
          T ry = T(0);
#pragma unroll
          for (int oy = -2; oy <= 2; ++oy) {
            const long long row = f0 + ((long long)oz * nf1 + oy) * nf1;
            T rx = T(0);
#pragma unroll
            for (int ox = -2; ox <= 2; ++ox) rx += wrest<T>(ox) * fine.R[row + ox];
            ry += wrest<T>(oy) * rx;
          }
          rs += wrest<T>(oz) * ry;
        }
        rho += rs;
      }
      if (part && lv.nodal[v]) acc = (double)rho * (double)rho;
    }
    lv.R[v] = rho;
  }
  if (part) {
    const double sum = block_sum(acc);
    if (threadIdx.x == 0) part[lv.part_off + blockIdx.x] = sum * hD;
  }
}

// g_l at the tile's vertices (zero where the vertex is not active)
template <int D, typename T>
__global__ void __launch_bounds__(kT)
    k_br_correct(const View<T> lv, const View<T> fine, const Stencil5<T> st, int variant, double omega,
                 double omega_t, double gscale, const Ctl* ctl) {
  if (halted(ctl)) return;
  int c[3];
  if (!tile_vertex<D>(lv.n, lv.tiles[blockIdx.x], c)) return;
  const int np1 = lv.n + 1;
  const long long v = vidx<D>(c, np1);
  const T im = lv.IM[v];
  const T om = T(omega);
  T g = T(0), bt = T(0);
  if (im > T(0)) {
    const T cl = om * (lv.R[v] + (lv.R0 ? lv.R0[v] : T(0))) * im;
    if (fine.n && variant == ADAFAC_VARIANT_JAC) {
      // b~_l = omega S~ r_{l+1} over the 5^D window, r_{l+1} zero where the
      // finer level's vertex is not active
      const int nf1 = fine.n + 1;
      const long long f0 = fine_of<D>(c, nf1);
      constexpr int OZ = D == 3 ? 2 : 0;
      T acc = T(0);
      for (int oz = -OZ; oz <= OZ; ++oz)
#pragma unroll
        for (int oy = -2; oy <= 2; ++oy)
#pragma unroll
          for (int ox = -2; ox <= 2; ++ox) {
            const long long f = f0 + ((long long)oz * nf1 + oy) * nf1 + ox;
            const T r = fine.IM[f] > T(0) ? fine.R[f] + (fine.R0 ? fine.R0[f] : T(0)) : T(0);
            acc += st.w[((oz + OZ) * 5 + oy + 2) * 5 + ox + 2] * r;
          }
      bt = om * acc;
      g = cl - T(omega_t) * bt * im;
    } else if (fine.n && variant == ADAFAC_VARIANT_PI) {
      // minus the finer level's correction at the coinciding vertex (I c_{l+1})
      const long long f = fine_of<D>(c, fine.n + 1);
      const T imf = fine.IM[f];
      g = cl - (imf > T(0) ? om * (fine.R[f] + (fine.R0 ? fine.R0[f] : T(0))) * imf : T(0));
    } else {
      g = T(gscale) * cl;
    }
  }
  lv.G[v] = g;
  if (lv.BT) lv.BT[v] = bt;
}

// T_l = g_l + P T_{l-1} (coarse.n == 0 on the coarsest level of the cycle);
// U_l += T_l
template <int D, typename T>
__global__ void __launch_bounds__(kT)
    k_br_prolong(const View<T> lv, const View<T> coarse, Ctl* ctl, int count) {
  if (halted(ctl)) return;
  if (count && blockIdx.x == 0 && threadIdx.x == 0) ctl->applied += 1;
  int c[3];
  if (!tile_vertex<D>(lv.n, lv.tiles[blockIdx.x], c)) return;
  const int n = lv.n, np1 = n + 1;
  const long long v = vidx<D>(c, np1);
  if (!inner<D>(c, n)) {
    if (lv.Tc) lv.Tc[v] = T(0);
    return;
  }
  T t = lv.G[v];
  if (coarse.n) {
    const int nc = coarse.n, ncp1 = nc + 1;
    int O[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < D; ++j) {
      O[j] = min(c[j] / 3, nc - 1);
      lo[j] = c[j] - 3 * O[j];
    }
    T acc = T(0);
#pragma unroll
    for (int e = 0; e < (1 << D); ++e) {
      bool zero = false;
      T w = T(1);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int bit = (e >> j) & 1;
        zero = zero || (bit && lo[j] == 0);
        const T tt = lo[j] == 0 ? T(0) : (lo[j] == 1 ? T(1.0 / 3.0) : T(2.0 / 3.0));
        w *= bit ? tt : T(1) - tt;
      }
      if (zero) continue;
      const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
      const long long cv = D == 2 ? (long long)(O[1] + ey) * ncp1 + O[0] + ex
                                  : ((long long)(O[2] + ez) * ncp1 + O[1] + ey) * ncp1 + O[0] + ex;
      acc += w * coarse.Tc[cv];
    }
    t += acc;
  }
  if (lv.Tc) lv.Tc[v] = t;
  lv.U[v] += t;
}

// The finest level in one pass: g_L = gscale c_L (nothing above it damps
// it), T_L = g_L + P T_{L-1}, U_L += T_L.  g_L is kept for inspection.
template <int D, typename T>
__global__ void __launch_bounds__(kT)
    k_br_finest(const View<T> lv, const View<T> coarse, double omega, double gscale, Ctl* ctl,
                int count) {
  if (halted(ctl)) return;
  if (count && blockIdx.x == 0 && threadIdx.x == 0) ctl->applied += 1;
  int c[3];
  if (!tile_vertex<D>(lv.n, lv.tiles[blockIdx.x], c)) return;
  const int n = lv.n, np1 = n + 1;
  const long long v = vidx<D>(c, np1);
  const T im = lv.IM[v];
  const T g = im > T(0) ? T(gscale) * (T(omega) * (lv.R[v] + (lv.R0 ? lv.R0[v] : T(0))) * im) : T(0);
  lv.G[v] = g;
  if (!inner<D>(c, n)) return;
  T t = g;
  if (coarse.n) {
    const int nc = coarse.n, ncp1 = nc + 1;
    int O[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < D; ++j) {
      O[j] = min(c[j] / 3, nc - 1);
      lo[j] = c[j] - 3 * O[j];
    }
    T acc = T(0);
#pragma unroll
    for (int e = 0; e < (1 << D); ++e) {
      bool zero = false;
      T w = T(1);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int bit = (e >> j) & 1;
        zero = zero || (bit && lo[j] == 0);
        const T tt = lo[j] == 0 ? T(0) : (lo[j] == 1 ? T(1.0 / 3.0) : T(2.0 / 3.0));
        w *= bit ? tt : T(1) - tt;
      }
      if (zero) continue;
      const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
      const long long cv = D == 2 ? (long long)(O[1] + ey) * ncp1 + O[0] + ex
                                  : ((long long)(O[2] + ez) * ncp1 + O[1] + ey) * ncp1 + O[0] + ex;
      acc += w * coarse.Tc[cv];
    }
    t += acc;
  }
  lv.U[v] += t;
}

// mixed solve: the step's FP64 rho_l rounded to FP32, over the level's tiles
template <int D>
__global__ void __launch_bounds__(kT)
    k_br_round(int n, const int2* __restrict__ tiles, const double* __restrict__ R,
               float* __restrict__ R32, const Ctl* ctl) {
  if (halted(ctl)) return;
  int c[3];
  if (!tile_vertex<D>(n, tiles[blockIdx.x], c)) return;
  const long long v = vidx<D>(c, n + 1);
  R32[v] = (float)R[v];
}

// mixed solve: U_l += E_l (FP64 += FP32), E_l = 0, over the level's tiles
template <int D>
__global__ void __launch_bounds__(kT)
    k_br_add_correction(int n, const int2* __restrict__ tiles, double* __restrict__ U,
                        float* __restrict__ E, const Ctl* ctl) {
  if (halted(ctl)) return;
  int c[3];
  if (!tile_vertex<D>(n, tiles[blockIdx.x], c)) return;
  const long long v = vidx<D>(c, n + 1);
  U[v] += (double)E[v];
  E[v] = 0.f;
}

// the norm of Eq. 10 from the partials (fixed order); in a solve, the test
// that ends it
__global__ void k_br_finalize(const double* __restrict__ part, int npart, Ctl* ctl, int query) {
  if (!query && halted(ctl)) return;
  __shared__ double red[kT];
  double a = 0.0;
  for (int i = threadIdx.x; i < npart; i += blockDim.x) a += part[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x) return;
  const double abs_ = sqrt(red[0]);
  const double rel = ctl->r0 > 0.0 ? abs_ / ctl->r0 : 0.0;
  ctl->abs = abs_;
  ctl->rel = rel;
  if (query) return;
  if (!(rel <= 1e6)) ctl->diverged = 1;
  else if (ctl->tol >= 0.0 && rel <= ctl->tol) ctl->done = 1;
}

// ---- setup ------------------------------------------------------------------------

template <int D>
__device__ __forceinline__ void decode_cell(long long i, int n, int* c) {
  c[0] = (int)(i % n);
  const long long r = i / n;
  c[1] = (int)(r % n);
  c[2] = D == 3 ? (int)(r / n) : 0;
}

template <int D>
__device__ __forceinline__ long long cidx(const int* c, int n) {
  return D == 2 ? (long long)c[1] * n + c[0] : ((long long)c[2] * n + c[1]) * n + c[0];
}

// mean eps of the level-l cells from their 3^D children (x fastest, fixed order)
template <int D>
__global__ void k_br_eps_mean(int n, const double* __restrict__ child, double* __restrict__ out) {
  const long long C = D == 2 ? (long long)n * n : (long long)n * n * n;
  const int nf = 3 * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < C;
       i += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decode_cell<D>(i, n, c);
    double acc = 0.0;
    for (int kz = 0; kz < (D == 3 ? 3 : 1); ++kz)
      for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) {
          const int q[3] = {3 * c[0] + kx, 3 * c[1] + ky, 3 * c[2] + kz};
          acc += child[cidx<D>(q, nf)];
        }
    out[i] = acc / (D == 2 ? 9.0 : 27.0);
  }
}

// eps of the leaf cells (state 1), zero elsewhere
__global__ void k_br_leaf_eps(long long C, const uint8_t* __restrict__ state,
                              const double* __restrict__ em, double eps0, double* __restrict__ el) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < C;
       i += (long long)gridDim.x * blockDim.x)
    el[i] = state[i] == 1 ? (em ? em[i] : eps0) : 0.0;
}

// lumped load: every corner of a leaf cell of width h takes h^D / 2^D f
template <int D>
__global__ void k_br_load(int n, int s, int N1, const uint8_t* __restrict__ state,
                          const double* __restrict__ f, double* __restrict__ B) {
  const int np1 = n + 1;
  const long long V = D == 2 ? (long long)np1 * np1 : (long long)np1 * np1 * np1;
  const double h = 1.0 / (double)n;
  const double w = D == 2 ? h * h / 4.0 : h * h * h / 8.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decode_cell<D>(v, np1, c);
    int cnt = 0;
    for (int e = 0; e < (1 << D); ++e) {
      int q[3] = {c[0] - (e & 1), c[1] - ((e >> 1) & 1), D == 3 ? c[2] - ((e >> 2) & 1) : 0};
      bool ok = true;
      for (int j = 0; j < D; ++j) ok = ok && q[j] >= 0 && q[j] < n;
      if (ok && state[cidx<D>(q, n)] == 1) ++cnt;
    }
    double fv = 0.0;
    if (cnt && f) {
      const int p[3] = {s * c[0], s * c[1], s * c[2]};
      fv = f[D == 2 ? (long long)p[1] * N1 + p[0] : ((long long)p[2] * N1 + p[1]) * N1 + p[0]];
    }
    B[v] = cnt * w * fv;
  }
}

// element stiffness of the reference cell by the Hamming distance of corners
__device__ __forceinline__ double kref(int D, int ham) {
  if (D == 2) return ham == 0 ? 2.0 / 3.0 : (ham == 1 ? -1.0 / 6.0 : -1.0 / 3.0);
  return ham == 0 ? 1.0 / 3.0 : (ham == 1 ? 0.0 : -1.0 / 12.0);
}

// The collapsed element matrix E_l(Q) (2^D x 2^D, row-major) of every cell of
// level l: a leaf cell's element matrix, or over a cut cell's children o the
// sum of W_o^T E_{l+1}(child) W_o, W_o[a][p] the value of Q's corner-p hat at
// the child's corner a.  E of the children comes from `echild`, or on the
// finest level from their eps (`elchild`).
template <int D>
__global__ void k_br_elem(int n, const uint8_t* __restrict__ state, const double* __restrict__ el,
                          const double* __restrict__ echild, const double* __restrict__ elchild,
                          double* __restrict__ E) {
  constexpr int NC = 1 << D;
  const long long C = D == 2 ? (long long)n * n : (long long)n * n * n;
  const double hf = D == 2 ? 1.0 : 1.0 / (double)n, hfc = D == 2 ? 1.0 : 1.0 / (3.0 * n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < C;
       i += (long long)gridDim.x * blockDim.x) {
    double acc[NC * NC];
    for (int k = 0; k < NC * NC; ++k) acc[k] = 0.0;
    const uint8_t st = state[i];
    if (st == 1) {
      for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) acc[a * NC + b] = el[i] * hf * kref(D, __popc(a ^ b));
    } else if (st == 2) {
      int c[3];
      decode_cell<D>(i, n, c);
      for (int oz = 0; oz < (D == 3 ? 3 : 1); ++oz)
        for (int oy = 0; oy < 3; ++oy)
          for (int ox = 0; ox < 3; ++ox) {
            const int q[3] = {3 * c[0] + ox, 3 * c[1] + oy, 3 * c[2] + oz};
            const long long ci = cidx<D>(q, 3 * n);
            double Ec[NC * NC];
            if (echild) {
              for (int k = 0; k < NC * NC; ++k) Ec[k] = echild[ci * NC * NC + k];
            } else {
              const double e = elchild[ci];
              for (int a = 0; a < NC; ++a)
                for (int b = 0; b < NC; ++b) Ec[a * NC + b] = e * hfc * kref(D, __popc(a ^ b));
            }
            const int o[3] = {ox, oy, oz};
            double W[NC * NC];  // W[a][p]
            for (int a = 0; a < NC; ++a)
              for (int p = 0; p < NC; ++p) {
                double w = 1.0;
                for (int j = 0; j < D; ++j) {
                  const double t = (double)(o[j] + ((a >> j) & 1)) / 3.0;
                  w *= ((p >> j) & 1) ? t : 1.0 - t;
                }
                W[a * NC + p] = w;
              }
            // acc += W^T Ec W
            for (int p = 0; p < NC; ++p)
              for (int q2 = 0; q2 < NC; ++q2) {
                double sum = 0.0;
                for (int a = 0; a < NC; ++a) {
                  double inner_ = 0.0;
                  for (int b = 0; b < NC; ++b) inner_ += Ec[a * NC + b] * W[b * NC + q2];
                  sum += W[a * NC + p] * inner_;
                }
                acc[p * NC + q2] += sum;
              }
          }
    }
    for (int k = 0; k < NC * NC; ++k) E[i * NC * NC + k] = acc[k];
  }
}

// 1 / M_l at the active vertices (interior, every surrounding cell exists),
// M_l(J) the sum of the diagonal entries of J in those cells' E_l
template <int D>
__global__ void k_br_diag(int n, const uint8_t* __restrict__ state, const double* __restrict__ E,
                          const double* __restrict__ el, double* __restrict__ IM) {
  constexpr int NC = 1 << D;
  const int np1 = n + 1;
  const long long V = D == 2 ? (long long)np1 * np1 : (long long)np1 * np1 * np1;
  const double hf = D == 2 ? 1.0 : 1.0 / (double)n;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decode_cell<D>(v, np1, c);
    bool act = inner<D>(c, n);
    double M = 0.0;
    for (int e = 0; act && e < NC; ++e) {
      // the cell that has J as its corner e
      const int q[3] = {c[0] - (e & 1), c[1] - ((e >> 1) & 1), D == 3 ? c[2] - ((e >> 2) & 1) : 0};
      const long long ci = cidx<D>(q, n);
      if (state[ci] == 0) {
        act = false;
        break;
      }
      M += E ? E[ci * NC * NC + e * NC + e] : el[ci] * hf * kref(D, 0);
    }
    IM[v] = act && M > 0.0 ? 1.0 / M : 0.0;
  }
}

// the position's finest active level is this one
template <int D>
__global__ void k_br_nodal(int n, const double* __restrict__ IM, const double* __restrict__ IMf,
                           uint8_t* __restrict__ nodal) {
  const int np1 = n + 1, nf1 = 3 * n + 1;
  const long long V = D == 2 ? (long long)np1 * np1 : (long long)np1 * np1 * np1;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decode_cell<D>(v, np1, c);
    bool nod = IM[v] > 0.0;
    if (nod && IMf) {
      const long long f = D == 2 ? (long long)(3 * c[1]) * nf1 + 3 * c[0]
                                 : ((long long)(3 * c[2]) * nf1 + 3 * c[1]) * nf1 + 3 * c[0];
      nod = !(IMf[f] > 0.0);
    }
    nodal[v] = nod ? 1 : 0;
  }
}

// FP32 copies of 1 / M_l and eps for the cycles of a mixed solve
__global__ void k_br_to_float(long long n, const double* __restrict__ a, float* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// ---- leaf-node vectors -------------------------------------------------------------

template <int D>
__device__ __forceinline__ void fine_coords(long long g, int N1, int* q) {
  q[0] = (int)(g % N1);
  const long long r = g / N1;
  q[1] = (int)(r % N1);
  q[2] = D == 3 ? (int)(r / N1) : 0;
}

// u at the leaf nodes from the level copies: a node is a corner of a leaf
// cell of some level l, where U_l holds its value
template <int D>
__global__ void k_br_gather(int nn, const long long* __restrict__ nodes, int L, int N1,
                            const Level* __restrict__ levs, double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int q[3];
  fine_coords<D>(nodes[i], N1, q);
  double val = 0.0;
  int s = 1;
  for (int l = L; l >= 1; --l, s *= 3) {
    bool on = true;
    for (int j = 0; j < D; ++j) on = on && q[j] % s == 0;
    if (!on) break;  // not on this grid, nor on a coarser one
    const Level& lv = levs[l];
    const int n = lv.n;
    const int J[3] = {q[0] / s, q[1] / s, q[2] / s};
    bool corner = false;
    for (int e = 0; e < (1 << D) && !corner; ++e) {
      int c[3] = {J[0] - (e & 1), J[1] - ((e >> 1) & 1), D == 3 ? J[2] - ((e >> 2) & 1) : 0};
      bool ok = true;
      for (int j = 0; j < D; ++j) ok = ok && c[j] >= 0 && c[j] < n;
      corner = ok && lv.leaf[cidx<D>(c, n)] == 1;
    }
    if (corner) {
      val = lv.U[vidx<D>(J, n + 1)];
      break;
    }
  }
  u[i] = val;
}

// the level copies from u at the leaf nodes: every level whose grid holds
// the node takes its value
template <int D>
__global__ void k_br_scatter(int nn, const long long* __restrict__ nodes, int L, int N1,
                             const Level* __restrict__ levs, const double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int q[3];
  fine_coords<D>(nodes[i], N1, q);
  int s = 1;
  for (int l = L; l >= 1; --l, s *= 3) {
    bool on = true;
    for (int j = 0; j < D; ++j) on = on && q[j] % s == 0;
    if (!on) break;
    const Level& lv = levs[l];
    const int J[3] = {q[0] / s, q[1] / s, q[2] / s};
    lv.U[vidx<D>(J, lv.n + 1)] = u[i];
  }
}

// transfer: T_l = v at the level's nodal-space vertices, else P T_{l-1};
// U_l = T_l (the function of the space with values v there)
template <int D>
__global__ void __launch_bounds__(kT)
    k_br_from_values(const Level lv, const Level coarse, int L, int N1, const int* __restrict__ node_map,
                     const double* __restrict__ vals) {
  int c[3];
  if (!tile_vertex<D>(lv.n, lv.tiles[blockIdx.x], c)) return;
  const int n = lv.n, np1 = n + 1;
  const long long v = vidx<D>(c, np1);
  double t = 0.0;
  if (inner<D>(c, n)) {
    if (lv.nodal[v]) {
      const long long g = D == 2 ? (long long)(lv.s * c[1]) * N1 + lv.s * c[0]
                                 : ((long long)(lv.s * c[2]) * N1 + lv.s * c[1]) * N1 + lv.s * c[0];
      const int p = node_map[g];
      t = p >= 0 ? vals[p] : 0.0;
    } else if (coarse.n) {
      const int nc = coarse.n, ncp1 = nc + 1;
      int O[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
      for (int j = 0; j < D; ++j) {
        O[j] = min(c[j] / 3, nc - 1);
        lo[j] = c[j] - 3 * O[j];
      }
      for (int e = 0; e < (1 << D); ++e) {
        bool zero = false;
        double w = 1.0;
        for (int j = 0; j < D; ++j) {
          const int bit = (e >> j) & 1;
          zero = zero || (bit && lo[j] == 0);
          const double tt = lo[j] == 0 ? 0.0 : (lo[j] == 1 ? 1.0 / 3.0 : 2.0 / 3.0);
          w *= bit ? tt : 1.0 - tt;
        }
        if (zero) continue;
        const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
        const long long cv = D == 2 ? (long long)(O[1] + ey) * ncp1 + O[0] + ex
                                    : ((long long)(O[2] + ez) * ncp1 + O[1] + ey) * ncp1 + O[0] + ex;
        t += w * coarse.T[cv];
      }
    }
  }
  lv.T[v] = t;
  lv.U[v] = t;
}

}  // namespace

namespace {

long long ipw(long long b, int e) {
  long long r = 1;
  while (e-- > 0) r *= b;
  return r;
}

int grid_for(long long n) {
  const long long b = (n + kT - 1) / kT;
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 64));
}

template <typename T>
T* dalloc(System& S, long long count) {
  void* p = nullptr;
  if (count <= 0) count = 1;
  if (cudaMalloc(&p, sizeof(T) * (size_t)count) != cudaSuccess) return nullptr;
  S.allocs.push_back(p);
  cudaMemset(p, 0, sizeof(T) * (size_t)count);
  return static_cast<T*>(p);
}

}  // namespace

void release(System& S) {
  for (void* p : S.allocs) cudaFree(p);
  S.allocs.clear();
  S.ctl = nullptr;
  S.part = nullptr;
}

adafac_status build(System& S, int D, int L, const Tree& tree, const double* eps, int eps_scalar,
                    const double* f, bool mixed, cudaStream_t s, std::string* err) {
  S.D = D;
  S.L = L;
  S.mixed = mixed;
  const int NC = 1 << D;
  const long long N = ipw(3, L), N1 = N + 1;
  auto fail = [&](const char* what) {
    cudaGetLastError();
    *err = what;
    return ADAFAC_ERR_OOM;
  };
  // levels: sizes, cell states, tiles
  int part = 0;
  for (int l = 1; l <= L; ++l) {
    Level& lv = S.lev[l];
    lv = Level();
    lv.n = (int)ipw(3, l);
    lv.s = (int)ipw(3, L - l);
    lv.V = ipw(lv.n + 1, D);
    lv.C = ipw(lv.n, D);
    std::vector<uint8_t> state(lv.C);
    for (long long i = 0; i < lv.C; ++i)
      state[i] = tree.exists[l][i] ? (tree.cut[l][i] ? 2 : 1) : 0;
    const int np1 = lv.n + 1;
    const int ntx = (np1 + kTX - 1) / kTX, nty = (np1 + kTY - 1) / kTY;
    const int ntz = D == 3 ? np1 : 1;
    std::vector<uint8_t> mark((size_t)ntx * nty * ntz, 0);
    for (long long i = 0; i < lv.C; ++i) {
      if (!state[i]) continue;
      const int cx = (int)(i % lv.n), cy = (int)((i / lv.n) % lv.n), cz = D == 3 ? (int)(i / lv.n / lv.n) : 0;
      for (int e = 0; e < NC; ++e) {
        const int x = cx + (e & 1), y = cy + ((e >> 1) & 1), z = D == 3 ? cz + ((e >> 2) & 1) : 0;
        mark[((size_t)z * nty + y / kTY) * ntx + x / kTX] = 1;
      }
    }
    std::vector<int2> tiles;
    for (size_t t = 0; t < mark.size(); ++t)
      if (mark[t]) {
        const int tx = (int)(t % ntx), ty = (int)((t / ntx) % nty), tz = (int)(t / ntx / nty);
        tiles.push_back(make_int2(tx | (ty << 16), tz));
      }
    lv.ntiles = (int)tiles.size();
    lv.part_off = part;
    part += lv.ntiles;
    lv.leaf = dalloc<uint8_t>(S, lv.C);
    lv.tiles = dalloc<int2>(S, lv.ntiles);
    lv.U = dalloc<double>(S, lv.V);
    lv.R = dalloc<double>(S, lv.V);
    lv.G = dalloc<double>(S, lv.V);
    lv.IM = dalloc<double>(S, lv.V);
    lv.B = dalloc<double>(S, lv.V);
    lv.EL = dalloc<double>(S, lv.C);
    lv.nodal = dalloc<uint8_t>(S, lv.V);
    if (l < L) {
      lv.T = dalloc<double>(S, lv.V);
      lv.BT = dalloc<double>(S, lv.V);
    }
    if (mixed) {
      lv.E32 = dalloc<float>(S, lv.V);
      lv.R32 = dalloc<float>(S, lv.V);
      lv.G32 = dalloc<float>(S, lv.V);
      lv.IM32 = dalloc<float>(S, lv.V);
      lv.RHS32 = dalloc<float>(S, lv.V);
      lv.EL32 = dalloc<float>(S, lv.C);
      if (l < L) lv.T32 = dalloc<float>(S, lv.V);
      if (!lv.E32 || !lv.R32 || !lv.G32 || !lv.IM32 || !lv.RHS32 || !lv.EL32 || (l < L && !lv.T32))
        return fail("brick engine: device allocation failed");
    }
    if (!lv.leaf || !lv.tiles || !lv.U || !lv.R || !lv.G || !lv.IM || !lv.B || !lv.EL ||
        !lv.nodal || (l < L && (!lv.T || !lv.BT)))
      return fail("brick engine: device allocation failed");
    if (cudaMemcpyAsync(lv.leaf, state.data(), lv.C, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (lv.ntiles && cudaMemcpyAsync(lv.tiles, tiles.data(), sizeof(int2) * tiles.size(),
                                      cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail("brick engine: copy of the tree failed");
  }
  S.npart = part;
  S.part = dalloc<double>(S, part);
  S.ctl = dalloc<Ctl>(S, 1);
  if (!S.part || !S.ctl) return fail("brick engine: device allocation failed");
  // eps of the leaf cells (means of the fine eps, level by level)
  double* em_child = nullptr;
  std::vector<double*> scratch;
  auto tmp = [&](long long count) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(double) * (size_t)std::max<long long>(count, 1)) != cudaSuccess)
      return (double*)nullptr;
    scratch.push_back(static_cast<double*>(p));
    return static_cast<double*>(p);
  };
  auto free_tmp = [&]() {
    cudaStreamSynchronize(s);
    for (double* p : scratch) cudaFree(p);
    scratch.clear();
  };
  for (int l = L; l >= 1; --l) {
    Level& lv = S.lev[l];
    double* em = nullptr;
    if (!eps_scalar) {
      em = tmp(lv.C);
      if (!em) {
        free_tmp();
        return fail("brick engine: device allocation failed");
      }
      if (l == L) {
        if (cudaMemcpyAsync(em, eps, sizeof(double) * lv.C, cudaMemcpyHostToDevice, s) != cudaSuccess) {
          free_tmp();
          return fail("brick engine: copy of eps failed");
        }
      } else if (D == 2) {
        k_br_eps_mean<2><<<grid_for(lv.C), kT, 0, s>>>(lv.n, em_child, em);
      } else {
        k_br_eps_mean<3><<<grid_for(lv.C), kT, 0, s>>>(lv.n, em_child, em);
      }
    }
    k_br_leaf_eps<<<grid_for(lv.C), kT, 0, s>>>(lv.C, lv.leaf, em, eps_scalar ? eps[0] : 0.0, lv.EL);
    em_child = em;
  }
  free_tmp();
  // lumped load
  {
    double* df = nullptr;
    if (f) {
      df = tmp(ipw(N1, D));
      if (!df || cudaMemcpyAsync(df, f, sizeof(double) * ipw(N1, D), cudaMemcpyHostToDevice, s) !=
                     cudaSuccess) {
        free_tmp();
        return fail("brick engine: copy of f failed");
      }
    }
    for (int l = 1; l <= L; ++l) {
      Level& lv = S.lev[l];
      if (D == 2) k_br_load<2><<<grid_for(lv.V), kT, 0, s>>>(lv.n, lv.s, (int)N1, lv.leaf, df, lv.B);
      else k_br_load<3><<<grid_for(lv.V), kT, 0, s>>>(lv.n, lv.s, (int)N1, lv.leaf, df, lv.B);
    }
    free_tmp();
  }
  // M_l from the collapsed element matrices, bottom-up
  {
    double* Echild = nullptr;
    for (int l = L; l >= 1; --l) {
      Level& lv = S.lev[l];
      double* E = nullptr;
      if (l < L) {
        E = tmp(lv.C * NC * NC);
        if (!E) {
          free_tmp();
          return fail("brick engine: device allocation failed");
        }
        const double* elc = S.lev[l + 1].EL;
        if (D == 2) k_br_elem<2><<<grid_for(lv.C), kT, 0, s>>>(lv.n, lv.leaf, lv.EL, Echild, elc, E);
        else k_br_elem<3><<<grid_for(lv.C), kT, 0, s>>>(lv.n, lv.leaf, lv.EL, Echild, elc, E);
      }
      if (D == 2) k_br_diag<2><<<grid_for(lv.V), kT, 0, s>>>(lv.n, lv.leaf, E, lv.EL, lv.IM);
      else k_br_diag<3><<<grid_for(lv.V), kT, 0, s>>>(lv.n, lv.leaf, E, lv.EL, lv.IM);
      // the child level's matrices are no longer needed once this level has its own
      if (Echild) {
        cudaStreamSynchronize(s);
        cudaFree(Echild);
        scratch.erase(std::find(scratch.begin(), scratch.end(), Echild));
      }
      Echild = E;
    }
    free_tmp();
  }
  for (int l = 1; l <= L; ++l) {
    Level& lv = S.lev[l];
    const double* IMf = l < L ? S.lev[l + 1].IM : nullptr;
    if (D == 2) k_br_nodal<2><<<grid_for(lv.V), kT, 0, s>>>(lv.n, lv.IM, IMf, lv.nodal);
    else k_br_nodal<3><<<grid_for(lv.V), kT, 0, s>>>(lv.n, lv.IM, IMf, lv.nodal);
  }
  if (mixed) {
    for (int l = 1; l <= L; ++l) {
      Level& lv = S.lev[l];
      k_br_to_float<<<grid_for(lv.V), kT, 0, s>>>(lv.V, lv.IM, lv.IM32);
      k_br_to_float<<<grid_for(lv.C), kT, 0, s>>>(lv.C, lv.EL, lv.EL32);
    }
  }
  smoothed_restriction_stencil(D, S.stilde);
  Ctl c{};
  c.tol = -1.0;
  if (cudaMemcpyAsync(S.ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail("brick engine: setup kernels failed");
  return ADAFAC_OK;
}

namespace {

template <typename T>
View<T> none() {
  return View<T>();
}

View<double> view64(const Level& lv) {
  View<double> v;
  v.n = lv.n;
  v.U = lv.U;
  v.R = lv.R;
  v.G = lv.G;
  v.Tc = lv.T;
  v.IM = lv.IM;
  v.B = lv.B;
  v.BT = lv.BT;
  v.EL = lv.EL;
  v.nodal = lv.nodal;
  v.tiles = lv.tiles;
  v.part_off = lv.part_off;
  return v;
}

View<float> view32(const Level& lv) {
  View<float> v;
  v.n = lv.n;
  v.U = lv.E32;
  v.R = lv.R32;
  v.G = lv.G32;
  v.Tc = lv.T32;
  v.IM = lv.IM32;
  v.R0 = lv.RHS32;
  v.EL = lv.EL32;
  v.nodal = lv.nodal;
  v.tiles = lv.tiles;
  v.part_off = lv.part_off;
  return v;
}

template <typename T>
View<T> view(const Level& lv);
template <>
View<double> view<double>(const Level& lv) {
  return view64(lv);
}
template <>
View<float> view<float>(const Level& lv) {
  return view32(lv);
}

// the residual chain of levels L .. lo; FP64 with the norm partials (and,
// in a mixed solve, the FP32 right-hand sides), FP32 without
template <int D, typename T>
void residual_chain(System& S, int lo, bool query, bool partials, cudaStream_t s) {
  for (int l = S.L; l >= lo; --l) {
    Level& lv = S.lev[l];
    if (!lv.ntiles) continue;
    const View<T> fine = l < S.L ? view<T>(S.lev[l + 1]) : none<T>();
    const double hD = std::pow(1.0 / (double)lv.n, D);
    k_br_residual<D, T><<<lv.ntiles, kT, 0, s>>>(view<T>(lv), fine, hD, partials ? S.part : nullptr,
                                                S.ctl, query ? 1 : 0);
  }
}

// corrections and prolongation of one cycle over levels lmin .. L
template <int D, typename T>
void corrections(System& S, const adafac_options& o, cudaStream_t s) {
  const int L = S.L, lmin = o.lmin;
  Stencil5<T> st;
  for (int k = 0; k < 125; ++k) st.w[k] = (T)S.stilde[k];
  // levels below the finest: corrections, then the prolongation chain; the
  // finest level's correction and update in one pass after them
  for (int l = lmin; l < L; ++l) {
    Level& lv = S.lev[l];
    if (!lv.ntiles) continue;
    const View<T> fine = view<T>(S.lev[l + 1]);
    const double gscale = o.variant == ADAFAC_VARIANT_EXP ? std::pow(o.omega_exp, L - l) : 1.0;
    k_br_correct<D, T><<<lv.ntiles, kT, 0, s>>>(view<T>(lv), fine, st, o.variant, o.omega,
                                               o.omega_tilde, gscale, S.ctl);
  }
  int lcount = lmin;  // the cycle is counted by the finest level that has cells
  for (int l = lmin; l <= L; ++l)
    if (S.lev[l].ntiles) lcount = l;
  for (int l = lmin; l < L; ++l) {
    Level& lv = S.lev[l];
    if (!lv.ntiles) continue;
    const View<T> coarse = l > lmin ? view<T>(S.lev[l - 1]) : none<T>();
    k_br_prolong<D, T><<<lv.ntiles, kT, 0, s>>>(view<T>(lv), coarse, S.ctl, l == lcount ? 1 : 0);
  }
  if (S.lev[L].ntiles) {
    const View<T> coarse = L > lmin ? view<T>(S.lev[L - 1]) : none<T>();
    k_br_finest<D, T><<<S.lev[L].ntiles, kT, 0, s>>>(view<T>(S.lev[L]), coarse, o.omega, 1.0,
                                                    S.ctl, L == lcount ? 1 : 0);
  }
}

template <int D>
void cycle_d(System& S, const adafac_options& o, bool with_norm, cudaStream_t s) {
  // the norm runs over every level's nodal-space vertices: the chain goes to
  // level 1 when it is evaluated
  residual_chain<D, double>(S, with_norm ? 1 : o.lmin, false, with_norm, s);
  if (with_norm) k_br_finalize<<<1, kT, 0, s>>>(S.part, S.npart, S.ctl, 0);
  corrections<D, double>(S, o, s);
}

// The correction equation's cycles see rho^e_l = Phi_l^T (r - K e) as the
// step's FP64 rho_l rounded to FP32 plus the FP32 chain of the leaf cells'
// -K e.  The FP64 rho_l tends to zero at the active vertices as the solve
// converges; the composite residual r itself does not (at hanging nodes,
// which carry no unknown, it stays of the load's size), so rounding r or
// the levels' parts of it to FP32 would stall the solve near FP32 epsilon.
template <int D>
void step_d(System& S, const adafac_options& o, int k, bool with_norm, cudaStream_t s) {
  residual_chain<D, double>(S, 1, false, true, s);
  if (with_norm) k_br_finalize<<<1, kT, 0, s>>>(S.part, S.npart, S.ctl, 0);
  for (int l = 1; l <= S.L; ++l) {
    Level& lv = S.lev[l];
    if (lv.ntiles) k_br_round<D><<<lv.ntiles, kT, 0, s>>>(lv.n, lv.tiles, lv.R, lv.RHS32, S.ctl);
  }
  for (int j = 0; j < k; ++j) {
    residual_chain<D, float>(S, o.lmin, false, false, s);
    corrections<D, float>(S, o, s);
  }
  for (int l = o.lmin; l <= S.L; ++l) {
    Level& lv = S.lev[l];
    if (!lv.ntiles) continue;
    k_br_add_correction<D><<<lv.ntiles, kT, 0, s>>>(lv.n, lv.tiles, lv.U, lv.E32, S.ctl);
  }
}

}  // namespace

void enqueue_cycle(System& S, const adafac_options& o, bool with_norm, cudaStream_t s) {
  if (S.D == 2) cycle_d<2>(S, o, with_norm, s);
  else cycle_d<3>(S, o, with_norm, s);
}

void enqueue_step(System& S, const adafac_options& o, int k, bool with_norm, cudaStream_t s) {
  if (S.D == 2) step_d<2>(S, o, k, with_norm, s);
  else step_d<3>(S, o, k, with_norm, s);
}

void enqueue_norm(System& S, cudaStream_t s) {
  if (S.D == 2) residual_chain<2, double>(S, 1, true, true, s);
  else residual_chain<3, double>(S, 1, true, true, s);
  k_br_finalize<<<1, kT, 0, s>>>(S.part, S.npart, S.ctl, 1);
}

namespace {

// the level table on the device for the leaf-node kernels (one allocation per call)
template <typename F>
void with_table(System& S, cudaStream_t s, F&& run) {
  Level* d = nullptr;
  if (cudaMalloc(&d, sizeof(Level) * (kMaxL + 1)) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaMemcpyAsync(d, S.lev, sizeof(Level) * (kMaxL + 1), cudaMemcpyHostToDevice, s);
  run(d);
  cudaStreamSynchronize(s);
  cudaFree(d);
}

}  // namespace

void gather_nodes(System& S, const long long* nodes, int nn, double* u, cudaStream_t s) {
  if (nn <= 0) return;
  const int N1 = (int)ipw(3, S.L) + 1;
  const int g = (nn + kT - 1) / kT;
  with_table(S, s, [&](const Level* d) {
    if (S.D == 2) k_br_gather<2><<<g, kT, 0, s>>>(nn, nodes, S.L, N1, d, u);
    else k_br_gather<3><<<g, kT, 0, s>>>(nn, nodes, S.L, N1, d, u);
  });
}

void scatter_nodes(System& S, const long long* nodes, int nn, const double* u, cudaStream_t s) {
  if (nn <= 0) return;
  const int N1 = (int)ipw(3, S.L) + 1;
  const int g = (nn + kT - 1) / kT;
  with_table(S, s, [&](const Level* d) {
    if (S.D == 2) k_br_scatter<2><<<g, kT, 0, s>>>(nn, nodes, S.L, N1, d, u);
    else k_br_scatter<3><<<g, kT, 0, s>>>(nn, nodes, S.L, N1, d, u);
  });
}

void from_node_values(System& S, const int* node_map, const double* v, cudaStream_t s) {
  const int N1 = (int)ipw(3, S.L) + 1;
  for (int l = 1; l <= S.L; ++l) {
    Level& lv = S.lev[l];
    if (!lv.ntiles) continue;
    Level cur = lv;
    if (!cur.T) cur.T = cur.G;  // the finest level keeps its chain value in G (scratch)
    const Level coarse = l > 1 ? S.lev[l - 1] : Level();
    if (S.D == 2)
      k_br_from_values<2><<<lv.ntiles, kT, 0, s>>>(cur, coarse, S.L, N1, node_map, v);
    else
      k_br_from_values<3><<<lv.ntiles, kT, 0, s>>>(cur, coarse, S.L, N1, node_map, v);
  }
}

}  // namespace brick
}  // namespace adafac
