// Additive cycles on adaptive 3:1 spacetrees (static trees, FP64).
//
// The tree is given level by level: level 1 exists in full, a level-l cell is
// cut into 3^D children where the caller's flag says so (Sec. 2.1).  Leaf
// cells carry the d-linear element of -div(eps grad u); the composite
// function is held by its values at the leaf nodes (every corner of a leaf
// cell, hanging positions included).  Level l's shape functions are the
// pagodas of its active vertices -- interior vertices whose 2^D surrounding
// level-l cells all exist -- and together they form the generating system of
// Sec. 2.1 and 2.3.  With Phi_l the pagodas' values at the leaf nodes and K
// the leaf cells' stiffness:
//   r_l = Phi_l^T (b - K u)                  (the residual level l sees)
//   A_l = Phi_l^T K Phi_l,  M_l = diag(A_l)  (Ritz-Galerkin, Sec. 2.2)
//   u  += sum_l Phi_l c_l - sum_{l > lmin} Phi_{l-1} c~_{l-1}   (Eq. 9)
// with c_l = omega M_l^-1 r_l and the damping equation c~_{l-1} =
// omega~ M_{l-1}^-1 R~ r_l (Eq. 7-8).  The truncated R~ applies the 5^D
// smoothed-restriction stencil to level l's residual held on its full grid
// (zero at inactive positions); the exact R~ is omega Phi_{l-1}^T K Phi_l
// M_l^-1.  Hanging vertices carry no unknown: their values follow from the
// pagodas, i.e. d-linear interpolation from the coarser level.
//
// Layout on the device: leaf-node vectors (u, b, r, du), K and every Phi_l in
// CSR over the leaf nodes, Phi_l^T in CSR over the active vertices, and per
// level the brick -- the level's full (3^l + 1)^D grid -- for r_l and c_l.
// The host builds the system once; every step of a cycle runs in the kernels
// below.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/adafac.h"
#include "adaptive_brick.h"
#include "engine.h"

namespace adafac {

void smoothed_restriction_stencil(int D, double* out);  // api.cu

namespace ad {

// the truncated smoothed-restriction stencil (5^D weights, x fastest)
struct Stencil {
  double w[125];
};

struct DevCsr {
  int rows = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  double* v = nullptr;
};

struct Level {
  int n = 0;                         // cells per axis
  long long G = 0;                   // grid points (n + 1)^D
  int na = 0;                        // active vertices
  std::vector<long long> act;        // their grid indices, ascending
  std::vector<int> fr;               // active ids whose finest level is this one
  std::vector<int> frnode;           // their leaf nodes
  std::vector<double> diag;
  DevCsr phi, phit;                  // Phi_l over the nodes, Phi_l^T over the active ids
  int phit_max = 0;                  // longest row of Phi_l^T (nodes a pagoda reaches)
  long long* d_act = nullptr;
  int* d_fr = nullptr;
  int* d_frnode = nullptr;
  double* d_diag = nullptr;
  double* d_rg = nullptr;            // r_l on the level grid
  double* d_cg = nullptr;            // c_l on the level grid
  double* d_g = nullptr;             // g_l = c_l - c~_l (scaled) per active id
  double* d_bt = nullptr;            // b~_l per active id
  double* d_x = nullptr;             // scratch per active id (exact R~)
};

}  // namespace ad

namespace {

using ad::DevCsr;
using ad::Level;
constexpr int kThreads = 256;

// ---- kernels ---------------------------------------------------------------------

// rr = b - K u at the leaf nodes
__global__ void k_ad_residual(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ kv, const double* __restrict__ b,
                              const double* __restrict__ u, double* __restrict__ rr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) acc += kv[k] * u[ci[k]];
  rr[i] = b[i] - acc;
}

// level l: r_l = Phi_l^T rr at the active vertices, onto the level grid; the
// Jacobi correction c_l = omega r_l / M_l onto the grid; g_l = scale c_l
__global__ void k_ad_restrict(int na, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ pv, const double* __restrict__ rr,
                              const long long* __restrict__ act, const double* __restrict__ diag,
                              double omega, double scale, double* __restrict__ rg,
                              double* __restrict__ cg, double* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= na) return;
  double r = 0.0;
  for (int k = rp[j]; k < rp[j + 1]; ++k) r += pv[k] * rr[ci[k]];
  const double c = omega * r / diag[j];
  rg[act[j]] = r;
  if (cg) cg[act[j]] = c;
  if (g) g[j] = scale * c;
}

// the same for levels whose pagodas reach many leaf nodes: a warp (WIDE =
// 32) or a block of kThreads threads (WIDE = kThreads) per active vertex,
// summing the row in a fixed order (strided partial sums, then a tree)
template <int WIDE>
__global__ void __launch_bounds__(kThreads)
    k_ad_restrict_wide(int na, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ pv, const double* __restrict__ rr,
                       const long long* __restrict__ act, const double* __restrict__ diag,
                       double omega, double scale, double* __restrict__ rg,
                       double* __restrict__ cg, double* __restrict__ g) {
  __shared__ double red[kThreads / 32];
  constexpr int PER = kThreads / WIDE;  // rows per block
  const int lane = threadIdx.x % WIDE;
  const int j = blockIdx.x * PER + threadIdx.x / WIDE;
  double acc = 0.0;
  if (j < na)
    for (int k = rp[j] + lane; k < rp[j + 1]; k += WIDE) acc += pv[k] * rr[ci[k]];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (WIDE > 32) {
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      acc = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) acc += red[w];
    }
  }
  if (lane != 0 || j >= na) return;
  const double c = omega * acc / diag[j];
  rg[act[j]] = acc;
  if (cg) cg[act[j]] = c;
  if (g) g[j] = scale * c;
}

// y = A x for a CSR matrix with long rows (a warp or a block per row)
template <int WIDE>
__global__ void __launch_bounds__(kThreads)
    k_ad_spmv_wide(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                   const double* __restrict__ av, const double* __restrict__ x,
                   double* __restrict__ y) {
  __shared__ double red[kThreads / 32];
  constexpr int PER = kThreads / WIDE;
  const int lane = threadIdx.x % WIDE;
  const int i = blockIdx.x * PER + threadIdx.x / WIDE;
  double acc = 0.0;
  if (i < n)
    for (int k = rp[i] + lane; k < rp[i + 1]; k += WIDE) acc += av[k] * x[ci[k]];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (WIDE > 32) {
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      acc = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) acc += red[w];
    }
  }
  if (lane == 0 && i < n) y[i] = acc;
}

// truncated damping equation of level l - 1 from level l's residual grid:
// b~ = omega sum_o S~[o] r_l(3J + o); g_{l-1} -= omega~ b~ / M_{l-1}
template <int D>
__global__ void k_ad_damp(int na, const long long* __restrict__ act, int nc,
                          const double* __restrict__ rg, const double* __restrict__ diag,
                          const ad::Stencil st, double omega, double omega_t,
                          double* __restrict__ bt, double* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= na) return;
  const long long ncp1 = nc + 1, nf1 = 3LL * nc + 1;
  long long v = act[j];
  int J[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) {
    J[k] = (int)(v % ncp1);
    v /= ncp1;
  }
  double acc = 0.0;
  constexpr int N5 = D == 2 ? 25 : 125;
  for (int s = 0; s < N5; ++s) {
    const double w = st.w[s];
    if (w == 0.0) continue;
    int t = s;
    long long idx = 0, stride = 1;
    for (int k = 0; k < D; ++k) {
      idx += (3LL * J[k] + (t % 5) - 2) * stride;
      t /= 5;
      stride *= nf1;
    }
    acc += w * rg[idx];
  }
  const double b = omega * acc;
  bt[j] = b;
  g[j] -= omega_t * b / diag[j];
}

// adAFAC-PI: g_{l-1} -= I c_l (level l's correction at the coinciding vertex)
template <int D>
__global__ void k_ad_inject(int na, const long long* __restrict__ act, int nc,
                            const double* __restrict__ cg, double* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= na) return;
  const long long ncp1 = nc + 1, nf1 = 3LL * nc + 1;
  long long v = act[j], idx = 0, stride = 1;
  for (int k = 0; k < D; ++k) {
    idx += 3LL * (v % ncp1) * stride;
    v /= ncp1;
    stride *= nf1;
  }
  g[j] -= cg[idx];
}

// y = alpha A x (+ y when accumulate) for a CSR matrix
__global__ void k_ad_spmv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                          const double* __restrict__ av, const double* __restrict__ x,
                          double alpha, int accumulate, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) acc += av[k] * x[ci[k]];
  y[i] = accumulate ? y[i] + alpha * acc : alpha * acc;
}

// x_j = r_l(act_j) / M_l,j (the exact damping equation's input)
__global__ void k_ad_scaled(int na, const long long* __restrict__ act,
                            const double* __restrict__ rg, const double* __restrict__ diag,
                            double* __restrict__ x) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < na) x[j] = rg[act[j]] / diag[j];
}

// exact damping equation: g_{l-1} -= omega~ b~ / M_{l-1}, b~ = omega y
__global__ void k_ad_damp_exact(int na, const double* __restrict__ y,
                                const double* __restrict__ diag, double omega, double omega_t,
                                double* __restrict__ bt, double* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= na) return;
  const double b = omega * y[j];
  bt[j] = b;
  g[j] -= omega_t * b / diag[j];
}

// the function of another tree's grid (leaf-node values uo, leaf flags per
// level, fine-position -> node map) at the leaf nodes of this tree: d-linear
// interpolation in the old leaf cell that holds each position
template <int D>
__global__ void k_ad_eval(int nn, const long long* __restrict__ nodes, int L, long long N1,
                          const unsigned char* __restrict__ leaf, const long long* __restrict__ loff,
                          const int* __restrict__ omap, const double* __restrict__ uo,
                          double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int q[3] = {0, 0, 0};
  long long g = nodes[i];
  for (int k = 0; k < D; ++k) {
    q[k] = (int)(g % N1);
    g /= N1;
  }
  double val = 0.0;
  long long s = N1 - 1, n = 1;
  for (int l = 1; l <= L; ++l) {
    s /= 3;
    n *= 3;
    int c[3] = {0, 0, 0};
    long long ci = 0, stride = 1;
    for (int k = 0; k < D; ++k) {
      c[k] = (int)min((long long)q[k] / s, n - 1);
      ci += c[k] * stride;
      stride *= n;
    }
    if (!leaf[loff[l] + ci]) continue;
    for (int a = 0; a < (1 << D); ++a) {
      double w = 1.0;
      long long p = 0, st = 1;
      for (int k = 0; k < D; ++k) {
        const int b = (a >> k) & 1;
        const double t = (double)(q[k] - s * c[k]) / (double)s;
        w *= b ? t : 1.0 - t;
        p += (s * (c[k] + b)) * st;
        st *= N1;
      }
      if (w != 0.0) val += w * uo[omap[p]];
    }
    break;
  }
  v[i] = val;
}

// the coefficients of one level's nodal-space vertices while the function is
// rebuilt from its vertex values: coef_j = v(p_j) - u(p_j)
__global__ void k_ad_coef(int nf, const int* __restrict__ fr, const int* __restrict__ frnode,
                          const double* __restrict__ v, const double* __restrict__ u,
                          double* __restrict__ coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nf) coef[fr[i]] = v[frnode[i]] - u[frnode[i]];
}

__global__ void k_ad_add(int n, const double* __restrict__ du, double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] += du[i];
}

// block sums of hD r_l^2 over the level's free vertices (Eq. 10)
__global__ void k_ad_norm(int nf, const int* __restrict__ fr, const long long* __restrict__ act,
                          const double* __restrict__ rg, double hD, double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    const double r = rg[act[fr[i]]];
    acc += r * r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    part[blockIdx.x] = hD * t;
  }
}

int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

// ---- host-side system ---------------------------------------------------------------

struct Csr {
  std::vector<int> rp, ci;
  std::vector<double> v;
};

}  // namespace
}  // namespace adafac

struct adafac_adaptive_s {
  int D = 0, L = 0, nn = 0;
  adafac_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  std::vector<long long> nodes;      // fine-grid index of every leaf node, ascending
  std::vector<int> node_map;         // fine position -> leaf node (-1: none)
  std::vector<unsigned char> leaf;   // leaf flags of every level's cells, levels 1 .. L
  std::vector<long long> leaf_off;   // offset of level l in leaf (index l)
  long long* d_nodes = nullptr;      // device copies for the transfer between trees
  int* d_node_map = nullptr;
  unsigned char* d_leaf = nullptr;
  long long* d_leaf_off = nullptr;
  std::vector<adafac::ad::Level> lev;  // 1 .. L
  adafac::ad::DevCsr K;
  adafac::ad::Stencil st{};
  double* d_b = nullptr;
  double* d_u = nullptr;
  double* d_rr = nullptr;
  double* d_du = nullptr;
  double* d_y = nullptr;             // scratch node vectors (exact R~)
  double* d_y2 = nullptr;
  double* d_part = nullptr;
  int npart = 0;
  double r0 = 0.0;
  std::vector<void*> allocs;
  // the brick engine (adaptive_brick.h) runs the cycles when it covers the
  // variant; the CSR arrays above are then not built
  bool brick = false;
  adafac::brick::System* bs = nullptr;
  // CUDA graphs of the brick engine's batches (key: kind, cycles, norm)
  std::map<long, cudaGraphExec_t> graphs;
  cudaStream_t cap = nullptr;
  bool use_graphs = true;
};

namespace adafac {
namespace {

adafac_status ad_fail(adafac_adaptive h, adafac_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

adafac_status ad_cuda(adafac_adaptive h, const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return ADAFAC_OK;
  return ad_fail(h, ADAFAC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
bool dev_copy(adafac_adaptive h, T** dst, const T* src, size_t count) {
  *dst = nullptr;
  if (count == 0) return true;
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return false;
  h->allocs.push_back(p);
  *dst = static_cast<T*>(p);
  if (src) return cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
  return cudaMemset(p, 0, count * sizeof(T)) == cudaSuccess;
}

bool upload_csr(adafac_adaptive h, const Csr& c, DevCsr* d) {
  d->rows = (int)c.rp.size() - 1;
  return dev_copy(h, &d->rp, c.rp.data(), c.rp.size()) &&
         dev_copy(h, &d->ci, c.ci.data(), c.ci.size()) &&
         dev_copy(h, &d->v, c.v.data(), c.v.size());
}

long long ipow(long long b, int e) {
  long long r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// element stiffness of the d-linear cell on the reference cell, by the
// Hamming distance of the two corners
double kref(int D, int ham) {
  if (D == 2) return ham == 0 ? 2.0 / 3.0 : (ham == 1 ? -1.0 / 6.0 : -1.0 / 3.0);
  return ham == 0 ? 1.0 / 3.0 : (ham == 1 ? 0.0 : -1.0 / 12.0);
}

void decode(long long v, long long np1, int D, int* c) {
  for (int k = 0; k < D; ++k) {
    c[k] = (int)(v % np1);
    v /= np1;
  }
}

long long encode(const int* c, long long np1, int D) {
  long long v = 0;
  for (int k = D - 1; k >= 0; --k) v = v * np1 + c[k];
  return v;
}

// the value at fine position q of the pagoda of width s centred at s v
double pagoda(const int* q, const int* v, int s, int D) {
  double w = 1.0;
  for (int k = 0; k < D; ++k) {
    const double t = 1.0 - std::fabs((double)(q[k] - s * v[k])) / s;
    if (t <= 0.0) return 0.0;
    w *= t;
  }
  return w;
}

adafac_status build(adafac_adaptive h, const uint8_t* const* refine, const double* eps,
                    int eps_scalar, const double* f) {
  const int D = h->D, L = h->L, NC = 1 << D;
  const long long N = ipow(3, L), N1 = N + 1, GF = ipow(N1, D);
  // cells of every level that exist / are cut (x fastest)
  std::vector<std::vector<uint8_t>> exists(L + 2), cut(L + 2);
  for (int l = 1; l <= L; ++l) {
    const long long n = ipow(3, l), cells = ipow(n, D);
    exists[l].assign(cells, 0);
    cut[l].assign(cells, 0);
    if (l == 1) std::fill(exists[l].begin(), exists[l].end(), 1);
    else {
      const long long np = n / 3;
      int c[3], pc[3];
      for (long long i = 0; i < cells; ++i) {
        decode(i, n, D, c);
        for (int k = 0; k < D; ++k) pc[k] = c[k] / 3;
        exists[l][i] = cut[l - 1][encode(pc, np, D)];
      }
    }
    if (l < L)
      for (long long i = 0; i < cells; ++i) cut[l][i] = exists[l][i] && refine[l - 1][i] ? 1 : 0;
  }
  // leaf nodes: every corner of a leaf cell, in fine-grid order
  std::vector<uint8_t> present(GF, 0);
  for (int l = 1; l <= L; ++l) {
    const long long n = ipow(3, l), cells = ipow(n, D), s = ipow(3, L - l);
    int c[3], q[3];
    for (long long i = 0; i < cells; ++i) {
      if (!exists[l][i] || cut[l][i]) continue;
      decode(i, n, D, c);
      for (int a = 0; a < NC; ++a) {
        for (int k = 0; k < D; ++k) q[k] = (int)(s * (c[k] + ((a >> k) & 1)));
        present[encode(q, N1, D)] = 1;
      }
    }
  }
  h->leaf_off.assign(L + 1, 0);
  h->leaf.clear();
  for (int l = 1; l <= L; ++l) {
    h->leaf_off[l] = (long long)h->leaf.size();
    for (size_t i = 0; i < exists[l].size(); ++i)
      h->leaf.push_back(exists[l][i] && !cut[l][i] ? 1 : 0);
  }
  std::vector<int>& node_id = h->node_map;
  node_id.assign(GF, -1);
  h->nodes.clear();
  for (long long g = 0; g < GF; ++g)
    if (present[g]) {
      node_id[g] = (int)h->nodes.size();
      h->nodes.push_back(g);
    }
  const int nn = (int)h->nodes.size();
  h->nn = nn;
  if (h->brick) {
    brick::Tree tree;
    tree.exists = std::move(exists);
    tree.cut = std::move(cut);
    h->bs = new (std::nothrow) brick::System();
    if (!h->bs) return ad_fail(h, ADAFAC_ERR_OOM, "brick engine: allocation failed");
    std::string why;
    const bool mixed = h->opt.precision == ADAFAC_PRECISION_MIXED;
    const adafac_status st =
        brick::build(*h->bs, D, L, tree, eps, eps_scalar, f, mixed, h->stream, &why);
    if (st != ADAFAC_OK) return ad_fail(h, st, why);
    if (!dev_copy(h, &h->d_u, (const double*)nullptr, nn) ||
        !dev_copy(h, &h->d_y, (const double*)nullptr, nn) ||
        !dev_copy(h, &h->d_nodes, h->nodes.data(), h->nodes.size())) {
      cudaGetLastError();
      return ad_fail(h, ADAFAC_ERR_OOM, "device allocation or copy failed");
    }
    return ADAFAC_OK;
  }
  // leaf stiffness (eps of a leaf cell: the mean of the fine cells it covers)
  // and lumped load (each corner of a leaf cell of width hc takes hc^D / 2^D f)
  struct Trip {
    int r, c;
    double v;
  };
  std::vector<Trip> trips;
  std::vector<double> b(nn, 0.0);
  for (int l = 1; l <= L; ++l) {
    const long long n = ipow(3, l), cells = ipow(n, D), s = ipow(3, L - l);
    const double hc = 1.0 / (double)n, scale = std::pow(hc, D - 2), load = std::pow(hc, D) / NC;
    int c[3], q[3], ids[8];
    for (long long i = 0; i < cells; ++i) {
      if (!exists[l][i] || cut[l][i]) continue;
      decode(i, n, D, c);
      double e;
      if (eps_scalar) {
        e = eps[0];
      } else {
        double acc = 0.0;
        const long long cnt = ipow(s, D);
        int fc[3];
        for (long long m = 0; m < cnt; ++m) {
          long long t = m;
          for (int k = 0; k < D; ++k) {
            fc[k] = (int)(s * c[k] + t % s);
            t /= s;
          }
          acc += eps[encode(fc, N, D)];
        }
        e = acc / (double)cnt;
      }
      for (int a = 0; a < NC; ++a) {
        for (int k = 0; k < D; ++k) q[k] = (int)(s * (c[k] + ((a >> k) & 1)));
        const long long g = encode(q, N1, D);
        ids[a] = node_id[g];
        b[ids[a]] += load * (f ? f[g] : 0.0);
      }
      for (int a = 0; a < NC; ++a)
        for (int bb = 0; bb < NC; ++bb) {
          const double kv = e * scale * kref(D, __builtin_popcount(a ^ bb));
          if (kv != 0.0) trips.push_back({ids[a], ids[bb], kv});
        }
    }
  }
  std::sort(trips.begin(), trips.end(),
            [](const Trip& x, const Trip& y) { return x.r != y.r ? x.r < y.r : x.c < y.c; });
  Csr K;
  K.rp.assign(nn + 1, 0);
  for (size_t i = 0; i < trips.size();) {
    size_t j = i;
    double acc = 0.0;
    while (j < trips.size() && trips[j].r == trips[i].r && trips[j].c == trips[i].c) acc += trips[j++].v;
    K.ci.push_back(trips[i].c);
    K.v.push_back(acc);
    K.rp[trips[i].r + 1]++;
    i = j;
  }
  for (int i = 0; i < nn; ++i) K.rp[i + 1] += K.rp[i];
  trips.clear();
  trips.shrink_to_fit();
  // levels: active vertices, pagodas at the leaf nodes, diagonals
  std::vector<int> finest(nn, 0), finest_id(nn, -1);
  h->lev.assign(L + 1, Level());
  std::vector<std::vector<int>> act_id(L + 1);
  std::vector<Csr> phi(L + 1), phit(L + 1);
  for (int l = 1; l <= L; ++l) {
    Level& lv = h->lev[l];
    const int n = (int)ipow(3, l), s = (int)ipow(3, L - l);
    lv.n = n;
    lv.G = ipow(n + 1, D);
    act_id[l].assign(lv.G, -1);
    int v[3], cc[3];
    for (long long g = 0; g < lv.G; ++g) {
      decode(g, n + 1, D, v);
      bool ok = true;
      for (int k = 0; k < D; ++k) ok = ok && v[k] >= 1 && v[k] <= n - 1;
      for (int a = 0; ok && a < NC; ++a) {
        for (int k = 0; k < D; ++k) cc[k] = v[k] - ((a >> k) & 1);
        ok = exists[l][encode(cc, n, D)] != 0;
      }
      if (ok) {
        act_id[l][g] = (int)lv.act.size();
        lv.act.push_back(g);
      }
    }
    lv.na = (int)lv.act.size();
    // Phi_l: a leaf node q lies in the level cell min(q / s, n - 1); only the
    // pagodas of that cell's corners reach it
    Csr& P = phi[l];
    P.rp.assign(nn + 1, 0);
    int q[3];
    for (int p = 0; p < nn; ++p) {
      decode(h->nodes[p], N1, D, q);
      int cell[3];
      for (int k = 0; k < D; ++k) cell[k] = std::min(q[k] / s, n - 1);
      for (int a = 0; a < NC; ++a) {
        for (int k = 0; k < D; ++k) v[k] = cell[k] + ((a >> k) & 1);
        const int j = act_id[l][encode(v, n + 1, D)];
        if (j < 0) continue;
        const double w = pagoda(q, v, s, D);
        if (w <= 0.0) continue;
        P.ci.push_back(j);
        P.v.push_back(w);
      }
      P.rp[p + 1] = (int)P.ci.size();
    }
    // Phi_l^T by columns
    Csr& T = phit[l];
    T.rp.assign(lv.na + 1, 0);
    for (int j : P.ci) T.rp[j + 1]++;
    for (int j = 0; j < lv.na; ++j) T.rp[j + 1] += T.rp[j];
    T.ci.resize(P.ci.size());
    T.v.resize(P.v.size());
    for (int j = 0; j < lv.na; ++j) lv.phit_max = std::max(lv.phit_max, T.rp[j + 1] - T.rp[j]);
    std::vector<int> fill(T.rp.begin(), T.rp.end() - 1);
    for (int p = 0; p < nn; ++p)
      for (int k = P.rp[p]; k < P.rp[p + 1]; ++k) {
        const int at = fill[P.ci[k]]++;
        T.ci[at] = p;
        T.v[at] = P.v[k];
      }
    // M_l = diag(Phi_l^T K Phi_l): sum over the support p of vertex j and
    // over the row of K at p
    lv.diag.assign(lv.na, 0.0);
    for (int j = 0; j < lv.na; ++j) {
      decode(lv.act[j], n + 1, D, v);
      double acc = 0.0;
      for (int k = T.rp[j]; k < T.rp[j + 1]; ++k) {
        const int p = T.ci[k];
        double row = 0.0;
        for (int m = K.rp[p]; m < K.rp[p + 1]; ++m) {
          decode(h->nodes[K.ci[m]], N1, D, q);
          row += K.v[m] * pagoda(q, v, s, D);
        }
        acc += T.v[k] * row;
      }
      lv.diag[j] = acc;
      if (!(acc > 0.0)) return ad_fail(h, ADAFAC_ERR_INVALID_ARG, "non-positive level diagonal");
    }
    // the nodal space's vertices: every active position on its finest level
    for (int j = 0; j < lv.na; ++j) {
      decode(lv.act[j], n + 1, D, v);
      for (int k = 0; k < D; ++k) q[k] = s * v[k];
      const int p = node_id[encode(q, N1, D)];
      if (p < 0) return ad_fail(h, ADAFAC_ERR_INVALID_ARG, "active vertex without a leaf node");
      finest[p] = l;
      finest_id[p] = j;
    }
  }
  for (int p = 0; p < nn; ++p)
    if (finest[p] > 0) {
      h->lev[finest[p]].fr.push_back(finest_id[p]);
      h->lev[finest[p]].frnode.push_back(p);
    }
  // device arrays
  bool ok = upload_csr(h, K, &h->K) && dev_copy(h, &h->d_b, b.data(), nn) &&
            dev_copy(h, &h->d_u, (const double*)nullptr, nn) &&
            dev_copy(h, &h->d_rr, (const double*)nullptr, nn) &&
            dev_copy(h, &h->d_du, (const double*)nullptr, nn) &&
            dev_copy(h, &h->d_y, (const double*)nullptr, nn) &&
            dev_copy(h, &h->d_y2, (const double*)nullptr, nn);
  int most = 1;
  for (int l = 1; ok && l <= L; ++l) {
    Level& lv = h->lev[l];
    ok = upload_csr(h, phi[l], &lv.phi) && upload_csr(h, phit[l], &lv.phit) &&
         dev_copy(h, &lv.d_act, lv.act.data(), lv.act.size()) &&
         dev_copy(h, &lv.d_fr, lv.fr.data(), lv.fr.size()) &&
         dev_copy(h, &lv.d_frnode, lv.frnode.data(), lv.frnode.size()) &&
         dev_copy(h, &lv.d_diag, lv.diag.data(), lv.diag.size()) &&
         dev_copy(h, &lv.d_rg, (const double*)nullptr, (size_t)lv.G) &&
         dev_copy(h, &lv.d_cg, (const double*)nullptr, (size_t)lv.G) &&
         dev_copy(h, &lv.d_g, (const double*)nullptr, (size_t)lv.na) &&
         dev_copy(h, &lv.d_bt, (const double*)nullptr, (size_t)lv.na) &&
         dev_copy(h, &lv.d_x, (const double*)nullptr, (size_t)lv.na);
    most = std::max(most, std::min(blocks_for((long long)lv.fr.size()), 1024));
  }
  h->npart = most * L;
  ok = ok && dev_copy(h, &h->d_part, (const double*)nullptr, (size_t)h->npart) &&
       dev_copy(h, &h->d_nodes, h->nodes.data(), h->nodes.size());
  if (!ok) {
    cudaGetLastError();
    return ad_fail(h, ADAFAC_ERR_OOM, "device allocation or copy failed");
  }
  smoothed_restriction_stencil(D, h->st.w);
  return ADAFAC_OK;
}

// r_l = Phi_l^T rr (with the Jacobi step): a thread, a warp or a block per
// active vertex, by the longest pagoda of the level
void launch_level_restrict(const Level& lv, const double* rr, double omega, double scale,
                           bool corrections, cudaStream_t s) {
  double* cg = corrections ? lv.d_cg : nullptr;
  double* g = corrections ? lv.d_g : nullptr;
  if (lv.phit_max > 1024)
    k_ad_restrict_wide<kThreads><<<lv.na, kThreads, 0, s>>>(lv.na, lv.phit.rp, lv.phit.ci,
                                                             lv.phit.v, rr, lv.d_act, lv.d_diag,
                                                             omega, scale, lv.d_rg, cg, g);
  else if (lv.phit_max > 32)
    k_ad_restrict_wide<32><<<(lv.na + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, s>>>(
        lv.na, lv.phit.rp, lv.phit.ci, lv.phit.v, rr, lv.d_act, lv.d_diag, omega, scale, lv.d_rg,
        cg, g);
  else
    k_ad_restrict<<<blocks_for(lv.na), kThreads, 0, s>>>(lv.na, lv.phit.rp, lv.phit.ci,
                                                          lv.phit.v, rr, lv.d_act, lv.d_diag,
                                                          omega, scale, lv.d_rg, cg, g);
}

// y = Phi_l^T x over the active ids of a level, by its longest row
void launch_level_phit(const Level& lv, const double* x, double* y, cudaStream_t s) {
  if (lv.phit_max > 1024)
    k_ad_spmv_wide<kThreads><<<lv.na, kThreads, 0, s>>>(lv.na, lv.phit.rp, lv.phit.ci, lv.phit.v,
                                                         x, y);
  else if (lv.phit_max > 32)
    k_ad_spmv_wide<32><<<(lv.na + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, s>>>(
        lv.na, lv.phit.rp, lv.phit.ci, lv.phit.v, x, y);
  else
    k_ad_spmv<<<blocks_for(lv.na), kThreads, 0, s>>>(lv.na, lv.phit.rp, lv.phit.ci, lv.phit.v, x,
                                                      1.0, 0, y);
}

// r_l of every level lmin .. L from the current u (and the Jacobi steps)
void level_residuals(adafac_adaptive h, int lmin, bool corrections) {
  cudaStream_t s = h->stream;
  const int nn = h->nn;
  k_ad_residual<<<blocks_for(nn), kThreads, 0, s>>>(nn, h->K.rp, h->K.ci, h->K.v, h->d_b, h->d_u,
                                                     h->d_rr);
  const adafac_options& o = h->opt;
  for (int l = lmin; l <= h->L; ++l) {
    Level& lv = h->lev[l];
    if (lv.na == 0) continue;
    const double scale = o.variant == ADAFAC_VARIANT_EXP ? std::pow(o.omega_exp, h->L - l) : 1.0;
    launch_level_restrict(lv, h->d_rr, o.omega, scale, corrections, s);
  }
}

void enqueue_cycle(adafac_adaptive h) {
  cudaStream_t s = h->stream;
  const adafac_options& o = h->opt;
  const int L = h->L, lmin = o.lmin, nn = h->nn;
  level_residuals(h, lmin, true);
  for (int l = lmin + 1; l <= L; ++l) {
    Level& f = h->lev[l];
    Level& c = h->lev[l - 1];
    if (c.na == 0) continue;
    if (o.variant == ADAFAC_VARIANT_JAC) {
      if (o.rtilde == ADAFAC_RTILDE_EXACT) {
        // b~ = omega Phi_{l-1}^T K Phi_l M_l^-1 r_l
        if (f.na > 0) {
          k_ad_scaled<<<blocks_for(f.na), kThreads, 0, s>>>(f.na, f.d_act, f.d_rg, f.d_diag, f.d_x);
          k_ad_spmv<<<blocks_for(nn), kThreads, 0, s>>>(nn, f.phi.rp, f.phi.ci, f.phi.v, f.d_x, 1.0,
                                                          0, h->d_y);
        } else {
          cudaMemsetAsync(h->d_y, 0, sizeof(double) * nn, s);
        }
        k_ad_spmv<<<blocks_for(nn), kThreads, 0, s>>>(nn, h->K.rp, h->K.ci, h->K.v, h->d_y, 1.0, 0,
                                                        h->d_y2);
        launch_level_phit(c, h->d_y2, c.d_x, s);
        k_ad_damp_exact<<<blocks_for(c.na), kThreads, 0, s>>>(c.na, c.d_x, c.d_diag, o.omega,
                                                                o.omega_tilde, c.d_bt, c.d_g);
      } else if (h->D == 2) {
        k_ad_damp<2><<<blocks_for(c.na), kThreads, 0, s>>>(c.na, c.d_act, c.n, f.d_rg, c.d_diag,
                                                             h->st, o.omega, o.omega_tilde, c.d_bt,
                                                             c.d_g);
      } else {
        k_ad_damp<3><<<blocks_for(c.na), kThreads, 0, s>>>(c.na, c.d_act, c.n, f.d_rg, c.d_diag,
                                                             h->st, o.omega, o.omega_tilde, c.d_bt,
                                                             c.d_g);
      }
    } else if (o.variant == ADAFAC_VARIANT_PI) {
      if (h->D == 2)
        k_ad_inject<2><<<blocks_for(c.na), kThreads, 0, s>>>(c.na, c.d_act, c.n, f.d_cg, c.d_g);
      else
        k_ad_inject<3><<<blocks_for(c.na), kThreads, 0, s>>>(c.na, c.d_act, c.n, f.d_cg, c.d_g);
    }
  }
  // du = sum_l Phi_l g_l, u += du
  bool first = true;
  for (int l = lmin; l <= L; ++l) {
    Level& lv = h->lev[l];
    if (lv.na == 0) continue;
    k_ad_spmv<<<blocks_for(nn), kThreads, 0, s>>>(nn, lv.phi.rp, lv.phi.ci, lv.phi.v, lv.d_g, 1.0,
                                                    first ? 0 : 1, h->d_du);
    first = false;
  }
  if (!first) k_ad_add<<<blocks_for(nn), kThreads, 0, s>>>(nn, h->d_du, h->d_u);
}

// ||b - K u||_h over the nodal space's vertices (Eq. 10); synchronises
adafac_status norm(adafac_adaptive h, double* out) {
  if (h->brick) {
    brick::enqueue_norm(*h->bs, h->stream);
    brick::Ctl c;
    if (cudaMemcpyAsync(&c, h->bs->ctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return ad_cuda(h, "norm");
    *out = c.abs;
    return ad_cuda(h, "norm");
  }
  level_residuals(h, 1, false);
  int off = 0;
  std::vector<int> used;
  for (int l = 1; l <= h->L; ++l) {
    Level& lv = h->lev[l];
    const int nf = (int)lv.fr.size();
    if (nf == 0) continue;
    const int nb = std::min(blocks_for(nf), 1024);
    const double hD = std::pow(1.0 / (double)lv.n, h->D);
    k_ad_norm<<<nb, kThreads, 0, h->stream>>>(nf, lv.d_fr, lv.d_act, lv.d_rg, hD, h->d_part + off);
    off += nb;
  }
  std::vector<double> part(off);
  if (off > 0 && cudaMemcpyAsync(part.data(), h->d_part, sizeof(double) * off,
                                 cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return ad_cuda(h, "norm copy");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return ad_cuda(h, "norm");
  double acc = 0.0;
  for (double v : part) acc += v;
  *out = std::sqrt(acc);
  return ad_cuda(h, "norm");
}

void release(adafac_adaptive h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->bs) {
    brick::release(*h->bs);
    delete h->bs;
    h->bs = nullptr;
  }
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  if (h->cap) cudaStreamDestroy(h->cap);
  h->cap = nullptr;
}

// Replays `enqueue` (launches on the stream it is given) as a CUDA graph
// captured once per key; launches directly when capture is unavailable.
template <typename F>
void run_graph(adafac_adaptive h, long key, F&& enqueue) {
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaGraphExec_t ex = nullptr;
    bool ok = h->use_graphs &&
              (h->cap || cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) == cudaSuccess);
    if (ok) ok = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      enqueue(h->cap);
      cudaGraph_t g = nullptr;
      ok = cudaStreamEndCapture(h->cap, &g) == cudaSuccess &&
           cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
    }
    if (!ok) {
      cudaGetLastError();
      h->use_graphs = false;
      enqueue(h->stream);
      return;
    }
    it = h->graphs.emplace(key, ex).first;
  }
  cudaGraphLaunch(it->second, h->stream);
}

// brick engine: n FP64 cycles, or a refinement step of n cycles (MIXED)
void brick_batch(adafac_adaptive h, int n, bool with_norm) {
  const bool mixed = h->bs->mixed;
  const long key = ((long)n << 2) | (with_norm ? 2 : 0) | (mixed ? 1 : 0);
  run_graph(h, key, [&](cudaStream_t s) {
    if (mixed) brick::enqueue_step(*h->bs, h->opt, n, with_norm, s);
    else
      for (int i = 0; i < n; ++i) brick::enqueue_cycle(*h->bs, h->opt, with_norm, s);
  });
}

// r0 of the brick engine's control block follows the host's
adafac_status set_r0(adafac_adaptive h, double r0) {
  h->r0 = r0;
  if (!h->brick) return ADAFAC_OK;
  if (cudaMemcpyAsync(&h->bs->ctl->r0, &h->r0, sizeof(double), cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return ad_cuda(h, "r0");
  return ADAFAC_OK;
}

// the iterate at the leaf nodes (the brick engine gathers it from its levels)
adafac_status sync_nodes(adafac_adaptive h) {
  if (!h->brick) return ADAFAC_OK;
  brick::gather_nodes(*h->bs, h->d_nodes, h->nn, h->d_u, h->stream);
  return ad_cuda(h, "gather");
}

}  // namespace
}  // namespace adafac

extern "C" {

adafac_status adafac_adaptive_setup(int dim, int depth, const uint8_t* const* refine,
                                    const double* eps, int eps_is_scalar, const double* f,
                                    const adafac_options* opt, void* stream,
                                    adafac_adaptive* out) {
  using namespace adafac;
  if (!out) return ADAFAC_ERR_INVALID_ARG;
  *out = nullptr;
  if ((dim != 2 && dim != 3) || depth < 1 || !opt || !eps || (depth > 1 && !refine))
    return ADAFAC_ERR_INVALID_ARG;
  if (ipow(ipow(3, depth) + 1, dim) > (1LL << 31) - 1) return ADAFAC_ERR_INVALID_ARG;
  const bool brick_engine =
      opt->path != ADAFAC_PATH_GENERIC &&
      !(opt->variant == ADAFAC_VARIANT_JAC && opt->rtilde == ADAFAC_RTILDE_EXACT);
  // MIXED precision (FP32 cycles, FP64 refinement steps) runs on the brick engine
  if ((opt->precision != ADAFAC_PRECISION_FP64 &&
       !(opt->precision == ADAFAC_PRECISION_MIXED && brick_engine)) ||
      opt->inner_cycles < 1 || opt->transfer != ADAFAC_TRANSFER_DLINEAR ||
      opt->coarse_op != ADAFAC_COARSE_GALERKIN || opt->variant < 0 || opt->variant > 3 ||
      opt->lmin < 1 || opt->lmin > depth || !(opt->omega > 0.0) || !(opt->omega_tilde > 0.0))
    return ADAFAC_ERR_INVALID_ARG;
  for (int l = 1; l < depth; ++l)
    if (!refine[l - 1]) return ADAFAC_ERR_INVALID_ARG;
  const long long ncells = ipow(ipow(3, depth), dim);
  for (long long i = 0; i < (eps_is_scalar ? 1 : ncells); ++i)
    if (!(eps[i] > 0.0) || !std::isfinite(eps[i])) return ADAFAC_ERR_INVALID_ARG;
  adafac_adaptive h = new (std::nothrow) adafac_adaptive_s();
  if (!h) return ADAFAC_ERR_OOM;
  h->D = dim;
  h->L = depth;
  h->opt = *opt;
  h->stream = static_cast<cudaStream_t>(stream);
  // the brick engine covers every variant but the exact R~ of Jac; path
  // GENERIC keeps the CSR engine
  h->brick = brick_engine;
  adafac_status st = build(h, refine, eps, eps_is_scalar, f);
  double r0 = 0.0;
  if (st == ADAFAC_OK) st = norm(h, &r0);
  if (st == ADAFAC_OK) st = set_r0(h, r0);
  if (st != ADAFAC_OK) {
    release(h);
    delete h;
    return st;
  }
  *out = h;
  return ADAFAC_OK;
}

adafac_status adafac_adaptive_cycle(adafac_adaptive h, int n_cycles) {
  using namespace adafac;
  if (!h || n_cycles < 0) return ADAFAC_ERR_INVALID_ARG;
  if (h->brick) {
    // FP64: one graph of the n cycles; MIXED: refinement steps of
    // inner_cycles FP32 cycles
    const int batch = h->bs->mixed ? h->opt.inner_cycles : n_cycles;
    for (int done = 0; done < n_cycles;) {
      const int k = std::min(batch, n_cycles - done);
      brick_batch(h, k, false);
      done += k;
    }
    return ad_cuda(h, "cycle");
  }
  for (int i = 0; i < n_cycles; ++i) {
    if (h->brick) brick::enqueue_cycle(*h->bs, h->opt, false, h->stream);
    else enqueue_cycle(h);
  }
  return ad_cuda(h, "cycle");
}

adafac_status adafac_adaptive_residual_norm(adafac_adaptive h, double* rel, double* abs_) {
  using namespace adafac;
  if (!h) return ADAFAC_ERR_INVALID_ARG;
  double a = 0.0;
  adafac_status st = norm(h, &a);
  if (st != ADAFAC_OK) return st;
  if (abs_) *abs_ = a;
  if (rel) *rel = h->r0 > 0.0 ? a / h->r0 : 0.0;
  return ADAFAC_OK;
}

adafac_status adafac_adaptive_solve(adafac_adaptive h, double rel_tol, int max_cycles,
                                    int* cycles_done, double* rel) {
  using namespace adafac;
  if (!h || max_cycles < 0) return ADAFAC_ERR_INVALID_ARG;
  if (h->brick) {
    // every cycle evaluates the norm of its residual first; the cycles after
    // the one that meets rel_tol return at entry, and the host reads the
    // control block after every batch of cycles
    brick::Ctl c0;
    if (cudaMemcpyAsync(&c0, h->bs->ctl, sizeof(c0), cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return ad_cuda(h, "solve");
    brick::Ctl c = c0;
    c.tol = rel_tol;
    c.done = 0;
    c.diverged = 0;
    if (cudaMemcpyAsync(h->bs->ctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream) !=
        cudaSuccess)
      return ad_cuda(h, "solve");
    int enq = 0;
    const bool mixed = h->bs->mixed;
    while (enq < max_cycles && !c.done && !c.diverged) {
      const int k = std::min(mixed ? h->opt.inner_cycles : 8, max_cycles - enq);
      brick_batch(h, k, true);
      enq += k;
      if (cudaMemcpyAsync(&c, h->bs->ctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess)
        return ad_cuda(h, "solve");
    }
    const int applied = c.applied - c0.applied;
    double r = c.rel;
    if (!c.done && !c.diverged) {
      // the norm of the final iterate
      double a = 0.0;
      adafac_status st = norm(h, &a);
      if (st != ADAFAC_OK) return st;
      r = h->r0 > 0.0 ? a / h->r0 : 0.0;
    }
    c.tol = -1.0;
    c.done = 0;
    if (cudaMemcpyAsync(&h->bs->ctl->tol, &c.tol, sizeof(double), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(&h->bs->ctl->done, &c.done, sizeof(int), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return ad_cuda(h, "solve");
    if (cycles_done) *cycles_done = applied;
    if (rel) *rel = r;
    if (c.diverged || !std::isfinite(r) || r > 1e6) return ADAFAC_ERR_DIVERGED;
    return r <= rel_tol ? ADAFAC_OK : ADAFAC_ERR_NOT_CONVERGED;
  }
  double r = 1.0;
  int c = 0;
  adafac_status st = adafac_adaptive_residual_norm(h, &r, nullptr);
  while (st == ADAFAC_OK && r > rel_tol && c < max_cycles) {
    enqueue_cycle(h);
    ++c;
    st = adafac_adaptive_residual_norm(h, &r, nullptr);
    if (st == ADAFAC_OK && (!std::isfinite(r) || r > 1e6)) st = ADAFAC_ERR_DIVERGED;
  }
  if (cycles_done) *cycles_done = c;
  if (rel) *rel = r;
  if (st == ADAFAC_OK && r > rel_tol) st = ADAFAC_ERR_NOT_CONVERGED;
  return st;
}

adafac_status adafac_adaptive_nodes(adafac_adaptive h, int64_t* idx, int64_t* count) {
  if (!h || !count) return ADAFAC_ERR_INVALID_ARG;
  *count = (int64_t)h->nodes.size();
  if (idx)
    for (size_t i = 0; i < h->nodes.size(); ++i) idx[i] = h->nodes[i];
  return ADAFAC_OK;
}

adafac_status adafac_adaptive_solution(adafac_adaptive h, double* dst) {
  using namespace adafac;
  if (!h || !dst) return ADAFAC_ERR_INVALID_ARG;
  adafac_status st = sync_nodes(h);
  if (st != ADAFAC_OK) return st;
  if (cudaMemcpyAsync(dst, h->d_u, sizeof(double) * h->nn, cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return ad_cuda(h, "solution");
  return ADAFAC_OK;
}

adafac_status adafac_adaptive_set_solution(adafac_adaptive h, const double* src) {
  using namespace adafac;
  if (!h || !src) return ADAFAC_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(h->d_u, src, sizeof(double) * h->nn, cudaMemcpyHostToDevice, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return ad_cuda(h, "set solution");
  if (h->brick) brick::scatter_nodes(*h->bs, h->d_nodes, h->nn, h->d_u, h->stream);
  double r0 = 0.0;
  adafac_status st = adafac_adaptive_residual_norm(h, nullptr, &r0);
  if (st != ADAFAC_OK) return st;
  return set_r0(h, r0);
}

adafac_status adafac_adaptive_level(adafac_adaptive h, int field, int level, double* dst,
                                    int64_t* count) {
  using namespace adafac;
  if (!h || !count || level < 1 || level > h->L) return ADAFAC_ERR_INVALID_ARG;
  if (h->brick) {
    // the level's bricks, read at its active vertices (1 / M_l > 0)
    const brick::Level& bl = h->bs->lev[level];
    if (field != ADAFAC_FIELD_ACTIVE && field != ADAFAC_FIELD_R && field != ADAFAC_FIELD_BT &&
        field != ADAFAC_FIELD_G && field != ADAFAC_FIELD_INVDIAG)
      return ADAFAC_ERR_INVALID_ARG;
    std::vector<double> im(bl.V), vals;
    const double* src = field == ADAFAC_FIELD_R ? bl.R
                        : field == ADAFAC_FIELD_BT ? bl.BT
                        : field == ADAFAC_FIELD_G ? bl.G
                                                  : nullptr;
    if (src) vals.assign(bl.V, 0.0);
    if (cudaMemcpyAsync(im.data(), bl.IM, sizeof(double) * bl.V, cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess ||
        (src && cudaMemcpyAsync(vals.data(), src, sizeof(double) * bl.V, cudaMemcpyDeviceToHost,
                                h->stream) != cudaSuccess) ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return ad_cuda(h, "level field");
    int64_t k = 0;
    for (long long v = 0; v < bl.V; ++v) {
      if (!(im[v] > 0.0)) continue;
      if (dst) {
        if (field == ADAFAC_FIELD_ACTIVE) dst[k] = (double)v;
        else if (field == ADAFAC_FIELD_INVDIAG) dst[k] = im[v];
        else dst[k] = vals.empty() ? 0.0 : vals[v];
      }
      ++k;
    }
    *count = k;
    return ADAFAC_OK;
  }
  ad::Level& lv = h->lev[level];
  if (field == ADAFAC_FIELD_ACTIVE) {
    *count = lv.na;
    if (dst)
      for (int j = 0; j < lv.na; ++j) dst[j] = (double)lv.act[j];
    return ADAFAC_OK;
  }
  if (field != ADAFAC_FIELD_R && field != ADAFAC_FIELD_BT && field != ADAFAC_FIELD_G &&
      field != ADAFAC_FIELD_INVDIAG)
    return ADAFAC_ERR_INVALID_ARG;
  *count = lv.na;
  if (!dst || lv.na == 0) return ADAFAC_OK;
  std::vector<double> tmp;
  const double* src = nullptr;
  if (field == ADAFAC_FIELD_R) {
    tmp.resize(lv.G);
    if (cudaMemcpyAsync(tmp.data(), lv.d_rg, sizeof(double) * lv.G, cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return ad_cuda(h, "level field");
    for (int j = 0; j < lv.na; ++j) dst[j] = tmp[lv.act[j]];
    return ADAFAC_OK;
  }
  if (field == ADAFAC_FIELD_INVDIAG) {
    for (int j = 0; j < lv.na; ++j) dst[j] = 1.0 / lv.diag[j];
    return ADAFAC_OK;
  }
  src = field == ADAFAC_FIELD_BT ? lv.d_bt : lv.d_g;
  if (cudaMemcpyAsync(dst, src, sizeof(double) * lv.na, cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return ad_cuda(h, "level field");
  return ADAFAC_OK;
}

adafac_status adafac_adaptive_transfer(adafac_adaptive dst, adafac_adaptive src) {
  using namespace adafac;
  if (!dst || !src || dst->D != src->D || dst->L != src->L) return ADAFAC_ERR_INVALID_ARG;
  if (sync_nodes(src) != ADAFAC_OK) return ad_fail(dst, ADAFAC_ERR_CUDA, "transfer: source gather");
  if (src->stream && cudaStreamSynchronize(src->stream) != cudaSuccess)
    return ad_cuda(dst, "transfer: source stream");
  // the source grid's leaf flags and node map, on the device once (each on
  // its own: a handle that was a transfer target already has its node map)
  if ((!src->d_node_map &&
       !dev_copy(src, &src->d_node_map, src->node_map.data(), src->node_map.size())) ||
      (!src->d_leaf && !dev_copy(src, &src->d_leaf, src->leaf.data(), src->leaf.size())) ||
      (!src->d_leaf_off &&
       !dev_copy(src, &src->d_leaf_off, src->leaf_off.data(), src->leaf_off.size())) ||
      !src->d_node_map || !src->d_leaf || !src->d_leaf_off) {
    cudaGetLastError();
    return ad_fail(dst, ADAFAC_ERR_OOM, "transfer: device allocation failed");
  }
  cudaStream_t s = dst->stream;
  const int nn = dst->nn;
  const long long N1 = ipow(3, dst->L) + 1;
  // v: the old function at the new leaf nodes (kept in d_y)
  if (dst->D == 2)
    k_ad_eval<2><<<blocks_for(nn), kThreads, 0, s>>>(nn, dst->d_nodes, dst->L, N1, src->d_leaf,
                                                       src->d_leaf_off, src->d_node_map, src->d_u,
                                                       dst->d_y);
  else
    k_ad_eval<3><<<blocks_for(nn), kThreads, 0, s>>>(nn, dst->d_nodes, dst->L, N1, src->d_leaf,
                                                       src->d_leaf_off, src->d_node_map, src->d_u,
                                                       dst->d_y);
  // the function of the new space with those values at the nodal-space
  // vertices (zero Dirichlet data): level by level from the coarsest, each
  // level's pagodas add what the coarser ones left over at its vertices
  if (dst->brick) {
    if (!dst->d_node_map &&
        !dev_copy(dst, &dst->d_node_map, dst->node_map.data(), dst->node_map.size())) {
      cudaGetLastError();
      return ad_fail(dst, ADAFAC_ERR_OOM, "transfer: device allocation failed");
    }
    brick::from_node_values(*dst->bs, dst->d_node_map, dst->d_y, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ad_cuda(dst, "transfer");
    return set_r0(dst, src->r0);
  }
  cudaMemsetAsync(dst->d_u, 0, sizeof(double) * nn, s);
  for (int l = 1; l <= dst->L; ++l) {
    ad::Level& lv = dst->lev[l];
    const int nf = (int)lv.fr.size();
    if (nf == 0) continue;
    cudaMemsetAsync(lv.d_x, 0, sizeof(double) * lv.na, s);
    k_ad_coef<<<blocks_for(nf), kThreads, 0, s>>>(nf, lv.d_fr, lv.d_frnode, dst->d_y, dst->d_u,
                                                   lv.d_x);
    k_ad_spmv<<<blocks_for(nn), kThreads, 0, s>>>(nn, lv.phi.rp, lv.phi.ci, lv.phi.v, lv.d_x, 1.0, 1,
                                                    dst->d_u);
  }
  dst->r0 = src->r0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ad_cuda(dst, "transfer");
  return ad_cuda(dst, "transfer");
}

const char* adafac_adaptive_last_error(adafac_adaptive h) { return h ? h->err.c_str() : ""; }

adafac_status adafac_adaptive_destroy(adafac_adaptive h) {
  if (!h) return ADAFAC_OK;
  adafac::release(h);
  delete h;
  return ADAFAC_OK;
}

}  // extern "C"
