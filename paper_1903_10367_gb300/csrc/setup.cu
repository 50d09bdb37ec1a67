// Setup kernels (FP64): load vector, fine inverse diagonal, BoxMG
// prolongation, cell-wise Galerkin coarse operators and stencil assembly.
// All run once per solve; one thread per vertex or per coarse cell.
#include "common.cuh"

namespace adafac {

namespace {

constexpr int kThreads = 128;

inline int blocks_for(long long n, int threads = kThreads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > (1LL << 30) ? (1LL << 30) : b));
}

// Load vector b = h^D f at interior vertices (lumped mass), 0 on the boundary.
template <int D>
__global__ void k_rhs(const double* __restrict__ f, double* __restrict__ b, int n) {
  const int np1 = n + 1;
  long long V = 1;
  for (int j = 0; j < D; ++j) V *= np1;
  const double h = 1.0 / n;
  double hD = 1.0;
  for (int j = 0; j < D; ++j) hD *= h;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D];
    decode<D>(v, np1, c);
    b[v] = (f && is_interior<D>(c, n)) ? hD * f[v] : 0.0;
  }
}

// Stencil entry s of vertex c of the fine level (from eps or uniform).
template <int D>
__device__ double fine_stencil_entry(const LevelView<double>& lv, const int* c, int s) {
  if (lv.opkind == OP_UNIFORM) return lv.cst[s];
  if (lv.opkind == OP_STORED) {
    return lv.st[(long long)s * lv.V + encode<D>(c, lv.np1)];
  }
  constexpr int NC = 1 << D;
  int o[D];
  int t = s;
  for (int j = 0; j < D; ++j) {
    o[j] = t % 3 - 1;
    t /= 3;
  }
  double acc = 0.0;
  for (int a = 0; a < NC; ++a) {
    int cell[D], bbits = 0;
    bool ok = true;
    for (int j = 0; j < D; ++j) {
      const int aj = (a >> j) & 1;
      cell[j] = c[j] - aj;
      if (cell[j] < 0 || cell[j] >= lv.n) ok = false;
      const int bj = aj + o[j];
      if (bj < 0 || bj > 1) ok = false;
      bbits |= (bj & 1) << j;
    }
    if (!ok) continue;
    acc += lv.eps[encode<D>(cell, lv.n)] * kref<D, double>(__popc(a ^ bbits));
  }
  return lv.hfac * acc;
}

// All 3^D stencil entries of vertex c at once: every cell a containing c (as
// its corner a) adds eps_cell K_ref(a, b) to the entry of the offset b - a of
// each of its corners b (Sec. 2.1).  Equals fine_stencil_entry for every s.
template <int D>
__device__ void fine_stencil_all(const LevelView<double>& lv, const int* c, double* st) {
  constexpr int NS = ipow_c(3, D), NC = 1 << D;
  if (lv.opkind == OP_UNIFORM) {
    for (int s = 0; s < NS; ++s) st[s] = lv.cst[s];
    return;
  }
  if (lv.opkind == OP_STORED) {
    const long long v = encode<D>(c, lv.np1);
    for (int s = 0; s < NS; ++s) st[s] = lv.st[(long long)s * lv.V + v];
    return;
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) st[s] = 0.0;
#pragma unroll
  for (int a = 0; a < NC; ++a) {
    int cell[D];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      cell[j] = c[j] - ((a >> j) & 1);
      if (cell[j] < 0 || cell[j] >= lv.n) ok = false;
    }
    if (!ok) continue;
    const double e = lv.eps[encode<D>(cell, lv.n)];
#pragma unroll
    for (int b = 0; b < NC; ++b) {
      int s = 0, mul = 1;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        s += (((b >> j) & 1) - ((a >> j) & 1) + 1) * mul;
        mul *= 3;
      }
      st[s] += e * kref<D, double>(__popc(a ^ b));
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) st[s] *= lv.hfac;
}

template <int D>
__global__ void k_fine_invdiag(LevelView<double> lv, double* __restrict__ invd) {
  constexpr int centre = (ipow_c(3, D) - 1) / 2;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < lv.V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D];
    decode<D>(v, lv.np1, c);
    invd[v] = is_interior<D>(c, lv.n) ? 1.0 / fine_stencil_entry<D>(lv, c, centre) : 0.0;
  }
}

// Solves M X = R for NR right-hand sides (m <= 8 unknowns; R is m x NR,
// row-major with stride NR) by Gaussian elimination with partial pivoting.
template <int NR>
__device__ void small_solve_multi(double* M, double* R, int m) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = fabs(M[k * 8 + k]);
    for (int i = k + 1; i < m; ++i)
      if (fabs(M[i * 8 + k]) > best) {
        best = fabs(M[i * 8 + k]);
        p = i;
      }
    if (p != k) {
      for (int j = 0; j < m; ++j) {
        const double t = M[k * 8 + j];
        M[k * 8 + j] = M[p * 8 + j];
        M[p * 8 + j] = t;
      }
      for (int r = 0; r < NR; ++r) {
        const double t = R[k * NR + r];
        R[k * NR + r] = R[p * NR + r];
        R[p * NR + r] = t;
      }
    }
    const double inv = 1.0 / M[k * 8 + k];
    for (int i = k + 1; i < m; ++i) {
      const double f = M[i * 8 + k] * inv;
      for (int j = k; j < m; ++j) M[i * 8 + j] -= f * M[k * 8 + j];
      for (int r = 0; r < NR; ++r) R[i * NR + r] -= f * R[k * NR + r];
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    const double inv = 1.0 / M[k * 8 + k];
    for (int r = 0; r < NR; ++r) {
      double t = R[k * NR + r];
      for (int j = k + 1; j < m; ++j) t -= M[k * 8 + j] * R[j * NR + r];
      R[k * NR + r] = t * inv;
    }
  }
}

// BoxMG prolongation for 3:1 coarsening (Sec. 2.4): one thread per coarse
// cell, all 2^D corners e at once.  For every corner e: value 1 at the c-point
// of e, 0 at the other corners; gamma-points on the cell's edges (and, in
// 3-D, faces) solve the stencil lumped along the sub-face normals with the rim
// as data; f-points solve the full stencil.  The matrix of a sub-face does not
// depend on e: it is assembled and factored once and solved for the 2^D
// right-hand sides.  Sub-faces on the domain boundary, and corners on the
// coarse boundary, keep zeros.  Writes the weights of the fine vertices the
// cell owns (local offset < 3, or = 3 on the last cell of a row).
template <int D>
__global__ void __launch_bounds__(64) k_boxmg(LevelView<double> fine, double* __restrict__ P, int n_c) {
  constexpr int NC = 1 << D;
  constexpr int NP = ipow_c(4, D);
  constexpr int NS = ipow_c(3, D);
  long long total = 1;
  for (int j = 0; j < D; ++j) total *= n_c;
  const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (E >= total) return;
  int ec[D];
  decode<D>(E, n_c, ec);
  double v[NP * NC];  // v[p * NC + e]: P e at closure point p
  for (int i = 0; i < NP * NC; ++i) v[i] = 0.0;
  for (int e = 0; e < NC; ++e) {
    // corners on the coarse boundary carry no unknown: their weights stay zero
    bool cb = false;
    int cp[D];
    for (int j = 0; j < D; ++j) {
      const int J = ec[j] + ((e >> j) & 1);
      if (J == 0 || J == n_c) cb = true;
      cp[j] = 3 * ((e >> j) & 1);
    }
    if (!cb) v[encode<D>(cp, 4) * NC + e] = 1.0;
  }
  for (int nfree = 1; nfree <= D; ++nfree) {
    for (int F = 0; F < NC; ++F) {
      if (__popc(F) != nfree) continue;
      const int nfix = D - nfree;
      for (int fb = 0; fb < (1 << nfix); ++fb) {
        // fixed coordinates of the bounding dims
        int lfix[D];
        bool on_bnd = false;
        int k = 0;
        for (int j = 0; j < D; ++j) {
          lfix[j] = 0;
          if (!((F >> j) & 1)) {
            lfix[j] = ((fb >> k) & 1) ? 3 : 0;
            ++k;
            if ((lfix[j] == 0 && ec[j] == 0) || (lfix[j] == 3 && ec[j] == n_c - 1)) on_bnd = true;
          }
        }
        if (on_bnd) continue;  // zeros
        const int m = 1 << nfree;
        double M[64], R[8 * NC];
        for (int i = 0; i < 64; ++i) M[i] = 0.0;
        for (int i = 0; i < 8 * NC; ++i) R[i] = 0.0;
        for (int p = 0; p < m; ++p) {
          // unknown point p: free coords 1 or 2 by the bits of p
          int lp[D];
          int q = 0;
          for (int j = 0; j < D; ++j) {
            if ((F >> j) & 1) {
              lp[j] = 1 + ((p >> q) & 1);
              ++q;
            } else {
              lp[j] = lfix[j];
            }
          }
          int fpc[D];
          for (int j = 0; j < D; ++j) fpc[j] = 3 * ec[j] + lp[j];
          double st[NS];
          fine_stencil_all<D>(fine, fpc, st);
          // collapsed stencil: offsets along the fixed dims fold onto the sub-face
          for (int s = 0; s < NS; ++s) {
            int o[D], t = s;
            for (int j = 0; j < D; ++j) {
              o[j] = t % 3 - 1;
              t /= 3;
            }
            int nb[D];
            for (int j = 0; j < D; ++j) nb[j] = ((F >> j) & 1) ? lp[j] + o[j] : lp[j];
            const double coef = st[s];
            bool unk = true;
            int qi = 0, qq = 0;
            for (int j = 0; j < D; ++j) {
              if ((F >> j) & 1) {
                if (nb[j] < 1 || nb[j] > 2) unk = false;
                qi |= (nb[j] - 1) << qq;
                ++qq;
              }
            }
            if (unk) {
              M[p * 8 + qi] += coef;
            } else {
              const double* vn = v + encode<D>(nb, 4) * NC;
              for (int e = 0; e < NC; ++e) R[p * NC + e] -= coef * vn[e];
            }
          }
        }
        small_solve_multi<NC>(M, R, m);
        for (int p = 0; p < m; ++p) {
          int lp[D];
          int q = 0;
          for (int j = 0; j < D; ++j) {
            if ((F >> j) & 1) {
              lp[j] = 1 + ((p >> q) & 1);
              ++q;
            } else {
              lp[j] = lfix[j];
            }
          }
          double* vp = v + encode<D>(lp, 4) * NC;
          for (int e = 0; e < NC; ++e) vp[e] = R[p * NC + e];
        }
      }
    }
  }
  // owned fine vertices
  const int np1f = 3 * n_c + 1;
  long long Vf = 1;
  for (int j = 0; j < D; ++j) Vf *= np1f;
  for (int p = 0; p < NP; ++p) {
    int lc[D], fc[D];
    decode<D>(p, 4, lc);
    bool owned = true, fbnd = false;
    for (int j = 0; j < D; ++j) {
      if (lc[j] == 3 && ec[j] != n_c - 1) owned = false;
      fc[j] = 3 * ec[j] + lc[j];
      if (fc[j] == 0 || fc[j] == 3 * n_c) fbnd = true;
    }
    if (!owned) continue;
    const long long fv = encode<D>(fc, np1f);
    for (int e = 0; e < NC; ++e) P[(long long)e * Vf + fv] = fbnd ? 0.0 : v[p * NC + e];
  }
}

// Closure weight W[l][e] of coarse cell E (fine vertex 3E + l towards corner e).
template <int D>
__device__ double closure_weight(const LevelView<double>& fine, int n_c, const int* ec,
                                 const int* l, int e) {
  int fc[D];
  bool fbnd = false, cbnd = false;
  for (int j = 0; j < D; ++j) {
    fc[j] = 3 * ec[j] + l[j];
    if (fc[j] == 0 || fc[j] == 3 * n_c) fbnd = true;
    const int J = ec[j] + ((e >> j) & 1);
    if (J == 0 || J == n_c) cbnd = true;
  }
  if (fbnd || cbnd) return 0.0;
  if (!fine.boxmg) {
    double w = 1.0;
    for (int j = 0; j < D; ++j) {
      const double t = l[j] / 3.0;
      w *= ((e >> j) & 1) ? t : 1.0 - t;
    }
    return w;
  }
  int eo = 0;
  for (int j = 0; j < D; ++j) {
    int own = fc[j] / 3;
    own = own < n_c - 1 ? own : n_c - 1;
    const int bit = ec[j] + ((e >> j) & 1) - own;
    if (bit < 0 || bit > 1) return 0.0;
    eo |= bit << j;
  }
  return fine.P[(long long)eo * fine.V + encode<D>(fc, fine.np1)];
}

// Structural zeros of the closure weights: the weight of closure point l
// (coordinates 0..3 in the coarse cell) towards corner f vanishes along any
// axis where the point lies on the cell face opposite the corner (l_j = 0
// and f_j = 1, or l_j = 3 and f_j = 0), for d-linear and BoxMG weights alike.
template <int D>
__device__ __forceinline__ bool closure_zero(const int* l, int f) {
  bool z = false;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int bit = (f >> j) & 1;
    z = z || (l[j] == 0 && bit) || (l[j] == 3 && !bit);
  }
  return z;
}

// Galerkin element matrices of the coarse level: K_E = sum over the 3^D
// children c of P_c^T K_c P_c (one thread per coarse cell).  The fine element
// matrices are eps_c h^(D-2) K_ref (fine level) or stored (Kc_fine).  FP64
// work is the cost here, so the products skip the terms that vanish by
// structure: the structural zeros of the closure weights, the zero entries
// of K_ref (in 3-D, corners one edge apart), and the lower triangle of the
// symmetric K_E (filled by symmetry at the end).
template <int D>
__global__ void __launch_bounds__(128) k_galerkin(LevelView<double> fine, const double* __restrict__ Kc_fine,
                                                  double* __restrict__ Kc, int n_c) {
  constexpr int NC = 1 << D;
  constexpr int NP = ipow_c(4, D);
  long long total = 1;
  for (int j = 0; j < D; ++j) total *= n_c;
  const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (E >= total) return;
  int ec[D];
  decode<D>(E, n_c, ec);
  double W[NP * NC];
  for (int p = 0; p < NP; ++p) {
    int l[D];
    decode<D>(p, 4, l);
    for (int e = 0; e < NC; ++e) W[p * NC + e] = closure_weight<D>(fine, n_c, ec, l, e);
  }
  double K[NC * NC];
  for (int i = 0; i < NC * NC; ++i) K[i] = 0.0;
  const int n_f = 3 * n_c;
  long long ncf = 1;
  for (int j = 0; j < D; ++j) ncf *= n_f;
  for (int k = 0; k < ipow_c(3, D); ++k) {
    int kc[D], child[D];
    int t = k;
    for (int j = 0; j < D; ++j) {
      kc[j] = t % 3;
      t /= 3;
      child[j] = 3 * ec[j] + kc[j];
    }
    const long long cidx = encode<D>(child, n_f);
    double Kf[NC * NC];
    const double eh = Kc_fine ? 0.0 : (fine.opkind == OP_EPS ? fine.eps[cidx] : fine.eps0) * fine.hfac;
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
      for (int b = 0; b < NC; ++b)
        Kf[a * NC + b] = Kc_fine ? Kc_fine[(long long)(a * NC + b) * ncf + cidx]
                                 : eh * kref<D, double>(__popc(a ^ b));
    // T = Kf * Pc  (Pc[b][f] = W[kc + b][f])
    double Tm[NC * NC];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
      for (int f = 0; f < NC; ++f) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < NC; ++b) {
          if (!Kc_fine && D == 3 && __popc(a ^ b) == 1) continue;  // K_ref entry 0
          int lb[D];
          for (int j = 0; j < D; ++j) lb[j] = kc[j] + ((b >> j) & 1);
          if (closure_zero<D>(lb, f)) continue;
          s += Kf[a * NC + b] * W[encode<D>(lb, 4) * NC + f];
        }
        Tm[a * NC + f] = s;
      }
    // K += Pc^T T on the upper triangle (e <= f)
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      int la[D];
      for (int j = 0; j < D; ++j) la[j] = kc[j] + ((a >> j) & 1);
      const int pa = encode<D>(la, 4);
#pragma unroll
      for (int e = 0; e < NC; ++e) {
        if (closure_zero<D>(la, e)) continue;
        const double wae = W[pa * NC + e];
#pragma unroll
        for (int f = e; f < NC; ++f) K[e * NC + f] += wae * Tm[a * NC + f];
      }
    }
  }
#pragma unroll
  for (int e = 0; e < NC; ++e)
#pragma unroll
    for (int f = 0; f < e; ++f) K[e * NC + f] = K[f * NC + e];
  for (int i = 0; i < NC * NC; ++i) Kc[(long long)i * total + E] = K[i];
}

// Rediscretised element matrices of the coarse level (one thread per coarse
// cell): eps_E = mean over the 3^D children c of eps_c, K_E = eps_E
// h_c^(D-2) K_ref.  The children's eps come from the fine eps, or from their
// stored element matrices (K_c = eps_c h^(D-2) K_ref: entry (0, 0)).
template <int D>
__global__ void __launch_bounds__(128) k_rediscretise(LevelView<double> fine,
                                                      const double* __restrict__ Kc_fine,
                                                      double* __restrict__ Kc, int n_c) {
  constexpr int NC = 1 << D;
  long long total = 1;
  for (int j = 0; j < D; ++j) total *= n_c;
  const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (E >= total) return;
  int ec[D];
  decode<D>(E, n_c, ec);
  const int n_f = 3 * n_c;
  long long ncf = 1;
  for (int j = 0; j < D; ++j) ncf *= n_f;
  double sum = 0.0;
  for (int k = 0; k < ipow_c(3, D); ++k) {
    int child[D], t = k;
    for (int j = 0; j < D; ++j) {
      child[j] = 3 * ec[j] + t % 3;
      t /= 3;
    }
    const long long c = encode<D>(child, n_f);
    double e;
    if (Kc_fine)
      e = Kc_fine[c] / (fine.hfac * kref<D, double>(0));
    else
      e = fine.opkind == OP_EPS ? fine.eps[c] : fine.eps0;
    sum += e;
  }
  const double eps = sum / (double)ipow_c(3, D);
  const double hfac = D == 2 ? 1.0 : 1.0 / n_c;
  for (int a = 0; a < NC; ++a)
    for (int b = 0; b < NC; ++b)
      Kc[(long long)(a * NC + b) * total + E] = eps * hfac * kref<D, double>(__popc(a ^ b));
}

// Assembled 3^D stencil and inverse diagonal of every vertex from the
// per-cell element matrices (entry-major layouts).
template <int D>
__global__ void k_assemble(const double* __restrict__ Kc, double* __restrict__ st,
                           double* __restrict__ invd, int n) {
  constexpr int NC = 1 << D;
  constexpr int NS = ipow_c(3, D);
  const int np1 = n + 1;
  long long V = 1, ncells = 1;
  for (int j = 0; j < D; ++j) {
    V *= np1;
    ncells *= n;
  }
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D];
    decode<D>(v, np1, c);
    for (int s = 0; s < NS; ++s) {
      int o[D], t = s;
      for (int j = 0; j < D; ++j) {
        o[j] = t % 3 - 1;
        t /= 3;
      }
      double acc = 0.0;
      for (int a = 0; a < NC; ++a) {
        int cell[D], b = 0;
        bool ok = true;
        for (int j = 0; j < D; ++j) {
          const int aj = (a >> j) & 1;
          cell[j] = c[j] - aj;
          if (cell[j] < 0 || cell[j] >= n) ok = false;
          const int bj = aj + o[j];
          if (bj < 0 || bj > 1) ok = false;
          b |= (bj & 1) << j;
        }
        if (!ok) continue;
        acc += Kc[(long long)(a * NC + b) * ncells + encode<D>(cell, n)];
      }
      st[(long long)s * V + v] = acc;
      if (s == (NS - 1) / 2) invd[v] = is_interior<D>(c, n) ? 1.0 / acc : 0.0;
    }
  }
}

__global__ void k_to_float(const double* __restrict__ src, float* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

__global__ void k_fill(double* __restrict__ dst, double value, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = value;
}

}  // namespace

template <int D>
void launch_rhs(const double* f, double* b, int n, cudaStream_t s) {
  long long V = 1;
  for (int j = 0; j < D; ++j) V *= n + 1;
  k_rhs<D><<<blocks_for(V, 256), 256, 0, s>>>(f, b, n);
}

template <int D>
void launch_fine_invdiag(const LevelView<double>& fine, double* invd, cudaStream_t s) {
  k_fine_invdiag<D><<<blocks_for(fine.V, 256), 256, 0, s>>>(fine, invd);
}

template <int D>
void launch_boxmg(const LevelView<double>& fine, double* P, int n_c, cudaStream_t s) {
  long long total = 1;
  for (int j = 0; j < D; ++j) total *= n_c;
  k_boxmg<D><<<blocks_for(total, 64), 64, 0, s>>>(fine, P, n_c);
}

template <int D>
void launch_galerkin(const LevelView<double>& fine, const double* Kc_fine, double* Kc_coarse,
                     int n_c, cudaStream_t s) {
  long long total = 1;
  for (int j = 0; j < D; ++j) total *= n_c;
  k_galerkin<D><<<blocks_for(total, 128), 128, 0, s>>>(fine, Kc_fine, Kc_coarse, n_c);
}

template <int D>
void launch_rediscretise(const LevelView<double>& fine, const double* Kc_fine, double* Kc,
                         int n_c, cudaStream_t s) {
  long long total = 1;
  for (int j = 0; j < D; ++j) total *= n_c;
  k_rediscretise<D><<<blocks_for(total, 128), 128, 0, s>>>(fine, Kc_fine, Kc, n_c);
}

template <int D>
void launch_assemble(const double* Kc, double* st, double* invd, int n, cudaStream_t s) {
  long long V = 1;
  for (int j = 0; j < D; ++j) V *= n + 1;
  k_assemble<D><<<blocks_for(V, 128), 128, 0, s>>>(Kc, st, invd, n);
}

void launch_to_float(const double* src, float* dst, long long count, cudaStream_t s) {
  k_to_float<<<blocks_for(count, 256) > 4096 ? 4096 : blocks_for(count, 256), 256, 0, s>>>(src, dst, count);
}

void launch_fill(double* dst, double value, long long count, cudaStream_t s) {
  k_fill<<<blocks_for(count, 256) > 4096 ? 4096 : blocks_for(count, 256), 256, 0, s>>>(dst, value, count);
}

#define ADAFAC_SETUP_INST(D)                                                                 \
  template void launch_rhs<D>(const double*, double*, int, cudaStream_t);                    \
  template void launch_fine_invdiag<D>(const LevelView<double>&, double*, cudaStream_t);     \
  template void launch_boxmg<D>(const LevelView<double>&, double*, int, cudaStream_t);       \
  template void launch_galerkin<D>(const LevelView<double>&, const double*, double*, int,    \
                                   cudaStream_t);                                            \
  template void launch_assemble<D>(const double*, double*, double*, int, cudaStream_t);    \
  template void launch_rediscretise<D>(const LevelView<double>&, const double*, double*, int, \
                                       cudaStream_t);

ADAFAC_SETUP_INST(2)
ADAFAC_SETUP_INST(3)

}  // namespace adafac
