// Batched refinement steps of the mixed-precision solve (ADAFAC_PATH_BATCHED).
//
// One launch advances every instance of a batch by one refinement step of
// iterative refinement around Algorithm 1:
//   r = b - A u in FP64, its Eq. 10 norm and the convergence test;
//   k FP32 cycles on the correction equation A e = r (Alg. 1, Eq. 9):
//     r_L = r - A e;
//     r_l = P^T r_{l+1}, b~_l = omega S~^T r_{l+1} (truncated R~, Eq. 8),
//       g_l = M_l^-1 (omega r_l - omega~ b~_l)          (l = L-1 .. lmin);
//     t_l = g_l + P q_{l-1}                              (l = lmin+1 .. L-1);
//     e  += omega M_L^-1 r_L + P q_{L-1};
//   u += e, e = 0.
// Every instance runs on its own cluster of C CTAs (the cluster index selects
// the instance), and the steps above follow each other separated by cluster
// barriers (a CTA barrier when C = 1): the launch boundaries of the level
// kernels become barriers inside one kernel, and one launch carries every
// request of a batch instead of a dozen launches per request and cycle.
//
// A step's work is cut into units of kBatchThreads consecutive vertices
// (linear index, x fastest): unit q belongs to CTA q mod C of the cluster,
// vertex q kBatchThreads + threadIdx.x to that thread.  The arithmetic of a
// vertex, and the norm partial of a unit (a fixed tree over the unit's
// threads), depend neither on C nor on the other instances, so a solve
// repeats bit for bit whatever it is batched with.
//
// Vectors written in the launch by other CTAs are read after a cluster
// barrier, whose arrive has release and whose wait has acquire semantics at
// cluster scope.  There are no spin waits: the barriers are the hardware's.
#include <atomic>

#include "common.cuh"

namespace adafac {

namespace {

constexpr int kBT = kBatchThreads;
constexpr int kWarps = kBT / 32;

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_count() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}

// the barrier between two steps of the cycle
__device__ __forceinline__ void step_barrier(unsigned C) {
  if (C == 1) {
    __syncthreads();
    return;
  }
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Sum of one value per thread of the CTA in a fixed order (warp trees, then
// the warps in order); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double acc, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kWarps; ++w) s += red[w];
  __syncthreads();  // red is reused by the next call
  return s;
}

template <int D>
__device__ __forceinline__ void coords(long long v, int np1, int* c) {
  const unsigned w = (unsigned)v, m = (unsigned)np1;
  const unsigned q = w / m;
  c[0] = (int)(w - q * m);
  if (D == 2) {
    c[1] = (int)q;
    c[2] = 0;
  } else {
    const unsigned q2 = q / m;
    c[1] = (int)(q - q2 * m);
    c[2] = (int)q2;
  }
}

template <int D>
__device__ __forceinline__ bool interior(const int* c, int n) {
  bool in = c[0] >= 1 && c[0] <= n - 1 && c[1] >= 1 && c[1] <= n - 1;
  if (D == 3) in = in && c[2] >= 1 && c[2] <= n - 1;
  return in;
}

// (b - A x)_v of the d-linear FEM operator with per-cell eps (or a scalar
// eps0 when eps is null) at an interior vertex c of a grid with n cells.
// Element matrices by the Hamming distance of two corners (Sec. 2.1):
//   2-D: 2/3, -1/6, -1/3;  3-D: 1/3, 0, -1/12, -1/12 (times h^(D-2)).
template <typename T>
__device__ __forceinline__ T residual2(const T* __restrict__ x, const T* __restrict__ b,
                                       const T* __restrict__ eps, T eps0, T hfac, int n,
                                       const int* c, long long v) {
  const int np1 = n + 1;
  T E[9];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) E[(dy + 1) * 3 + dx + 1] = x[v + dy * np1 + dx];
  const long long c0 = (long long)(c[1] - 1) * n + c[0] - 1;
  const T K0 = T(2.0 / 3.0), K1 = T(-1.0 / 6.0), K2 = T(-1.0 / 3.0);
  T Ax = T(0);
#pragma unroll
  for (int sy = 0; sy < 2; ++sy)
#pragma unroll
    for (int sx = 0; sx < 2; ++sx) {
      const T e = eps ? eps[c0 + sy * n + sx] : eps0;
      // the cell on side (sx, sy): the corners one edge away, then the
      // opposite corner
      const T near = E[3 + 2 * sx] + E[6 * sy + 1];
      Ax += e * (K0 * E[4] + K1 * near + K2 * E[6 * sy + 2 * sx]);
    }
  return b[v] - hfac * Ax;
}

template <typename T>
__device__ __forceinline__ T residual3(const T* __restrict__ x, const T* __restrict__ b,
                                       const T* __restrict__ eps, T eps0, T hfac, int n,
                                       const int* c, long long v) {
  const int np1 = n + 1;
  const long long P = (long long)np1 * np1;
  // planes z - 1, z, z + 1 of the 3 x 3 neighbourhood ([dy + 1][dx + 1])
  T E[3][9];
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx)
        E[dz + 1][(dy + 1) * 3 + dx + 1] = x[v + dz * P + dy * np1 + dx];
  // In the cell on side (sx, sy, sz) the corners with two or three offsets
  // couple with -1/12, the ones with a single offset not at all.
  T esum = T(0), far = T(0);
#pragma unroll
  for (int sz = 0; sz < 2; ++sz) {
    const T* S = E[2 * sz];
    const long long cz = (long long)(c[2] - 1 + sz) * n;
#pragma unroll
    for (int sy = 0; sy < 2; ++sy)
#pragma unroll
      for (int sx = 0; sx < 2; ++sx) {
        const T e = eps ? eps[(cz + c[1] - 1 + sy) * n + c[0] - 1 + sx] : eps0;
        const T f = (E[1][6 * sy + 2 * sx] + S[3 + 2 * sx]) + (S[6 * sy + 1] + S[6 * sy + 2 * sx]);
        esum += e;
        far += e * f;
      }
  }
  const T Ax = hfac * (T(1.0 / 3.0) * E[1][4] * esum + T(-1.0 / 12.0) * far);
  return b[v] - Ax;
}

// the norm evaluation of a refinement step (records the history, sets done /
// diverged like the level path's norm kernel)
__device__ void norm_update(Control* ctl, double sq, double* hist, int hist_cap) {
  if (ctl->set_r0) {
    ctl->r0sq = sq;
    ctl->set_r0 = 0;
  }
  double rel;
  if (!isfinite(sq) || !isfinite(ctl->r0sq)) rel = NAN;
  else rel = ctl->r0sq > 0.0 ? sqrt(sq / ctl->r0sq) : (sq > 0.0 ? INFINITY : 0.0);
  ctl->lastsq = sq;
  ctl->rel = rel;
  if (ctl->nhist < hist_cap) hist[ctl->nhist] = rel;
  ctl->nhist += 1;
  if (!(rel <= 1e6)) ctl->diverged = 1;
  else if (ctl->tol >= 0.0 && rel <= ctl->tol) ctl->done = 1;
}

// ---- the steps of a cycle ----------------------------------------------------
//
// A step loops over its units NV at a time: a thread computes its vertices
// of units q, q + C, .., q + (NV - 1) C before it stores any of them, so the
// loads of NV vertices are in flight together.  Which thread computes a
// vertex, and how, does not depend on NV.

template <int D>
constexpr int nv_fine() { return D == 2 ? 2 : 1; }

// vertex of unit q0 + s C handled by this thread
__device__ __forceinline__ long long unit_vertex(long long q0, int s, unsigned C) {
  return (q0 + (long long)s * C) * kBT + threadIdx.x;
}

// FP64 residual of u onto rhs (FP32), one norm partial h^D sum r^2 per unit:
// warp trees, then the unit's warps in order
template <int D>
__device__ void step_refine_residual(const BatchItem& it, unsigned rank, unsigned C,
                                     double* red) {
  constexpr int NV = nv_fine<D>();
  const BatchLevel& F = it.lev[it.L];
  const int n = F.n;
  const long long units = it.nunits;
  for (long long q0 = rank; q0 < units; q0 += (long long)C * NV) {
    double r[NV];
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const long long v = unit_vertex(q0, s, C);
      r[s] = 0.0;
      if (v < F.V) {
        int c[3];
        coords<D>(v, n + 1, c);
        if (interior<D>(c, n))
          r[s] = D == 2 ? residual2<double>(it.u, it.b, it.eps, it.eps0, it.hfac, n, c, v)
                        : residual3<double>(it.u, it.b, it.eps, it.eps0, it.hfac, n, c, v);
      }
    }
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const long long v = unit_vertex(q0, s, C);
      if (v < F.V) it.rhs[v] = (float)r[s];
      double a = r[s] * r[s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if ((threadIdx.x & 31) == 0) red[s * kWarps + (threadIdx.x >> 5)] = a;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
      const long long q = q0 + (long long)threadIdx.x * C;
      if (q < units) {
        double sum = 0.0;
        for (int w = 0; w < kWarps; ++w) sum += red[threadIdx.x * kWarps + w];
        it.partials[q] = sum * it.hD;
      }
    }
    __syncthreads();
  }
}

// FP32 residual of the correction equation: r_L = rhs - A e
template <int D>
__device__ void step_residual32(const BatchItem& it, unsigned rank, unsigned C) {
  constexpr int NV = nv_fine<D>();
  const BatchLevel& F = it.lev[it.L];
  const int n = F.n;
  for (long long q0 = rank; q0 < it.nunits; q0 += (long long)C * NV) {
    float r[NV];
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const long long v = unit_vertex(q0, s, C);
      r[s] = 0.f;
      if (v < F.V) {
        int c[3];
        coords<D>(v, n + 1, c);
        if (interior<D>(c, n))
          r[s] = D == 2 ? residual2<float>(it.e, it.rhs, it.eps32, it.eps0f, it.hfac32, n, c, v)
                        : residual3<float>(it.e, it.rhs, it.eps32, it.eps0f, it.hfac32, n, c, v);
      }
    }
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const long long v = unit_vertex(q0, s, C);
      if (v < F.V) F.r[v] = r[s];
    }
  }
}

// Level l from level l + 1: r_l = P^T r_{l+1} over the 5^D window 3J + o,
// b~_l and g_l.  Weight of fine vertex 3J + o towards J: d-linear
// prod_j (1 - |o_j| / 3); BoxMG the stored weight towards corner e of the
// fine vertex's own coarse cell, e_j = 1 where o_j < 0.
struct Restricted {
  float r, bt, g;
};

template <int D>
__device__ __forceinline__ Restricted restrict_at(const BatchItem& it, const BatchLevel& F,
                                                  const BatchLevel& Lc, const float* sst,
                                                  long long vc) {
  const int nc = Lc.n, np1 = F.n + 1;
  int J[3];
  coords<D>(vc, nc + 1, J);
  Restricted out = {0.f, 0.f, 0.f};
  if (!interior<D>(J, nc)) return out;
  const long long f0 = ((long long)(3 * J[2]) * np1 + 3 * J[1]) * np1 + 3 * J[0];
  float rs[5], bs[5];  // one partial per window row, summed in a fixed order
#pragma unroll
  for (int i = 0; i < 5; ++i) rs[i] = bs[i] = 0.f;
  constexpr int OZ = D == 3 ? 2 : 0;
#pragma unroll 1
  for (int oz = -OZ; oz <= OZ; ++oz)
#pragma unroll
    for (int oy = -2; oy <= 2; ++oy) {
      const long long row = f0 + ((long long)oz * np1 + oy) * np1;
#pragma unroll
      for (int ox = -2; ox <= 2; ++ox) {
        const long long f = row + ox;
        const float rv = F.r[f];
        float w;
        if (F.P) {
          const int e = (ox < 0 ? 1 : 0) | (oy < 0 ? 2 : 0) | (oz < 0 ? 4 : 0);
          w = F.P[e * F.V + f];
        } else {
          w = (1.f - (ox < 0 ? -ox : ox) * (1.f / 3.f)) * (1.f - (oy < 0 ? -oy : oy) * (1.f / 3.f));
          if (D == 3) w *= 1.f - (oz < 0 ? -oz : oz) * (1.f / 3.f);
        }
        rs[oy + 2] = fmaf(w, rv, rs[oy + 2]);
        bs[oy + 2] = fmaf(sst[((oz + OZ) * 5 + oy + 2) * 5 + ox + 2], rv, bs[oy + 2]);
      }
    }
  out.r = (rs[0] + rs[1]) + (rs[2] + (rs[3] + rs[4]));
  const float id = Lc.invd ? Lc.invd[vc] : Lc.invd0;
  if (it.variant == V_JAC) {
    out.bt = it.omega * ((bs[0] + bs[1]) + (bs[2] + (bs[3] + bs[4])));
    out.g = id * (it.omega * out.r - it.omega_t * out.bt);
  } else {
    out.g = Lc.gscale * it.omega * id * out.r;
  }
  return out;
}

template <int D>
__device__ void step_restrict(const BatchItem& it, int l, const float* __restrict__ sst,
                              unsigned rank, unsigned C) {
  constexpr int NV = D == 2 ? 2 : 1;
  const BatchLevel& F = it.lev[l + 1];
  const BatchLevel& Lc = it.lev[l];
  const long long units = (Lc.V + kBT - 1) / kBT;
  for (long long q0 = rank; q0 < units; q0 += (long long)C * NV) {
    Restricted x[NV];
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const long long vc = unit_vertex(q0, s, C);
      if (vc < Lc.V) x[s] = restrict_at<D>(it, F, Lc, sst, vc);
    }
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const long long vc = unit_vertex(q0, s, C);
      if (vc >= Lc.V) continue;
      Lc.r[vc] = x[s].r;
      Lc.bt[vc] = x[s].bt;
      Lc.g[vc] = x[s].g;
    }
  }
}

// Prolongation onto level l (UPDATE: the finest level) from level l - 1:
//   UPDATE  e += omega M^-1 r_L + P q        else  t_l = g_l + P q
// q = t_{l-1} (g_lmin on the coarsest level), minus for adAFAC-PI the
// level's own Jacobi correction at the vertex that coincides with the coarse
// corner.  Corners e with e_j = 1 where the vertex lies on the coarse plane
// (local offset 0) carry no weight and are skipped.
template <int D, bool UPDATE>
__device__ __forceinline__ float prolong_at(const BatchItem& it, const BatchLevel& F,
                                            const BatchLevel& Lc, const float* tc, bool coarse,
                                            const int* c, long long v) {
  constexpr int NC = 1 << D;
  const int np1 = F.n + 1;
  float du = UPDATE ? it.omega * (F.invd ? F.invd[v] : F.invd0) * F.r[v] : F.g[v];
  if (!coarse) return du;
  const int nc = Lc.n, ncp1 = nc + 1;
  int O[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
#pragma unroll
  for (int j = 0; j < D; ++j) {
    O[j] = min(c[j] / 3, nc - 1);
    lo[j] = c[j] - 3 * O[j];
  }
  const long long cbase = ((long long)O[2] * ncp1 + O[1]) * ncp1 + O[0];
  float acc = 0.f;
#pragma unroll
  for (int e = 0; e < NC; ++e) {
    bool zero = false;
    float w = 1.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int bit = (e >> j) & 1;
      zero = zero || (bit && lo[j] == 0);
      const float t = (float)lo[j] * (1.f / 3.f);
      w *= bit ? t : 1.f - t;
    }
    if (zero) continue;
    if (F.P) w = F.P[e * F.V + v];
    const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
    float qv = tc[cbase + ((long long)ez * ncp1 + ey) * ncp1 + ex];
    if (it.variant == V_PI) {
      const long long fc =
          ((long long)(D == 3 ? 3 * (O[2] + ez) : 0) * np1 + 3 * (O[1] + ey)) * np1 + 3 * (O[0] + ex);
      qv -= UPDATE ? it.omega * (F.invd ? F.invd[fc] : F.invd0) * F.r[fc] : F.g[fc];
    }
    acc += w * qv;
  }
  return du + acc;
}

template <int D, bool UPDATE>
__device__ void step_prolong(const BatchItem& it, int l, unsigned rank, unsigned C) {
  constexpr int NV = nv_fine<D>();
  const BatchLevel& F = it.lev[l];
  const int n = F.n;
  const bool coarse = l > it.lmin;
  const BatchLevel& Lc = it.lev[coarse ? l - 1 : l];
  const float* tc = coarse ? (l - 1 == it.lmin ? Lc.g : Lc.t) : nullptr;
  const long long units = (F.V + kBT - 1) / kBT;
  for (long long q0 = rank; q0 < units; q0 += (long long)C * NV) {
    float x[NV];
    bool in[NV];
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const long long v = unit_vertex(q0, s, C);
      in[s] = false;
      x[s] = 0.f;
      if (v < F.V) {
        int c[3];
        coords<D>(v, n + 1, c);
        in[s] = interior<D>(c, n);
        if (in[s]) {
          x[s] = prolong_at<D, UPDATE>(it, F, Lc, tc, coarse, c, v);
          if (UPDATE) x[s] = it.e[v] + x[s];
        }
      }
    }
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const long long v = unit_vertex(q0, s, C);
      if (v >= F.V) continue;
      if (UPDATE) {
        if (in[s]) it.e[v] = x[s];
      } else {
        F.t[v] = x[s];  // zero on the boundary
      }
    }
  }
}

// u += e, e = 0 on the finest level (the global e when e is held on chip)
__device__ void step_refine_update(const BatchItem& it, float* e_global, unsigned rank,
                                   unsigned C) {
  const long long V = it.lev[it.L].V;
  for (long long q = rank; q < it.nunits; q += C) {
    const long long v = q * kBT + threadIdx.x;
    if (v >= V) continue;
    it.u[v] += (double)it.e[v];
    if (e_global == it.e) it.e[v] = 0.f;
  }
}

// One refinement step; returns 0 when the solve had already ended, 1 when
// the residual's norm ended it, 2 when the cycles ran.
template <int D>
__device__ int refinement_step(const BatchItem& it, int k, float* e_global, const float* sst,
                               double* red, unsigned rank, unsigned C) {
  Control* ctl = it.ctl;
  // nothing writes the control block before the first barrier: every CTA of
  // the cluster takes the same decision here
  if (halted(ctl)) return 0;
  step_refine_residual<D>(it, rank, C, red);
  step_barrier(C);
  if (rank == 0) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < it.nunits; i += kBT) acc += it.partials[i];
    const double sq = block_sum(acc, red);
    if (threadIdx.x == 0) norm_update(ctl, sq, it.hist, it.hist_cap);
  }
  step_barrier(C);
  if (halted(ctl)) return 1;  // converged or diverged: u stays as evaluated
  const int L = it.L, lmin = it.lmin;
  for (int j = 0; j < k; ++j) {
    step_residual32<D>(it, rank, C);
    step_barrier(C);
    for (int l = L - 1; l >= lmin; --l) {
      step_restrict<D>(it, l, sst, rank, C);
      step_barrier(C);
    }
    for (int l = lmin + 1; l <= L - 1; ++l) {
      step_prolong<D, false>(it, l, rank, C);
      step_barrier(C);
    }
    step_prolong<D, true>(it, L, rank, C);
    if (rank == 0 && threadIdx.x == 0) ctl->applied += 1;
    step_barrier(C);
  }
  step_refine_update(it, e_global, rank, C);
  return 2;
}

// Floats an instance keeps on chip when it runs on one CTA: e, rhs and r on
// the finest level, r, b~, g, t on the coarser ones (0: more than fits).
__host__ __device__ inline long long onchip_floats(const BatchItem& it) {
  long long f = 3 * it.lev[it.L].V;
  for (int l = it.lmin; l < it.L; ++l) f += 4 * it.lev[l].V;
  return f;
}

template <int D>
__global__ void __launch_bounds__(kBT, 1) k_batch_step(const BatchLaunch bl) {
  __shared__ __align__(16) unsigned char raw[sizeof(BatchItem)];
  __shared__ float sst[125];
  __shared__ double red[4 * kWarps];
  extern __shared__ float dyn[];
  const unsigned rank = cluster_rank(), C = cluster_count(), item = cluster_index();
  if (item >= (unsigned)bl.count) return;  // whole clusters only: uniform
  const BatchItem& src = *bl.item[item];
  {
    const unsigned* from = reinterpret_cast<const unsigned*>(&src);
    unsigned* to = reinterpret_cast<unsigned*>(raw);
    for (int i = threadIdx.x; i < (int)(sizeof(BatchItem) / 4); i += kBT) to[i] = from[i];
  }
  __syncthreads();
  BatchItem& it = *reinterpret_cast<BatchItem*>(raw);
  // A one-CTA instance that fits keeps its FP32 vectors in shared memory:
  // the steps read them at shared-memory latency instead of L2's.  e starts
  // at zero; the level vectors go back to the device arrays at the end.
  const long long need = onchip_floats(it);
  const bool onchip = C == 1 && need * (long long)sizeof(float) <= bl.dyn_bytes;
  if (onchip) {
    if (threadIdx.x == 0) {
      float* p = dyn;
      it.e = p;
      p += it.lev[it.L].V;
      it.rhs = p;
      p += it.lev[it.L].V;
      it.lev[it.L].r = p;
      p += it.lev[it.L].V;
      for (int l = it.lmin; l < it.L; ++l) {
        const long long V = it.lev[l].V;
        it.lev[l].r = p;
        it.lev[l].bt = p + V;
        it.lev[l].g = p + 2 * V;
        it.lev[l].t = p + 3 * V;
        p += 4 * V;
      }
    }
    for (long long i = threadIdx.x; i < need; i += kBT) dyn[i] = 0.f;
  }
  for (int i = threadIdx.x; i < 125; i += kBT) sst[i] = it.stilde[i];
  __syncthreads();
  const int stage = refinement_step<D>(it, bl.k[item], src.e, sst, red, rank, C);
  if (onchip && stage >= 1) {
    __syncthreads();
    const long long VL = it.lev[it.L].V;
    for (long long i = threadIdx.x; i < VL; i += kBT) src.rhs[i] = it.rhs[i];
    if (stage == 2 && bl.k[item] > 0) {
      for (long long i = threadIdx.x; i < VL; i += kBT) src.lev[it.L].r[i] = it.lev[it.L].r[i];
      for (int l = it.lmin; l < it.L; ++l)
        for (long long i = threadIdx.x; i < it.lev[l].V; i += kBT) {
          src.lev[l].r[i] = it.lev[l].r[i];
          src.lev[l].bt[i] = it.lev[l].bt[i];
          src.lev[l].g[i] = it.lev[l].g[i];
          src.lev[l].t[i] = it.lev[l].t[i];
        }
    }
  }
  // the control block is written by this thread alone
  if (bl.mirror && rank == 0 && threadIdx.x == 0) bl.mirror[item] = *it.ctl;
}

static_assert(sizeof(BatchItem) % 4 == 0, "item copied as 32-bit words");

std::atomic<int> g_max_cluster{0};

int max_cluster() {
  int m = g_max_cluster.load();
  if (m) return m;
  // 16 CTAs per cluster is beyond the portable size: allowed where the
  // device can place such a cluster, else 8
  m = 8;
  if (cudaFuncSetAttribute(k_batch_step<2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(k_batch_step<3>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kBT);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n2 = 0, n3 = 0;
    if (cudaOccupancyMaxActiveClusters(&n2, k_batch_step<2>, &cfg) == cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&n3, k_batch_step<3>, &cfg) == cudaSuccess && n2 > 0 &&
        n3 > 0)
      m = 16;
  }
  cudaGetLastError();
  g_max_cluster.store(m);
  return m;
}

}  // namespace

int batch_max_cluster() { return max_cluster(); }

int batch_onchip_bytes(const BatchItem& host_item) {
  const long long b = onchip_floats(host_item) * (long long)sizeof(float);
  return b <= kBatchOnchipBytes ? (int)b : 0;
}

int batch_cluster_size(long long V, int onchip_bytes) {
  if (onchip_bytes > 0) return 1;
  const int cap = max_cluster();
  // about 8 vertices per thread on the finest level, at most the cap
  int C = 1;
  while (C < cap && (long long)C * kBT * 8 < V) C *= 2;
  return C;
}

cudaError_t launch_batch_step(int D, int C, const BatchLaunch& bl, cudaStream_t s) {
  if (bl.count <= 0) return cudaSuccess;
  if (bl.count > kBatchMax || (D != 2 && D != 3) || C < 1 || C > max_cluster() || (C & (C - 1)))
    return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  if (bl.dyn_bytes < 0 || bl.dyn_bytes > kBatchOnchipBytes) return cudaErrorInvalidValue;
  static std::atomic<int> smem_set{0};
  if (!smem_set.load()) {
    if (cudaFuncSetAttribute(k_batch_step<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kBatchOnchipBytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_batch_step<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kBatchOnchipBytes) != cudaSuccess)
      return cudaGetLastError();
    smem_set.store(1);
  }
  cfg.gridDim = dim3((unsigned)(C * bl.count));
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = C == 1 ? (size_t)bl.dyn_bytes : 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return D == 2 ? cudaLaunchKernelEx(&cfg, k_batch_step<2>, bl)
                : cudaLaunchKernelEx(&cfg, k_batch_step<3>, bl);
}

}  // namespace adafac
