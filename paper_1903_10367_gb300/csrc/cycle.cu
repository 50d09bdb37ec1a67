// Level-by-level cycle kernels (the reference path of the library: every
// step of Algorithm 1 as its own launch).  Templated on the dimension and on
// the element type (double: FP64 mode and the FP64 refinement residual;
// float: the FP32 cycles of the mixed mode).
#include "common.cuh"

namespace adafac {

namespace {

inline int grid_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// ---------------------------------------------------------------------------
// r = b - A x at interior vertices (Alg. 1 first line; Eq. 4 hierarchical
// residuals); per-block partial sums of h^D r^2 (Eq. 10) in FP64.
template <int D, typename T, typename TX>
__global__ void k_residual(LevelView<T> lv, const TX* __restrict__ x, const TX* __restrict__ b,
                           TX* __restrict__ r, float* __restrict__ r32,
                           double* __restrict__ partials, double hD, const Control* ctl) {
  if (halted(ctl)) return;
  double acc = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < lv.V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D];
    decode<D>(v, lv.np1, c);
    T rv = T(0);
    if (is_interior<D>(c, lv.n)) {
      rv = (b ? T(b[v]) : T(0)) - apply_op<D, T, TX>(lv, x, c, v);
      acc += (double)rv * (double)rv;
    }
    if (r) r[v] = TX(rv);
    if (r32) r32[v] = (float)rv;
  }
  if (!partials) return;
  // block reduction in a fixed order
  __shared__ double red[256];
  red[threadIdx.x] = acc * hD;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// Restriction to the coarse level and the level's combined correction.
//   r_c = P^T r_f                          (b_l = R^{L-l} r_L, Alg. 1)
//   b~_c = omega S~^T r_f  or  omega P^T y_f with y = A (M^-1 r)   (Eq. 8)
//   g_c = M_c^-1 (omega r_c - omega~ b~_c)  (c_l - c~_l, Eq. 9)  [JAC]
//       = gscale omega M_c^-1 r_c                        [ADDITIVE/EXP/PI]
template <int D, typename T>
__global__ void __launch_bounds__(256) k_restrict(LevelView<T> lf, LevelView<T> lc,
                                                  CycleParams<T> cp, const T* __restrict__ r_f,
                                                  const T* __restrict__ y_f, T* __restrict__ r_c,
                                                  int rc_given, T* __restrict__ bt_c,
                                                  T* __restrict__ g_c, T gscale,
                                                  const Control* ctl) {
  if (halted(ctl)) return;
  constexpr int N5 = ipow_c(5, D);
  constexpr int PER = (N5 + 31) / 32;  // window points per lane
  // one warp per coarse vertex: lane l takes the window points l, l + 32, ...
  __shared__ T s_st[N5];
  for (int k = threadIdx.x; k < N5; k += blockDim.x) s_st[k] = cp.stilde[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long v = w0; v < lc.V; v += nw) {
    int J[D];
    decode<D>(v, lc.np1, J);
    if (!is_interior<D>(J, lc.n)) {
      if (lane == 0) {
        if (!rc_given) r_c[v] = T(0);
        if (bt_c) bt_c[v] = T(0);
        g_c[v] = T(0);
      }
      continue;
    }
    T rc = T(0), bt = T(0);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int k = lane + 32 * i;
      if (k >= N5) break;
      int fc[D], t = k;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        fc[j] = 3 * J[j] + (t % 5) - 2;
        t /= 5;
      }
      const long long fv = encode<D>(fc, lf.np1);
      const T rv = r_f[fv];
      const T w = p_weight<D, T>(lf, lc.n, fc, fv, J);
      if (!rc_given) rc += w * rv;
      if (cp.variant == V_JAC) {
        if (cp.rtilde_exact)
          bt += w * y_f[fv];
        else
          bt += s_st[k] * rv;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rc += __shfl_xor_sync(0xffffffffu, rc, o);
      bt += __shfl_xor_sync(0xffffffffu, bt, o);
    }
    if (lane != 0) continue;
    if (rc_given) rc = r_c[v];
    else r_c[v] = rc;
    const T id = inv_diag(lc, v);
    T g;
    if (cp.variant == V_JAC) {
      bt *= cp.omega;
      if (bt_c) bt_c[v] = bt;
      g = id * (cp.omega * rc - cp.omega_tilde * bt);
    } else {
      if (bt_c) bt_c[v] = T(0);
      g = gscale * cp.omega * id * rc;
    }
    g_c[v] = g;
  }
}

// y = A (M^-1 r) on level lv (input of the exact smoothed restriction).
template <int D, typename T>
__global__ void k_apply_scaled(LevelView<T> lv, const T* __restrict__ r, T* __restrict__ y,
                               const Control* ctl) {
  if (halted(ctl)) return;
  constexpr int NS = ipow_c(3, D);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < lv.V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D];
    decode<D>(v, lv.np1, c);
    if (!is_interior<D>(c, lv.n)) {
      y[v] = T(0);
      continue;
    }
    // (A z)_v with z = invd .* r, evaluated on the fly
    T acc = T(0);
    if (lv.opkind == OP_EPS) {
      constexpr int NC = 1 << D;
      for (int a = 0; a < NC; ++a) {
        int cell[D];
        for (int j = 0; j < D; ++j) cell[j] = c[j] - ((a >> j) & 1);
        const T e = lv.eps[encode<D>(cell, lv.n)];
        T inner = T(0);
        for (int bb = 0; bb < NC; ++bb) {
          int w[D];
          for (int j = 0; j < D; ++j) w[j] = cell[j] + ((bb >> j) & 1);
          const long long wv = encode<D>(w, lv.np1);
          inner += kref<D, T>(__popc(a ^ bb)) * r[wv] * inv_diag(lv, wv);
        }
        acc += e * inner;
      }
      acc *= lv.hfac;
    } else {
      for (int s = 0; s < NS; ++s) {
        const long long wv = v + stencil_offset<D>(s, lv.np1);
        const T coef = lv.opkind == OP_STORED ? lv.st[(long long)s * lv.V + v] : lv.cst[s];
        acc += coef * r[wv] * inv_diag(lv, wv);
      }
    }
    y[v] = acc;
  }
}

// Value prolonged from coarse vertex Jv: t_c (minus I c_f for adAFAC-PI,
// where c_f at the coinciding fine vertex is g_f there).
template <int D, typename T>
__device__ __forceinline__ T coarse_q(const CycleParams<T>& cp, const T* __restrict__ t_c,
                                      long long Jv, const int* Jc, int np1f,
                                      const T* __restrict__ cf) {
  T q = t_c[Jv];
  if (cp.variant == V_PI) {
    int fc[D];
    for (int j = 0; j < D; ++j) fc[j] = 3 * Jc[j];
    q -= cf[encode<D>(fc, np1f)];
  }
  return q;
}

// t_f = g_f + P q_c on a coarse level (the nested form of Eq. 9).
template <int D, typename T>
__global__ void k_prolong(LevelView<T> lf, LevelView<T> lc, CycleParams<T> cp,
                          const T* __restrict__ t_c, const T* __restrict__ g_f,
                          T* __restrict__ t_f, const Control* ctl) {
  if (halted(ctl)) return;
  constexpr int NC = 1 << D;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < lf.V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D];
    decode<D>(v, lf.np1, c);
    if (!is_interior<D>(c, lf.n)) {
      t_f[v] = T(0);
      continue;
    }
    int O[D], l[D];
    for (int j = 0; j < D; ++j) {
      O[j] = c[j] / 3;
      O[j] = O[j] < lc.n - 1 ? O[j] : lc.n - 1;
      l[j] = c[j] - 3 * O[j];
    }
    T acc = T(0);
    for (int e = 0; e < NC; ++e) {
      int Jc[D];
      for (int j = 0; j < D; ++j) Jc[j] = O[j] + ((e >> j) & 1);
      const T w = p_corner_weight<D, T>(lf, l, e, v);
      if (w == T(0)) continue;
      acc += w * coarse_q<D, T>(cp, t_c, encode<D>(Jc, lc.np1), Jc, lf.np1, g_f);
    }
    t_f[v] = g_f[v] + acc;
  }
}

// Fine update x += c_L + P q_{L-1} with c_L = omega M_L^-1 r_L.
template <int D, typename T, typename TX>
__global__ void k_update(LevelView<T> lf, LevelView<T> lc, CycleParams<T> cp,
                         const T* __restrict__ r_f, const T* __restrict__ t_c,
                         TX* __restrict__ x, Control* ctl) {
  if (halted(ctl)) return;
  constexpr int NC = 1 << D;
  if (blockIdx.x == 0 && threadIdx.x == 0 && ctl) atomicAdd(&ctl->applied, 1);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < lf.V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D];
    decode<D>(v, lf.np1, c);
    if (!is_interior<D>(c, lf.n)) continue;
    T du = cp.omega * inv_diag(lf, v) * r_f[v];
    if (lc.n > 0) {
      int O[D], l[D];
      for (int j = 0; j < D; ++j) {
        O[j] = c[j] / 3;
        O[j] = O[j] < lc.n - 1 ? O[j] : lc.n - 1;
        l[j] = c[j] - 3 * O[j];
      }
      T acc = T(0);
      for (int e = 0; e < NC; ++e) {
        int Jc[D];
        for (int j = 0; j < D; ++j) Jc[j] = O[j] + ((e >> j) & 1);
        const T w = p_corner_weight<D, T>(lf, l, e, v);
        if (w == T(0)) continue;
        T q = t_c[encode<D>(Jc, lc.np1)];
        if (cp.variant == V_PI) {
          int fc[D];
          for (int j = 0; j < D; ++j) fc[j] = 3 * Jc[j];
          const long long fv = encode<D>(fc, lf.np1);
          q -= cp.omega * inv_diag(lf, fv) * r_f[fv];
        }
        acc += w * q;
      }
      du += acc;
    }
    x[v] = TX(x[v] + du);
  }
}

// FAS (Eq. 4): injection u_c = I u_f.
template <int D>
__global__ void k_inject(const double* __restrict__ u_f, int n_f, double* __restrict__ u_c,
                         const Control* ctl) {
  if (halted(ctl)) return;
  const int n_c = n_f / 3, np1c = n_c + 1, np1f = n_f + 1;
  long long V = 1;
  for (int j = 0; j < D; ++j) V *= np1c;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D], fc[D];
    decode<D>(v, np1c, c);
    for (int j = 0; j < D; ++j) fc[j] = 3 * c[j];
    u_c[v] = is_interior<D>(c, n_c) ? u_f[encode<D>(fc, np1f)] : 0.0;
  }
}

// FAS: u^_f = u_f - P u_c.
template <int D>
__global__ void k_hierarchical(LevelView<double> lf, LevelView<double> lc,
                               const double* __restrict__ u_f, const double* __restrict__ u_c,
                               double* __restrict__ uhat, const Control* ctl) {
  if (halted(ctl)) return;
  constexpr int NC = 1 << D;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < lf.V;
       v += (long long)gridDim.x * blockDim.x) {
    int c[D];
    decode<D>(v, lf.np1, c);
    if (!is_interior<D>(c, lf.n)) {
      uhat[v] = 0.0;
      continue;
    }
    int O[D], l[D];
    for (int j = 0; j < D; ++j) {
      O[j] = c[j] / 3;
      O[j] = O[j] < lc.n - 1 ? O[j] : lc.n - 1;
      l[j] = c[j] - 3 * O[j];
    }
    double acc = 0.0;
    for (int e = 0; e < NC; ++e) {
      int Jc[D];
      for (int j = 0; j < D; ++j) Jc[j] = O[j] + ((e >> j) & 1);
      acc += p_corner_weight<D, double>(lf, l, e, v) * u_c[encode<D>(Jc, lc.np1)];
    }
    uhat[v] = u_f[v] - acc;
  }
}

// FAS: b_c = P^T rhat_f.
template <int D>
__global__ void k_restrict_plain(LevelView<double> lf, LevelView<double> lc,
                                 const double* __restrict__ r_f, double* __restrict__ b_c,
                                 const Control* ctl) {
  if (halted(ctl)) return;
  constexpr int N5 = ipow_c(5, D);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < lc.V;
       v += (long long)gridDim.x * blockDim.x) {
    int J[D];
    decode<D>(v, lc.np1, J);
    if (!is_interior<D>(J, lc.n)) {
      b_c[v] = 0.0;
      continue;
    }
    double acc = 0.0;
    for (int k = 0; k < N5; ++k) {
      int fc[D], t = k;
      for (int j = 0; j < D; ++j) {
        fc[j] = 3 * J[j] + (t % 5) - 2;
        t /= 5;
      }
      const long long fv = encode<D>(fc, lf.np1);
      acc += p_weight<D, double>(lf, lc.n, fc, fv, J) * r_f[fv];
    }
    b_c[v] = acc;
  }
}

// Norm of one residual evaluation: partial sums added in a fixed order.
__global__ void k_norm_finalize(const double* __restrict__ partials, int nblocks, Control* ctl,
                                double* __restrict__ hist, int hist_cap, int query) {
  // a cycle evaluation after the end of the solve, or after a bounded wait
  // gave up (its residual kernel returned at entry), records nothing
  if (!query && (ctl->done || ctl->diverged || ctl->fault)) return;
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double sq = red[0];
  if (ctl->set_r0) {
    ctl->r0sq = sq;
    ctl->set_r0 = 0;
  }
  double rel;
  if (!isfinite(sq) || !isfinite(ctl->r0sq)) rel = NAN;  // reported as divergence
  else rel = ctl->r0sq > 0.0 ? sqrt(sq / ctl->r0sq) : (sq > 0.0 ? INFINITY : 0.0);
  if (query) {
    ctl->qsq = sq;
    ctl->qrel = rel;
    return;
  }
  ctl->lastsq = sq;
  ctl->rel = rel;
  if (ctl->nhist < hist_cap) hist[ctl->nhist] = rel;
  ctl->nhist += 1;
  if (!(rel <= 1e6)) ctl->diverged = 1;  // also catches NaN
  else if (ctl->tol >= 0.0 && rel <= ctl->tol) ctl->done = 1;
}

__global__ void k_reset_control(Control* ctl) {
  ctl->r0sq = 0.0;
  ctl->lastsq = 0.0;
  ctl->rel = 0.0;
  ctl->tol = -1.0;
  ctl->qsq = 0.0;
  ctl->qrel = 0.0;
  ctl->done = 0;
  ctl->diverged = 0;
  ctl->nhist = 0;
  ctl->applied = 0;
  ctl->set_r0 = 1;
  ctl->fault = 0;
  ctl->uexp = ctl->bdexp;  // u = the Dirichlet values (callers that set u raise it)
}

__global__ void k_refine_update(double* __restrict__ u, float* __restrict__ e, long long V,
                                const Control* ctl) {
  if (halted(ctl)) return;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    u[v] += (double)e[v];
    e[v] = 0.0f;
  }
}

}  // namespace

constexpr int kT = 256;
constexpr int kCap = 152 * 16;

template <int D, typename T, typename TX>
void launch_residual(const LevelView<T>& lv, const TX* x, const TX* b, TX* r, float* r32,
                     double* partials, int nblocks, double hD, const Control* ctl,
                     cudaStream_t s) {
  const int g = partials ? nblocks : grid_for(lv.V, kT, kCap);
  k_residual<D, T, TX><<<g, kT, 0, s>>>(lv, x, b, r, r32, partials, hD, ctl);
}

template <int D, typename T>
void launch_restrict(const LevelView<T>& lf, const LevelView<T>& lc, const CycleParams<T>& cp,
                     const T* r_f, const T* y_f, T* r_c, int rc_given, T* bt_c, T* g_c,
                     T gscale, const Control* ctl, cudaStream_t s) {
  // one warp per coarse vertex
  k_restrict<D, T><<<grid_for(lc.V * 32, kT, kCap), kT, 0, s>>>(lf, lc, cp, r_f, y_f, r_c,
                                                               rc_given, bt_c, g_c, gscale, ctl);
}

template <int D, typename T>
void launch_apply_scaled(const LevelView<T>& lv, const T* r, T* y, const Control* ctl,
                         cudaStream_t s) {
  k_apply_scaled<D, T><<<grid_for(lv.V, kT, kCap), kT, 0, s>>>(lv, r, y, ctl);
}

template <int D, typename T>
void launch_prolong(const LevelView<T>& lf, const LevelView<T>& lc, const CycleParams<T>& cp,
                    const T* t_c, const T* g_f, T* t_f, const Control* ctl, cudaStream_t s) {
  k_prolong<D, T><<<grid_for(lf.V, kT, kCap), kT, 0, s>>>(lf, lc, cp, t_c, g_f, t_f, ctl);
}

template <int D, typename T, typename TX>
void launch_update(const LevelView<T>& lf, const LevelView<T>& lc, const CycleParams<T>& cp,
                   const T* r_f, const T* t_c, TX* x, const Control* ctl, cudaStream_t s) {
  k_update<D, T, TX><<<grid_for(lf.V, kT, kCap), kT, 0, s>>>(lf, lc, cp, r_f, t_c, x,
                                                            const_cast<Control*>(ctl));
}

template <int D>
void launch_hierarchical(const LevelView<double>& lf, const LevelView<double>& lc,
                         const double* u_f, const double* u_c, double* uhat, const Control* ctl,
                         cudaStream_t s) {
  k_hierarchical<D><<<grid_for(lf.V, kT, kCap), kT, 0, s>>>(lf, lc, u_f, u_c, uhat, ctl);
}

template <int D>
void launch_inject(const double* u_f, int n_f, double* u_c, const Control* ctl, cudaStream_t s) {
  long long V = 1;
  for (int j = 0; j < D; ++j) V *= n_f / 3 + 1;
  k_inject<D><<<grid_for(V, kT, kCap), kT, 0, s>>>(u_f, n_f, u_c, ctl);
}

template <int D>
void launch_restrict_plain(const LevelView<double>& lf, const LevelView<double>& lc,
                           const double* r_f, double* b_c, const Control* ctl, cudaStream_t s) {
  k_restrict_plain<D><<<grid_for(lc.V, kT, kCap), kT, 0, s>>>(lf, lc, r_f, b_c, ctl);
}

void launch_norm_finalize(const double* partials, int nblocks, Control* ctl, double* hist,
                          int hist_cap, int query, cudaStream_t s) {
  k_norm_finalize<<<1, 256, 0, s>>>(partials, nblocks, ctl, hist, hist_cap, query);
}

void launch_reset_control(Control* ctl, cudaStream_t s) { k_reset_control<<<1, 1, 0, s>>>(ctl); }

void launch_refine_update(double* u, float* e, long long V, const Control* ctl, cudaStream_t s) {
  k_refine_update<<<grid_for(V, kT, kCap), kT, 0, s>>>(u, e, V, ctl);
}

#define ADAFAC_CYCLE_INST_T(D, T)                                                               \
  template void launch_residual<D, T, T>(const LevelView<T>&, const T*, const T*, T*, float*,   \
                                         double*, int, double, const Control*, cudaStream_t);   \
  template void launch_restrict<D, T>(const LevelView<T>&, const LevelView<T>&,                 \
                                      const CycleParams<T>&, const T*, const T*, T*, int, T*,   \
                                      T*, T, const Control*, cudaStream_t);                     \
  template void launch_apply_scaled<D, T>(const LevelView<T>&, const T*, T*, const Control*,    \
                                          cudaStream_t);                                        \
  template void launch_prolong<D, T>(const LevelView<T>&, const LevelView<T>&,                  \
                                     const CycleParams<T>&, const T*, const T*, T*,             \
                                     const Control*, cudaStream_t);                             \
  template void launch_update<D, T, T>(const LevelView<T>&, const LevelView<T>&,                \
                                       const CycleParams<T>&, const T*, const T*, T*,           \
                                       const Control*, cudaStream_t);

#define ADAFAC_CYCLE_INST(D)                                                                    \
  ADAFAC_CYCLE_INST_T(D, double)                                                                \
  ADAFAC_CYCLE_INST_T(D, float)                                                                 \
  template void launch_hierarchical<D>(const LevelView<double>&, const LevelView<double>&,      \
                                       const double*, const double*, double*, const Control*,   \
                                       cudaStream_t);                                           \
  template void launch_inject<D>(const double*, int, double*, const Control*, cudaStream_t);    \
  template void launch_restrict_plain<D>(const LevelView<double>&, const LevelView<double>&,    \
                                         const double*, double*, const Control*, cudaStream_t);

ADAFAC_CYCLE_INST(2)
ADAFAC_CYCLE_INST(3)

}  // namespace adafac
