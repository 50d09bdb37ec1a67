// Device helpers shared by the setup and cycle kernels.
#pragma once

#include "engine.h"

namespace adafac {

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

// Linear index -> coordinates.  Every array of the library has fewer than
// 2^31 entries, so 32-bit unsigned division suffices (much cheaper than the
// 64-bit form).
template <int D>
__device__ __forceinline__ void decode(long long v, int np1, int* c) {
  unsigned w = (unsigned)v;
  const unsigned m = (unsigned)np1;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const unsigned q = w / m;
    c[j] = (int)(w - q * m);
    w = q;
  }
}

template <int D>
__device__ __forceinline__ long long encode(const int* c, int np1) {
  long long r = c[D - 1];
#pragma unroll
  for (int j = D - 2; j >= 0; --j) r = r * np1 + c[j];
  return r;
}

template <int D>
__device__ __forceinline__ bool is_interior(const int* c, int n) {
#pragma unroll
  for (int j = 0; j < D; ++j)
    if (c[j] <= 0 || c[j] >= n) return false;
  return true;
}

// Linear offset of stencil entry s (offsets in {-1,0,1}^D).
template <int D>
__device__ __forceinline__ long long stencil_offset(int s, int np1) {
  long long off = 0, stride = 1;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    off += (long long)((s % 3) - 1) * stride;
    s /= 3;
    stride *= np1;
  }
  return off;
}

// d-linear element stiffness on the reference cell, by the Hamming distance
// of the two corners (Sec. 2.1: bi-/trilinear shape functions):
//   2-D: 2/3, -1/6, -1/3      3-D: 1/3, 0, -1/12, -1/12
template <int D, typename T>
__device__ __forceinline__ T kref(int ham) {
  if (D == 2) return ham == 0 ? T(2.0 / 3.0) : (ham == 1 ? T(-1.0 / 6.0) : T(-1.0 / 3.0));
  return ham == 0 ? T(1.0 / 3.0) : (ham == 1 ? T(0) : T(-1.0 / 12.0));
}

// (A x)_v at an interior vertex with coordinates c.
template <int D, typename T, typename TX>
__device__ __forceinline__ T apply_op(const LevelView<T>& lv, const TX* __restrict__ x,
                                      const int* c, long long v) {
  constexpr int NC = 1 << D;
  if (lv.opkind == OP_EPS) {
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      int cell[D];
#pragma unroll
      for (int j = 0; j < D; ++j) cell[j] = c[j] - ((a >> j) & 1);
      const T e = lv.eps[encode<D>(cell, lv.n)];
      T inner = T(0);
#pragma unroll
      for (int b = 0; b < NC; ++b) {
        int w[D];
#pragma unroll
        for (int j = 0; j < D; ++j) w[j] = cell[j] + ((b >> j) & 1);
        inner += kref<D, T>(__popc(a ^ b)) * T(x[encode<D>(w, lv.np1)]);
      }
      acc += e * inner;
    }
    return lv.hfac * acc;
  }
  constexpr int NS = ipow_c(3, D);
  T acc = T(0);
  if (lv.opkind == OP_STORED) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
      acc += lv.st[(long long)s * lv.V + v] * T(x[v + stencil_offset<D>(s, lv.np1)]);
  } else {
#pragma unroll
    for (int s = 0; s < NS; ++s)
      acc += lv.cst[s] * T(x[v + stencil_offset<D>(s, lv.np1)]);
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ T inv_diag(const LevelView<T>& lv, long long v) {
  return lv.invd ? lv.invd[v] : lv.invd0;
}

// Weight of fine vertex fc (coords on the fine level) towards the coarse
// vertex J, for fine points within [-2, 2]^D of 3J.
template <int D, typename T>
__device__ __forceinline__ T p_weight(const LevelView<T>& lf, int n_c, const int* fc,
                                      long long fv, const int* J) {
  if (!lf.boxmg) {
    T w = T(1);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      int o = fc[j] - 3 * J[j];
      o = o < 0 ? -o : o;
      w *= T(1) - T(o) * T(1.0 / 3.0);
    }
    return w;
  }
  int e = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    int own = fc[j] / 3;
    own = own < n_c - 1 ? own : n_c - 1;
    const int bit = J[j] - own;
    if (bit < 0 || bit > 1) return T(0);
    e |= bit << j;
  }
  return lf.P[(long long)e * lf.V + fv];
}

// Prolongation weight of fine vertex (owning cell O, local offset l in 0..3)
// towards corner e of O.
template <int D, typename T>
__device__ __forceinline__ T p_corner_weight(const LevelView<T>& lf, const int* l, int e,
                                             long long fv) {
  if (!lf.boxmg) {
    T w = T(1);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const T t = T(l[j]) * T(1.0 / 3.0);
      w *= ((e >> j) & 1) ? t : T(1) - t;
    }
    return w;
  }
  return lf.P[(long long)e * lf.V + fv];
}

// a kernel of a batch returns at entry once the solve has converged or
// diverged, or once a bounded device-side wait of an earlier kernel gave up
__device__ __forceinline__ bool halted(const Control* ctl) {
  return ctl && (ctl->done || ctl->diverged || ctl->fault);
}

}  // namespace adafac
