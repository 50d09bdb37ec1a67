// Level kernels of the mixed-precision cycles for every configuration the
// fused 3-D sweeps do not cover: varying eps (per-cell), BoxMG transfers,
// adAFAC-PI, exact R~, fewer levels.  Each step of Algorithm 1 is one launch
// per level, as in cycle.cu, but the launches are shaped like the grids:
// threads map to vertices (or coarse vertices) through the block and grid
// coordinates, with no index decoding, and the stencil offsets, transfer
// weights and window positions are compile-time constants.
//
//   residual  r = b - A x at the vertices of the finest level (Alg. 1), A the
//             d-linear FEM operator assembled on the fly from per-cell eps
//             (Sec. 2.1).  3-D: each thread marches a column of vertices in
//             z and keeps three planes of its 3 x 3 neighbourhood and two
//             layers of its cells' eps in registers.  FP32 for the cycles;
//             FP64 for the refinement residual, with per-block sums of
//             h^D r^2 (Eq. 10).
//   restrict  r_c = P^T r_f, b~_c = omega S~^T r_f (Eq. 8, truncated R~),
//             g_c = M_c^-1 (omega r_c - omega~ b~_c) (Eq. 9), one thread per
//             coarse vertex over the 5^D window of fine vertices.
//   prolong   t_f = g_f + P q_c (the nested form of Eq. 9) on coarse levels.
//   update    x += omega M^-1 r + P q_c on the finest level (Alg. 1, Eq. 9).
//
// Element matrix of the d-linear element by the Hamming distance of the two
// corners (Sec. 2.1; eps = 1, without the h^(D-2) factor):
//   2-D: 2/3, -1/6, -1/3          3-D: 1/3, 0, -1/12, -1/12
// so in 3-D a vertex and the 4 corners of an adjacent cell that do not share
// a cell edge with it couple with the same weight, and the 3 that do share
// one do not couple at all.
#include "common.cuh"

namespace adafac {

namespace {

constexpr int FX = 32, FY = 8;   // default threads per block on vertex grids (x, y)
constexpr int kMaxThreads = 256; // largest block of the vertex-grid kernels
constexpr int ZRMAX = 16;        // most planes per thread column of the 3-D residual
constexpr int CX = 32, CY = 4;   // threads per block of the restriction (x, y)

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Planes per thread column of the 3-D residual: long columns (fewer plane
// reloads) as long as the grid still has about two blocks per SM of a
// 152-SM GPU; one plane per column on small grids.
inline int residual_zr(int np1, int bx = FX, int by = FY) {
  const int xy = cdiv(np1, bx) * cdiv(np1, by);
  const int zr = np1 * xy / (2 * 152);
  return zr < 1 ? 1 : (zr > ZRMAX ? ZRMAX : zr);
}

template <int D>
inline int zblocks_residual(int np1, int zr) {
  return D == 3 ? cdiv(np1, zr) : 1;
}

// The launch shape actually used: zr = 0 takes the size rule above.
inline GridShape resolve(GridShape g, int np1) {
  if (g.bx <= 0 || g.by <= 0) g.bx = FX, g.by = FY;
  if (g.zr <= 0) g.zr = residual_zr(np1, g.bx, g.by);
  return g;
}

// Block sum of acc in a fixed order (warp shuffles, then the warps in order),
// written to partials[block] scaled by hD.
__device__ __forceinline__ void block_partial(double acc, double hD, double* partials) {
  __shared__ double red[kMaxThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int nw = (blockDim.x * blockDim.y) >> 5;  // block shapes are whole warps
  if ((t & 31) == 0) red[t >> 5] = acc;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s * hD;
  }
}

// ---------------------------------------------------------------------------
// 3-D residual: thread (x, y) marches z = z0 .. z0 + zr - 1.  E0, E1, E2 hold
// x at planes z - 1, z, z + 1 on the 3 x 3 neighbourhood ([dy + 1][dx + 1]);
// cb / ca the eps of the 4 cells below / above vertex z ([sy][sx], cell x - 1
// + sx, y - 1 + sy).  For the cell on side (sx, sy, sz) the corners without a
// shared cell edge are (sx, sy, 0), (sx, 0, sz), (0, sy, sz), (sx, sy, sz).
template <typename T, typename TO, bool EPS, bool NORM>
__global__ void __launch_bounds__(kMaxThreads)
    k_residual3g(const LevelView<T> lv, const T* __restrict__ x, const T* __restrict__ b,
                 TO* __restrict__ r, double* __restrict__ partials, double hD, int zr,
                 const Control* ctl) {
  if (halted(ctl)) return;
  constexpr T K0 = T(1.0 / 3.0), KD = T(-1.0 / 12.0);
  const int n = lv.n, np1 = n + 1;
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y * blockDim.y + threadIdx.y;
  const int z0 = blockIdx.z * zr, z1 = min(z0 + zr, np1);
  const int P = np1 * np1;
  double acc = 0.0;
  if (ix <= n && iy <= n) {
    int v = (z0 * np1 + iy) * np1 + ix;
    const bool col = ix >= 1 && ix <= n - 1 && iy >= 1 && iy <= n - 1;
    if (!col) {
      for (int z = z0; z < z1; ++z, v += P) r[v] = TO(0);
    } else {
      T E0[9], E1[9], E2[9], cb[4], ca[4];
      auto load_plane = [&](T* E, int vz) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) E[(dy + 1) * 3 + dx + 1] = x[vz + dy * np1 + dx];
      };
      auto load_cells = [&](T* c, int z) {
        const int cz = (z * n + iy - 1) * n + ix - 1;
#pragma unroll
        for (int sy = 0; sy < 2; ++sy)
#pragma unroll
          for (int sx = 0; sx < 2; ++sx) c[sy * 2 + sx] = EPS ? lv.eps[cz + sy * n + sx] : lv.eps0;
      };
      if (z0 >= 1) {
        load_plane(E0, v - P);
        load_cells(cb, z0 - 1);
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) E0[k] = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) cb[k] = T(0);
      }
      load_plane(E1, v);
      for (int z = z0; z < z1; ++z, v += P) {
        if (z + 1 <= n) {
          load_plane(E2, v + P);
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) E2[k] = T(0);
        }
        if (z <= n - 1) {
          load_cells(ca, z);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) ca[k] = T(0);
        }
        T rv = T(0);
        if (z >= 1 && z <= n - 1) {
          T esum = T(0), far = T(0);
#pragma unroll
          for (int sz = 0; sz < 2; ++sz) {
            const T* S = sz ? E2 : E0;
            const T* ce = sz ? ca : cb;
#pragma unroll
            for (int sy = 0; sy < 2; ++sy)
#pragma unroll
              for (int sx = 0; sx < 2; ++sx) {
                const int iy3 = 2 * sy, ix3 = 2 * sx;  // neighbour index 0 (-1) or 2 (+1)
                const T f = (E1[iy3 * 3 + ix3] + S[3 + ix3]) + (S[iy3 * 3 + 1] + S[iy3 * 3 + ix3]);
                const T e = ce[sy * 2 + sx];
                esum += e;
                far += e * f;
              }
          }
          const T Ax = lv.hfac * (K0 * E1[4] * esum + KD * far);
          rv = b[v] - Ax;
          if (NORM) acc += (double)rv * (double)rv;
        }
        r[v] = TO(rv);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          E0[k] = E1[k];
          E1[k] = E2[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) cb[k] = ca[k];
      }
    }
  }
  if (NORM) block_partial(acc, hD, partials);
}

// 2-D residual: one thread per vertex.  For the cell on side (sx, sy) the
// corners at Hamming distance 1 are (sx, 0) and (0, sy), at distance 2 (sx, sy).
template <typename T, typename TO, bool EPS, bool NORM>
__global__ void __launch_bounds__(kMaxThreads)
    k_residual2g(const LevelView<T> lv, const T* __restrict__ x, const T* __restrict__ b,
                 TO* __restrict__ r, double* __restrict__ partials, double hD,
                 const Control* ctl) {
  if (halted(ctl)) return;
  constexpr T K0 = T(2.0 / 3.0), K1 = T(-1.0 / 6.0), K2 = T(-1.0 / 3.0);
  const int n = lv.n, np1 = n + 1;
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y * blockDim.y + threadIdx.y;
  double acc = 0.0;
  if (ix <= n && iy <= n) {
    const int v = iy * np1 + ix;
    T rv = T(0);
    if (ix >= 1 && ix <= n - 1 && iy >= 1 && iy <= n - 1) {
      T E[9];
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) E[(dy + 1) * 3 + dx + 1] = x[v + dy * np1 + dx];
      const int c0 = (iy - 1) * n + ix - 1;
      T Ax = T(0);
#pragma unroll
      for (int sy = 0; sy < 2; ++sy)
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
          const T e = EPS ? lv.eps[c0 + sy * n + sx] : lv.eps0;
          const int iy3 = 2 * sy, ix3 = 2 * sx;
          const T inner = K0 * E[4] + K1 * (E[3 + ix3] + E[iy3 * 3 + 1]) + K2 * E[iy3 * 3 + ix3];
          Ax += e * inner;
        }
      rv = b[v] - lv.hfac * Ax;
      if (NORM) acc += (double)rv * (double)rv;
    }
    r[v] = TO(rv);
  }
  if (NORM) block_partial(acc, hD, partials);
}

// ---------------------------------------------------------------------------
// Restriction to coarse level lc and the level's combined correction, one
// thread per coarse vertex J over the fine window 3J + o, o in [-2, 2]^D.
// The weight of fine vertex 3J + o towards J: d-linear prod_j (1 - |o_j|/3);
// BoxMG the stored weight towards corner e of the fine vertex's own coarse
// cell, e_j = 1 where o_j < 0 (the cell below J along j), else 0.
template <int D, bool BOXMG, bool JAC>
__global__ void __launch_bounds__(CX* CY)
    k_restrict_g(const LevelView<float> lf, const LevelView<float> lc,
                 const CycleParams<float> cp, const float* __restrict__ r_f,
                 float* __restrict__ r_c, float* __restrict__ bt_c, float* __restrict__ g_c,
                 float gscale, const Control* ctl) {
  if (halted(ctl)) return;
  constexpr int NC = 1 << D;
  const int nc = lc.n, ncp1 = nc + 1, np1 = lf.np1;
  const int Jx = blockIdx.x * CX + threadIdx.x, Jy = blockIdx.y * CY + threadIdx.y;
  const int Jz = D == 3 ? (int)blockIdx.z : 0;
  if (Jx > nc || Jy > nc) return;
  const int vc = (Jz * ncp1 + Jy) * ncp1 + Jx;
  const bool interior = Jx >= 1 && Jx <= nc - 1 && Jy >= 1 && Jy <= nc - 1 &&
                        (D == 2 || (Jz >= 1 && Jz <= nc - 1));
  if (!interior) {
    r_c[vc] = 0.f;
    if (bt_c) bt_c[vc] = 0.f;
    g_c[vc] = 0.f;
    return;
  }
  const int f0 = ((3 * Jz) * np1 + 3 * Jy) * np1 + 3 * Jx;
  const float* Pe[NC];
#pragma unroll
  for (int e = 0; e < NC; ++e) Pe[e] = BOXMG ? lf.P + (long long)e * lf.V : nullptr;
  // one partial sum per window row (oy), added in a fixed order at the end:
  // five independent FMA chains instead of one
  float rcs[5], bts[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) rcs[i] = bts[i] = 0.f;
  constexpr int OZ = D == 3 ? 2 : 0;
#pragma unroll
  for (int oz = -OZ; oz <= OZ; ++oz)
#pragma unroll
    for (int oy = -2; oy <= 2; ++oy) {
      const int row = f0 + (oz * np1 + oy) * np1;
#pragma unroll
      for (int ox = -2; ox <= 2; ++ox) {
        const int f = row + ox;
        const float rv = r_f[f];
        float w;
        if (BOXMG) {
          const int e = (ox < 0 ? 1 : 0) | (oy < 0 ? 2 : 0) | (oz < 0 ? 4 : 0);
          w = Pe[e][f];
        } else {
          w = (1.f - (ox < 0 ? -ox : ox) * (1.f / 3.f)) * (1.f - (oy < 0 ? -oy : oy) * (1.f / 3.f)) *
              (1.f - (oz < 0 ? -oz : oz) * (1.f / 3.f));
        }
        rcs[oy + 2] = fmaf(w, rv, rcs[oy + 2]);
        if (JAC) {
          const int k = ((oz + OZ) * 5 + (oy + 2)) * 5 + (ox + 2);
          bts[oy + 2] = fmaf(cp.stilde[k], rv, bts[oy + 2]);
        }
      }
    }
  float rc = (rcs[0] + rcs[1]) + (rcs[2] + (rcs[3] + rcs[4]));
  float bt = (bts[0] + bts[1]) + (bts[2] + (bts[3] + bts[4]));
  const float id = lc.invd ? lc.invd[vc] : lc.invd0;
  r_c[vc] = rc;
  float g;
  if (JAC) {
    bt *= cp.omega;
    bt_c[vc] = bt;
    g = id * (cp.omega * rc - cp.omega_tilde * bt);
  } else {
    if (bt_c) bt_c[vc] = 0.f;
    g = gscale * cp.omega * id * rc;
  }
  g_c[vc] = g;
}

// ---------------------------------------------------------------------------
// Prolongation onto level lf from its coarse level lc, one thread per vertex:
//   UPDATE  (finest level)  x += omega M^-1 r + P q
//   else    (coarse level)  t = g + P q, zero on the boundary
// q = t_c, minus (for adAFAC-PI) the level's own Jacobi correction at the
// fine vertex that coincides with the coarse corner.  A fine vertex with
// local offset l_j = 0 inside its coarse cell takes no weight from the
// corners with e_j = 1 (for BoxMG as for d-linear weights): those corners are
// skipped; every other corner is summed, also where its weight is zero.
template <int D, bool UPDATE, bool BOXMG, bool PI>
__global__ void __launch_bounds__(kMaxThreads)
    k_prolong_g(const LevelView<float> lf, const LevelView<float> lc, const CycleParams<float> cp,
                const float* __restrict__ r_f, const float* __restrict__ g_f,
                const float* __restrict__ t_c, float* __restrict__ x, Control* ctl) {
  if (halted(ctl)) return;
  constexpr int NC = 1 << D;
  if (UPDATE && ctl && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 &&
      threadIdx.x == 0 && threadIdx.y == 0)
    atomicAdd(&ctl->applied, 1);
  const int n = lf.n, np1 = n + 1;
  const int c[3] = {(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(blockIdx.y * blockDim.y + threadIdx.y),
                    D == 3 ? (int)blockIdx.z : 0};
  if (c[0] > n || c[1] > n) return;
  const int v = (c[2] * np1 + c[1]) * np1 + c[0];
  bool interior = true;
#pragma unroll
  for (int j = 0; j < D; ++j) interior = interior && c[j] >= 1 && c[j] <= n - 1;
  if (!interior) {
    if (!UPDATE) x[v] = 0.f;
    return;
  }
  float du = UPDATE ? cp.omega * (lf.invd ? lf.invd[v] : lf.invd0) * r_f[v] : g_f[v];
  if (lc.n > 0) {
    const int nc = lc.n, ncp1 = nc + 1;
    int O[3] = {0, 0, 0}, l[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < D; ++j) {
      O[j] = min(c[j] / 3, nc - 1);
      l[j] = c[j] - 3 * O[j];
    }
    const int cbase = (O[2] * ncp1 + O[1]) * ncp1 + O[0];
    float acc = 0.f;
#pragma unroll
    for (int e = 0; e < NC; ++e) {
      bool zero = false;
      float w = 1.f;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int bit = (e >> j) & 1;
        zero = zero || (bit && l[j] == 0);
        if (!BOXMG) {
          const float t = (float)l[j] * (1.f / 3.f);
          w *= bit ? t : 1.f - t;
        }
      }
      if (zero) continue;
      if (BOXMG) w = lf.P[(long long)e * lf.V + v];
      const int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
      float q = t_c[cbase + (ez * ncp1 + ey) * ncp1 + ex];
      if (PI) {
        // the level's Jacobi correction at the fine vertex 3 (O + e): on the
        // finest level omega M^-1 r, on a coarse level its g
        const int fx = 3 * (O[0] + ex), fy = 3 * (O[1] + ey), fz = D == 3 ? 3 * (O[2] + ez) : 0;
        const int fc = (fz * np1 + fy) * np1 + fx;
        if (UPDATE)
          q -= cp.omega * (lf.invd ? lf.invd[fc] : lf.invd0) * r_f[fc];
        else
          q -= g_f[fc];
      }
      acc += w * q;
    }
    du += acc;
  }
  if (UPDATE) x[v] = x[v] + du;
  else x[v] = du;
}

}  // namespace

template <int D>
int residual_g_blocks(int n) {
  const int np1 = n + 1;
  const GridShape g = resolve(GridShape(), np1);
  return cdiv(np1, g.bx) * cdiv(np1, g.by) * zblocks_residual<D>(np1, g.zr);
}

template <int D, typename T, typename TO>
void launch_residual_g(const LevelView<T>& lv, const T* x, const T* b, TO* r, double* partials,
                       double hD, const Control* ctl, cudaStream_t s, GridShape shape) {
  const int np1 = lv.n + 1;
  const GridShape g = resolve(shape, np1);
  const dim3 grid(cdiv(np1, g.bx), cdiv(np1, g.by), zblocks_residual<D>(np1, g.zr)), block(g.bx, g.by);
  const bool eps = lv.opkind == OP_EPS;
  if (D == 3) {
    const int zr = g.zr;
    if (eps) {
      if (partials) k_residual3g<T, TO, true, true><<<grid, block, 0, s>>>(lv, x, b, r, partials, hD, zr, ctl);
      else k_residual3g<T, TO, true, false><<<grid, block, 0, s>>>(lv, x, b, r, partials, hD, zr, ctl);
    } else {
      if (partials) k_residual3g<T, TO, false, true><<<grid, block, 0, s>>>(lv, x, b, r, partials, hD, zr, ctl);
      else k_residual3g<T, TO, false, false><<<grid, block, 0, s>>>(lv, x, b, r, partials, hD, zr, ctl);
    }
  } else {
    if (eps) {
      if (partials) k_residual2g<T, TO, true, true><<<grid, block, 0, s>>>(lv, x, b, r, partials, hD, ctl);
      else k_residual2g<T, TO, true, false><<<grid, block, 0, s>>>(lv, x, b, r, partials, hD, ctl);
    } else {
      if (partials) k_residual2g<T, TO, false, true><<<grid, block, 0, s>>>(lv, x, b, r, partials, hD, ctl);
      else k_residual2g<T, TO, false, false><<<grid, block, 0, s>>>(lv, x, b, r, partials, hD, ctl);
    }
  }
}

template <int D>
void launch_restrict_g(const LevelView<float>& lf, const LevelView<float>& lc,
                       const CycleParams<float>& cp, const float* r_f, float* r_c, float* bt_c,
                       float* g_c, float gscale, const Control* ctl, cudaStream_t s) {
  const int ncp1 = lc.n + 1;
  const dim3 grid(cdiv(ncp1, CX), cdiv(ncp1, CY), D == 3 ? ncp1 : 1), block(CX, CY);
  const bool jac = cp.variant == V_JAC;
  if (lf.boxmg) {
    if (jac) k_restrict_g<D, true, true><<<grid, block, 0, s>>>(lf, lc, cp, r_f, r_c, bt_c, g_c, gscale, ctl);
    else k_restrict_g<D, true, false><<<grid, block, 0, s>>>(lf, lc, cp, r_f, r_c, bt_c, g_c, gscale, ctl);
  } else {
    if (jac) k_restrict_g<D, false, true><<<grid, block, 0, s>>>(lf, lc, cp, r_f, r_c, bt_c, g_c, gscale, ctl);
    else k_restrict_g<D, false, false><<<grid, block, 0, s>>>(lf, lc, cp, r_f, r_c, bt_c, g_c, gscale, ctl);
  }
}

template <int D, bool UPDATE>
void launch_prolong_g(const LevelView<float>& lf, const LevelView<float>& lc,
                      const CycleParams<float>& cp, const float* r_f, const float* g_f,
                      const float* t_c, float* x, Control* ctl, cudaStream_t s,
                      GridShape shape) {
  const int np1 = lf.n + 1;
  const GridShape g = resolve(shape, np1);
  const dim3 grid(cdiv(np1, g.bx), cdiv(np1, g.by), D == 3 ? np1 : 1), block(g.bx, g.by);
  const bool pi = cp.variant == V_PI;
  if (lf.boxmg) {
    if (pi) k_prolong_g<D, UPDATE, true, true><<<grid, block, 0, s>>>(lf, lc, cp, r_f, g_f, t_c, x, ctl);
    else k_prolong_g<D, UPDATE, true, false><<<grid, block, 0, s>>>(lf, lc, cp, r_f, g_f, t_c, x, ctl);
  } else {
    if (pi) k_prolong_g<D, UPDATE, false, true><<<grid, block, 0, s>>>(lf, lc, cp, r_f, g_f, t_c, x, ctl);
    else k_prolong_g<D, UPDATE, false, false><<<grid, block, 0, s>>>(lf, lc, cp, r_f, g_f, t_c, x, ctl);
  }
}

#define ADAFAC_LEVEL_INST(D)                                                                   \
  template int residual_g_blocks<D>(int);                                                      \
  template void launch_residual_g<D, float, float>(const LevelView<float>&, const float*,      \
                                                   const float*, float*, double*, double,      \
                                                   const Control*, cudaStream_t, GridShape);   \
  template void launch_residual_g<D, double, float>(const LevelView<double>&, const double*,   \
                                                    const double*, float*, double*, double,    \
                                                    const Control*, cudaStream_t, GridShape);  \
  template void launch_restrict_g<D>(const LevelView<float>&, const LevelView<float>&,         \
                                     const CycleParams<float>&, const float*, float*, float*,  \
                                     float*, float, const Control*, cudaStream_t);             \
  template void launch_prolong_g<D, true>(const LevelView<float>&, const LevelView<float>&,    \
                                          const CycleParams<float>&, const float*,             \
                                          const float*, const float*, float*, Control*,        \
                                          cudaStream_t, GridShape);                            \
  template void launch_prolong_g<D, false>(const LevelView<float>&, const LevelView<float>&,   \
                                           const CycleParams<float>&, const float*,            \
                                           const float*, const float*, float*, Control*,       \
                                           cudaStream_t, GridShape);

ADAFAC_LEVEL_INST(2)
ADAFAC_LEVEL_INST(3)

}  // namespace adafac
