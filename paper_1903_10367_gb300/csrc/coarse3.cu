// The coarse levels of the 3-D uniform path (d-linear transfers, uniform
// coarse operators, FP32): every cycle restricts level by level from L - 1
// down to lmin and prolongs back up (the nested form of Eq. 9):
//   r_l = P^T r_{l+1},  b~_l = omega S~^T r_{l+1},
//   g_l = M_l^-1 (omega r_l - omega~ b~_l)            [adAFAC-Jac]
//       = gscale_l omega M_l^-1 r_l                   [additive, exponential]
//   t_lmin = g_lmin,  t_l = g_l + P t_{l-1}.
// With the d-linear weights as constants and the grid coordinates taken from
// the launch shape, each step is one short launch: the restriction spreads a
// coarse vertex's 5^3 window over five threads (one plane each), the
// prolongation gives a row of fine vertices to a block.  With lmin = 1 the
// bottom of the chain (restriction 2 -> 1, prolongations 1 -> 2 and 2 -> 3)
// is one launch: every block of the 2 -> 3 prolongation recomputes the eight
// interior vertices of level 1 from level 2 (1000 values, staged in shared
// memory) and the level-2 values its row interpolates from, with the same
// arithmetic as the separate kernels.
#include "coarse3.cuh"
#include "common.cuh"
#include "sweep3.cuh"

namespace adafac {

namespace {

// weights of fine index i towards coarse I = min(i / 3, nc - 1) and I + 1
__device__ __forceinline__ void lerp_at(int i, int nc, int* I, float* t) {
  int c = i / 3;
  c = c < nc - 1 ? c : nc - 1;
  *I = c;
  *t = (float)(i - 3 * c) * (1.f / 3.f);
}

// The restriction's sums over plane oz of a coarse vertex's 5^3 window (the
// plane's 25 values, x fastest): the d-linear weights (times the z factor)
// and the S~ block of the plane.
__device__ __forceinline__ void restrict_plane(const float (&val)[25], int oz,
                                               const float* stilde, float* rs, float* bs) {
  constexpr float kW[5] = {1.f / 3.f, 2.f / 3.f, 1.f, 2.f / 3.f, 1.f / 3.f};
  // the weights of plane oz: the z factor and the S~ block are selected once
  const float wz = kW[oz];
  float r0 = 0.f, r1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
  for (int k = 0; k < 25; ++k) {
    const float wr = kW[k % 5] * kW[k / 5];
    const float ws = stilde[oz * 25 + k];
    if (k & 1) {
      r1 = fmaf(wr, val[k], r1);
      b1 = fmaf(ws, val[k], b1);
    } else {
      r0 = fmaf(wr, val[k], r0);
      b0 = fmaf(ws, val[k], b0);
    }
  }
  *rs = wz * (r0 + r1);
  *bs = b0 + b1;
}

// r, b~ and g of an interior coarse vertex from its five plane sums (added in
// the order oz = 0 .. 4)
__device__ __forceinline__ void restrict_finish(const Level3Params& p, const float* prs,
                                                const float* pbs, int stride, float id,
                                                float* r, float* bt, float* g) {
  float rc = 0.f, b = 0.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    rc += prs[k * stride];
    b += pbs[k * stride];
  }
  float gv;
  if (p.variant == V_JAC) {
    b *= p.omega;
    gv = id * (p.omega * rc - p.omega_t * b);
  } else {
    b = 0.f;
    gv = p.gscale * p.omega * id * rc;
  }
  *r = rc;
  *bt = b;
  *g = gv;
}

// Restriction to level l: five threads per coarse vertex, one per plane oz of
// its window (25 loads issued together, the d-linear weights and S~ as
// immediates); the plane sums are added in the order oz = 0 .. 4 through
// shared memory.  Boundary vertices get zeros.
constexpr int kRestrictVerts = 64;
__global__ void __launch_bounds__(5 * kRestrictVerts)
    k_restrict3u(const __grid_constant__ Level3Params p) {
  __shared__ float s_r[5][kRestrictVerts], s_b[5][kRestrictVerts];
  if (halted(p.ctl)) return;
  const int nc = p.nc, ncp1 = nc + 1, nfp1 = 3 * nc + 1;
  const int oz = threadIdx.y;
  const int v = blockIdx.x * kRestrictVerts + threadIdx.x;
  const int Vc = ncp1 * ncp1 * ncp1;
  const int x = v % ncp1, yz = v / ncp1, y = yz % ncp1, z = yz / ncp1;
  const bool interior = v < Vc && x > 0 && x < nc && y > 0 && y < nc && z > 0 && z < nc;
  float rs = 0.f, bs = 0.f;
  if (interior) {
    const float* w0 =
        p.r_f + ((long long)(3 * z - 2 + oz) * nfp1 + (3 * y - 2)) * nfp1 + (3 * x - 2);
    float val[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) val[k] = __ldg(w0 + (long long)(k / 5) * nfp1 + k % 5);
    restrict_plane(val, oz, p.stilde, &rs, &bs);
  }
  s_r[oz][threadIdx.x] = rs;
  s_b[oz][threadIdx.x] = bs;
  __syncthreads();
  if (oz != 0 || v >= Vc) return;
  if (!interior) {
    p.r_c[v] = 0.f;
    p.bt_c[v] = 0.f;
    p.g_c[v] = 0.f;
    return;
  }
  float rc, b, gv;
  restrict_finish(p, &s_r[0][threadIdx.x], &s_b[0][threadIdx.x], kRestrictVerts, p.invd_c[v],
                  &rc, &b, &gv);
  p.r_c[v] = rc;
  p.bt_c[v] = b;
  p.g_c[v] = gv;
}

// P t_c at a fine vertex from the 8 coarse values around it (c[0] .. c[7]:
// the corners (x, y, z) in the order 000 100 010 110 001 101 011 111)
__device__ __forceinline__ float trilinear(const float (&c)[8], float tx, float ty, float tz) {
  const float c000 = c[0], c100 = c[1], c010 = c[2], c110 = c[3], c001 = c[4], c101 = c[5],
              c011 = c[6], c111 = c[7];
  const float a00 = (1.f - tx) * c000 + tx * c100, a10 = (1.f - tx) * c010 + tx * c110;
  const float a01 = (1.f - tx) * c001 + tx * c101, a11 = (1.f - tx) * c011 + tx * c111;
  const float b0 = (1.f - ty) * a00 + ty * a10, b1 = (1.f - ty) * a01 + ty * a11;
  return (1.f - tz) * b0 + tz * b1;
}

// Prolongation to level l: t_f = g_f + P t_c, one row of fine vertices per
// block (x along the threads), zero on the boundary.
constexpr int kProlongRowThreads = 96;
__global__ void __launch_bounds__(kProlongRowThreads)
    k_prolong3u(const __grid_constant__ Level3Params p) {
  if (halted(p.ctl)) return;
  const int nf = p.nf, nfp1 = nf + 1, nc = p.nc, ncp1 = nc + 1;
  const int row = blockIdx.x;  // (y, z) of the fine level
  const int y = row % nfp1, z = row / nfp1;
  for (int x = threadIdx.x; x < nfp1; x += kProlongRowThreads) {
    const long long v = (long long)row * nfp1 + x;
    if (x == 0 || x == nf || y == 0 || y == nf || z == 0 || z == nf) {
      p.t_f[v] = 0.f;
      continue;
    }
    int X, Y, Z;
    float tx, ty, tz;
    lerp_at(x, nc, &X, &tx);
    lerp_at(y, nc, &Y, &ty);
    lerp_at(z, nc, &Z, &tz);
    const float* c = p.t_c + ((long long)Z * ncp1 + Y) * ncp1 + X;
    const long long sy = ncp1, sz = (long long)ncp1 * ncp1;
    const float cc[8] = {__ldg(c),      __ldg(c + 1),      __ldg(c + sy),      __ldg(c + sy + 1),
                         __ldg(c + sz), __ldg(c + sz + 1), __ldg(c + sz + sy), __ldg(c + sz + sy + 1)};
    p.t_f[v] = p.g_f[v] + trilinear(cc, tx, ty, tz);
  }
}

// The bottom of the chain with lmin = 1 (levels 1, 2, 3: 3, 9, 27 cells per
// axis) in one launch, a block per row (y, z) of level 3:
//   r_1, b~_1, g_1 from r_2 (each block, the eight interior vertices of
//   level 1; block 0 stores them), t_2 = g_2 + P g_1 on the two rows and
//   planes of level 2 the block's row interpolates from (the block whose row
//   is (3 Y, 3 Z) stores the level-2 row (Y, Z)), t_3 = g_3 + P t_2 on the
//   block's row.
constexpr int kBottomThreads = 128;
constexpr int kN1 = 3, kN2 = 9, kN3 = 27;
constexpr int kV2 = (kN2 + 1) * (kN2 + 1) * (kN2 + 1);   // 1000
__global__ void __launch_bounds__(kBottomThreads)
    k_bottom3u(const __grid_constant__ Bottom3Params p) {
  __shared__ float s_r2[kV2];
  __shared__ float s_pr[5][8], s_pb[5][8];
  __shared__ float s_g1[(kN1 + 1) * (kN1 + 1) * (kN1 + 1)];
  __shared__ float s_t2[2][2][kN2 + 1];
  const Level3Params& q21 = p.r21;
  if (halted(q21.ctl)) return;
  const int tid = threadIdx.x;
  for (int i = tid; i < kV2; i += kBottomThreads) s_r2[i] = __ldg(q21.r_f + i);
  for (int i = tid; i < (kN1 + 1) * (kN1 + 1) * (kN1 + 1); i += kBottomThreads) s_g1[i] = 0.f;
  __syncthreads();
  // level 1: interior vertex (1 + (j & 1), 1 + (j >> 1 & 1), 1 + (j >> 2)), plane oz
  constexpr int np1 = kN2 + 1;
  if (tid < 40) {
    const int j = tid % 8, oz = tid / 8;
    const int x = 1 + (j & 1), y = 1 + ((j >> 1) & 1), z = 1 + (j >> 2);
    const float* w0 = s_r2 + ((3 * z - 2 + oz) * np1 + (3 * y - 2)) * np1 + (3 * x - 2);
    float val[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) val[k] = w0[(k / 5) * np1 + k % 5];
    float rs, bs;
    restrict_plane(val, oz, q21.stilde, &rs, &bs);
    s_pr[oz][j] = rs;
    s_pb[oz][j] = bs;
  }
  __syncthreads();
  if (tid < 8) {
    const int x = 1 + (tid & 1), y = 1 + ((tid >> 1) & 1), z = 1 + (tid >> 2);
    const int v = (z * (kN1 + 1) + y) * (kN1 + 1) + x;
    float rc, b, gv;
    restrict_finish(q21, &s_pr[0][tid], &s_pb[0][tid], 8, q21.invd_c[v], &rc, &b, &gv);
    s_g1[v] = gv;
    if (blockIdx.x == 0) {
      q21.r_c[v] = rc;
      q21.bt_c[v] = b;
      q21.g_c[v] = gv;
    }
  }
  if (blockIdx.x == 0) {  // the boundary of level 1
    for (int v = tid; v < (kN1 + 1) * (kN1 + 1) * (kN1 + 1); v += kBottomThreads) {
      const int x = v % (kN1 + 1), y = (v / (kN1 + 1)) % (kN1 + 1), z = v / ((kN1 + 1) * (kN1 + 1));
      if (x == 0 || x == kN1 || y == 0 || y == kN1 || z == 0 || z == kN1) {
        q21.r_c[v] = 0.f;
        q21.bt_c[v] = 0.f;
        q21.g_c[v] = 0.f;
      }
    }
  }
  __syncthreads();
  // level 2 on the block's window: rows Y0, Y0 + 1 and planes Z0, Z0 + 1
  const int row = blockIdx.x, y3 = row % (kN3 + 1), z3 = row / (kN3 + 1);
  int Y0, Z0;
  float ty3, tz3;
  lerp_at(y3, kN2, &Y0, &ty3);
  lerp_at(z3, kN2, &Z0, &tz3);
  if (tid < 4 * np1) {
    const int X = tid % np1, a = (tid / np1) & 1, b = tid / (2 * np1);
    const int Y = Y0 + a, Z = Z0 + b;
    float t = 0.f;
    if (X != 0 && X != kN2 && Y != 0 && Y != kN2 && Z != 0 && Z != kN2) {
      int X1, Y1, Z1;
      float tx, ty, tz;
      lerp_at(X, kN1, &X1, &tx);
      lerp_at(Y, kN1, &Y1, &ty);
      lerp_at(Z, kN1, &Z1, &tz);
      const float* c = s_g1 + (Z1 * (kN1 + 1) + Y1) * (kN1 + 1) + X1;
      constexpr int sy = kN1 + 1, sz = (kN1 + 1) * (kN1 + 1);
      const float cc[8] = {c[0], c[1], c[sy], c[sy + 1], c[sz], c[sz + 1], c[sz + sy], c[sz + sy + 1]};
      t = p.p12.g_f[(Z * np1 + Y) * np1 + X] + trilinear(cc, tx, ty, tz);
    }
    s_t2[b][a][X] = t;
    // the level-2 row (Y, Z) = (y3 / 3, z3 / 3) is stored by one block
    if (y3 % 3 == 0 && z3 % 3 == 0 && Y == y3 / 3 && Z == z3 / 3)
      p.p12.t_f[(Z * np1 + Y) * np1 + X] = t;
  }
  __syncthreads();
  // level 3: the block's row
  constexpr int n3p1 = kN3 + 1;
  for (int x = tid; x < n3p1; x += kBottomThreads) {
    const long long v = (long long)row * n3p1 + x;
    if (x == 0 || x == kN3 || y3 == 0 || y3 == kN3 || z3 == 0 || z3 == kN3) {
      p.p23.t_f[v] = 0.f;
      continue;
    }
    int X;
    float tx;
    lerp_at(x, kN2, &X, &tx);
    const float cc[8] = {s_t2[0][0][X], s_t2[0][0][X + 1], s_t2[0][1][X], s_t2[0][1][X + 1],
                         s_t2[1][0][X], s_t2[1][0][X + 1], s_t2[1][1][X], s_t2[1][1][X + 1]};
    p.p23.t_f[v] = p.p23.g_f[v] + trilinear(cc, tx, ty3, tz3);
  }
}

}  // namespace

void launch_restrict3u(const Level3Params& p, cudaStream_t s) {
  const int ncp1 = p.nc + 1;
  const int V = ncp1 * ncp1 * ncp1;
  k_restrict3u<<<(V + kRestrictVerts - 1) / kRestrictVerts, dim3(kRestrictVerts, 5), 0, s>>>(p);
}

void launch_prolong3u(const Level3Params& p, cudaStream_t s) {
  const int nfp1 = p.nf + 1;
  k_prolong3u<<<nfp1 * nfp1, kProlongRowThreads, 0, s>>>(p);
}

bool bottom3u_applies(const Bottom3Params& p) {
  return p.r21.nc == kN1 && p.r21.nf == kN2 && p.p12.nc == kN1 && p.p12.nf == kN2 &&
         p.p23.nc == kN2 && p.p23.nf == kN3;
}

void launch_bottom3u(const Bottom3Params& p, cudaStream_t s) {
  k_bottom3u<<<(kN3 + 1) * (kN3 + 1), kBottomThreads, 0, s>>>(p);
}

}  // namespace adafac
