// Fused fine-level sweeps for 3-D trees whose finest operator is uniform
// (scalar eps) and whose transfers are d-linear: the hot path of the mixed
// precision cycle.
//
// One FULL sweep does, in a single pass over the finest level,
//   down of cycle k-1:  e_{k-1} = e_{k-2} + omega M^-1 (rhs - A e_{k-2}) + P q
//   up of cycle k:      rho_k = rhs - A e_{k-1},
//                       r_{L-1} = P^T rho_k,  b~_{L-1} = omega S~^T rho_k,
//                       g_{L-1} = M^-1 (omega r_{L-1} - omega~ b~_{L-1})
// (Algorithm 1 / Eq. 9 with c_L = omega M^-1 rho).  The residual of the
// previous cycle is recomputed on a halo instead of being stored, so the
// sweep reads e_{k-2} and rhs and writes e_{k-1}: 12 bytes per unknown.
//
// Blocking: a block owns BJX x BJY coarse columns of level L-1 and ZC coarse
// planes, i.e. the fine vertices whose nearest coarse vertex lies in that box
// (3 per coarse vertex and direction).  It marches through the fine planes
// in z; a plane of e_{k-2} is staged in shared memory with a halo of 3
// (stencil of the recomputed residual, stencil of the new residual,
// restriction support), per-plane in-plane sums X (4 face neighbours) and D
// (4 in-plane diagonals) are kept in registers for the three planes a 27-point
// stencil needs.  The restriction and the damping right-hand side are
// accumulated per coarse column while the planes stream by.
#include "common.cuh"
#include "sweep3.cuh"

namespace adafac {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int mod3(int t) { return (t % 3 + 3) % 3; }

template <int BJX, int BJY, int MODE>
__global__ void __launch_bounds__(NT, 2) k_sweep3(const Sweep3Params p) {
  if (halted(p.ctl)) return;
  if (MODE != SWEEP_UP && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 &&
      threadIdx.x == 0 && p.applied)
    atomicAdd(p.applied, 1);  // one down-pass (a cycle's update) per launch
  constexpr int OW = 3 * BJX, OH = 3 * BJY;            // owned fine columns
  constexpr int HB = MODE == SWEEP_FULL ? 2 : 0;       // halo of stage B (new e)
  constexpr int HA = MODE == SWEEP_UP ? 0 : HB + 1;    // halo of loaded e
  constexpr bool HAS_B = MODE != SWEEP_UP;
  constexpr bool HAS_C = MODE != SWEEP_DOWNU;
  constexpr int AW = OW + 2 * HA, AH = OH + 2 * HA;
  constexpr int BW = OW + 2 * HB, BH = OH + 2 * HB;
  constexpr int CW = OW + 2, CH = OH + 2;              // residual + restriction
  constexpr int NB = HAS_B ? (BW * BH + NT - 1) / NT : 1;
  constexpr int NCC = (CW * CH + NT - 1) / NT;
  constexpr int QW = BJX + 4, QH = BJY + 4;            // coarse q, origin J0 - 2
  constexpr int NJ = BJX * BJY;
  static_assert(2 * NJ <= NT, "one thread per coarse column and accumulator");

  __shared__ float sA[HAS_B ? 3 : 1][HAS_B ? AW * AH : 1];
  __shared__ float sB[MODE == SWEEP_FULL ? 3 : 1][MODE == SWEEP_FULL ? BW * BH : 1];
  __shared__ float sR[HAS_C ? CW * CH : 1];
  __shared__ float sQ[HAS_B ? QW * QH : 1];
  __shared__ float sX[HAS_C ? NJ : 1];

  const int n = p.n, nc = p.nc, np1 = n + 1, ncp1 = nc + 1;
  const int tid = threadIdx.x;
  const int Jx0 = blockIdx.x * BJX, Jy0 = blockIdx.y * BJY;
  const int Jz0 = blockIdx.z * p.zc;
  const int Jz1 = min(Jz0 + p.zc, ncp1);
  const int ox0 = 3 * Jx0 - 1, oy0 = 3 * Jy0 - 1;      // owned fine origin
  const int oz0 = 3 * Jz0 - 1, oz1 = 3 * Jz1 - 1;      // owned fine planes [oz0, oz1)
  // plane ranges of the stages
  const int zB0 = oz0 - HB, zB1 = oz1 + HB;            // stage B planes [zB0, zB1)
  const int zC0 = oz0 - 1, zC1 = oz1 + 1;              // stage C planes
  // pipeline: load plane t, stage B at t-1, stage C at t-2 (FULL);
  // DOWNU: stage B at t-1; UP: stage C at t (rho = rhs)
  int t0, t1;
  if (MODE == SWEEP_FULL) {
    t0 = zB0 - 1;
    t1 = zC1 + 2;
  } else if (MODE == SWEEP_DOWNU) {
    t0 = zB0 - 1;
    t1 = zB1 + 1;
  } else {
    t0 = zC0;
    t1 = zC1;
  }
  const float a_c = p.a_c, a_f = p.a_f, a_e = p.a_e, a_k = p.a_k;

  // per-thread rolling in-plane sums of the loaded e (planes t-2, t-1, t)
  float X[NB][3], Dg[NB][3];
  // per-thread rolling sums of the new e (planes s-2, s-1, s)
  float XB[NCC][3], DB[NCC][3];
#pragma unroll
  for (int k = 0; k < NB; ++k) X[k][0] = X[k][1] = X[k][2] = Dg[k][0] = Dg[k][1] = Dg[k][2] = 0.f;
#pragma unroll
  for (int k = 0; k < NCC; ++k) XB[k][0] = XB[k][1] = XB[k][2] = DB[k][0] = DB[k][1] = DB[k][2] = 0.f;
  float acc[2] = {0.f, 0.f};  // restriction (tid < NJ) or damping (NJ <= tid < 2NJ)
  const bool is_res = tid < NJ;
  const int cj = is_res ? tid : tid - NJ;
  const int cjx = cj % BJX, cjy = cj / BJX;

  for (int t = t0; t < t1; ++t) {
    const int s = t - 1;                                   // stage B plane
    const int r = MODE == SWEEP_FULL ? t - 2 : t;          // stage C plane
    // ---- (1) stage loaded plane t of e_in; coarse q for plane s ----------
    if (HAS_B) {
      const bool zin = t >= 0 && t <= n;
      float* dst = sA[mod3(t)];
      for (int i = tid; i < AW * AH; i += NT) {
        const int x = ox0 - HA + i % AW, y = oy0 - HA + i / AW;
        float v = 0.f;
        if (zin && x >= 0 && x <= n && y >= 0 && y <= n)
          v = p.e_in[((long long)t * np1 + y) * np1 + x];
        dst[i] = v;
      }
      if (s >= zB0 && s < zB1 && s >= 1 && s <= n - 1) {
        int Oz = s / 3;
        Oz = Oz < nc - 1 ? Oz : nc - 1;
        const float tz = (float)(s - 3 * Oz) * (1.f / 3.f);
        for (int i = tid; i < QW * QH; i += NT) {
          const int Jx = Jx0 - 2 + i % QW, Jy = Jy0 - 2 + i / QW;
          float v = 0.f;
          if (Jx >= 0 && Jx <= nc && Jy >= 0 && Jy <= nc) {
            const float q0 = p.q[((long long)Oz * ncp1 + Jy) * ncp1 + Jx];
            const float q1 = p.q[((long long)(Oz + 1) * ncp1 + Jy) * ncp1 + Jx];
            v = q0 + tz * (q1 - q0);
          }
          sQ[i] = v;
        }
      }
    }
    __syncthreads();
    // ---- (2) in-plane sums of plane t; stage B at plane s -----------------
    if (HAS_B) {
      const float* a = sA[mod3(t)];
      const bool doB = s >= zB0 && s < zB1;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const int i = tid + k * NT;
        if (i >= BW * BH) continue;
        const int bx = i % BW, by = i / BW;
        const int ai = (by + 1) * AW + bx + 1;             // A = B + 1 on each side
        const float xs = a[ai - 1] + a[ai + 1] + a[ai - AW] + a[ai + AW];
        const float ds = a[ai - AW - 1] + a[ai - AW + 1] + a[ai + AW - 1] + a[ai + AW + 1];
        X[k][0] = X[k][1];
        X[k][1] = X[k][2];
        X[k][2] = xs;
        Dg[k][0] = Dg[k][1];
        Dg[k][1] = Dg[k][2];
        Dg[k][2] = ds;
        if (!doB) continue;
        const int x = ox0 - HB + bx, y = oy0 - HB + by;
        float ek = 0.f;
        if (x >= 1 && x <= n - 1 && y >= 1 && y <= n - 1 && s >= 1 && s <= n - 1) {
          const float ec = sA[mod3(s)][ai];
          const float em = sA[mod3(s - 1)][ai];
          const float ep = a[ai];
          const float Ae = a_c * ec + a_f * (X[k][1] + em + ep) +
                           a_e * (Dg[k][1] + X[k][0] + X[k][2]) + a_k * (Dg[k][0] + Dg[k][2]);
          const float rho = p.rhs[((long long)s * np1 + y) * np1 + x] - Ae;
          // P q: bilinear in-plane interpolation of the z-interpolated q
          int Ox = x / 3, Oy = y / 3;
          Ox = Ox < nc - 1 ? Ox : nc - 1;
          Oy = Oy < nc - 1 ? Oy : nc - 1;
          const float tx = (float)(x - 3 * Ox) * (1.f / 3.f);
          const float ty = (float)(y - 3 * Oy) * (1.f / 3.f);
          const int qi = (Oy - (Jy0 - 2)) * QW + (Ox - (Jx0 - 2));
          const float q00 = sQ[qi], q10 = sQ[qi + 1], q01 = sQ[qi + QW], q11 = sQ[qi + QW + 1];
          const float qy0 = q00 + tx * (q10 - q00), qy1 = q01 + tx * (q11 - q01);
          const float pq = qy0 + ty * (qy1 - qy0);
          ek = ec + p.w_invd * rho + pq;
        }
        if (MODE == SWEEP_FULL) {
          sB[mod3(s)][i] = ek;
        } else {  // SWEEP_DOWNU: B region is the owned region
          if (x >= 1 && x <= n - 1 && y >= 1 && y <= n - 1 && s >= 1 && s <= n - 1 &&
              s >= oz0 && s < oz1) {
            const long long gi = ((long long)s * np1 + y) * np1 + x;
            p.u[gi] += (double)ek;
            p.e_out[gi] = 0.f;  // the zero buffer of the next refinement step
          }
        }
      }
    }
    if (!HAS_C) {
      __syncthreads();
      continue;
    }
    if (MODE == SWEEP_FULL) __syncthreads();
    // ---- (3) stage C: residual of the new e at plane r --------------------
    {
      const bool doC = r >= zC0 && r < zC1;
#pragma unroll
      for (int k = 0; k < NCC; ++k) {
        const int i = tid + k * NT;
        if (i >= CW * CH) continue;
        const int cx = i % CW, cy = i / CW;
        const int x = ox0 - 1 + cx, y = oy0 - 1 + cy;
        if (MODE == SWEEP_FULL) {
          const float* b = sB[mod3(s)];
          const int bi = (cy + 1) * BW + cx + 1;           // B = C + 1 on each side
          const float xs = b[bi - 1] + b[bi + 1] + b[bi - BW] + b[bi + BW];
          const float ds = b[bi - BW - 1] + b[bi - BW + 1] + b[bi + BW - 1] + b[bi + BW + 1];
          XB[k][0] = XB[k][1];
          XB[k][1] = XB[k][2];
          XB[k][2] = xs;
          DB[k][0] = DB[k][1];
          DB[k][1] = DB[k][2];
          DB[k][2] = ds;
          if (!doC) continue;
          float rho = 0.f;
          if (x >= 1 && x <= n - 1 && y >= 1 && y <= n - 1 && r >= 1 && r <= n - 1) {
            const float ec = sB[mod3(r)][bi];
            const float em = sB[mod3(r - 1)][bi];
            const float ep = b[bi];
            const float Ae = a_c * ec + a_f * (XB[k][1] + em + ep) +
                             a_e * (DB[k][1] + XB[k][0] + XB[k][2]) + a_k * (DB[k][0] + DB[k][2]);
            rho = p.rhs[((long long)r * np1 + y) * np1 + x] - Ae;
            if (cx >= 1 && cx <= OW && cy >= 1 && cy <= OH && r >= oz0 && r < oz1)
              p.e_out[((long long)r * np1 + y) * np1 + x] = ec;
          }
          sR[i] = rho;
        } else {  // SWEEP_UP: e = 0, rho = rhs
          if (!doC) continue;
          float rho = 0.f;
          if (x >= 1 && x <= n - 1 && y >= 1 && y <= n - 1 && r >= 1 && r <= n - 1)
            rho = p.rhs[((long long)r * np1 + y) * np1 + x];
          sR[i] = rho;
        }
      }
    }
    __syncthreads();
    // ---- (4) restriction and damping right-hand side of plane r ----------
    if (r >= zC0 && r < zC1 && tid < 2 * NJ) {
      const float* w = is_res ? p.wres : p.wdamp;
      // coarse planes receiving plane r: Jz with |r - 3 Jz| <= 2 (r >= -2)
      const int jtop = (r + 2) / 3;
      for (int Jz = jtop - 1; Jz <= jtop; ++Jz) {
        const int oz = r - 3 * Jz;
        if (oz < -2 || oz > 2 || Jz < Jz0 || Jz >= Jz1) continue;
        if (oz == -2) acc[Jz & 1] = 0.f;  // first plane of this coarse plane
        const float* wz = w + (oz + 2) * 25;
        const float* row = sR + (3 * cjy) * CW + 3 * cjx;  // window [3c, 3c + 4]
        float sum = 0.f;
#pragma unroll
        for (int oy = 0; oy < 5; ++oy)
#pragma unroll
          for (int ox = 0; ox < 5; ++ox) sum += wz[oy * 5 + ox] * row[oy * CW + ox];
        acc[Jz & 1] += sum;
      }
    }
    // finalize the coarse plane completed by plane r = 3 Jz + 2
    const int Jf = r - 2;
    const bool fin = r >= zC0 && r < zC1 && Jf >= 0 && Jf % 3 == 0 && Jf / 3 >= Jz0 &&
                     Jf / 3 < Jz1;
    if (fin && !is_res && tid < 2 * NJ) sX[cj] = acc[(Jf / 3) & 1];
    __syncthreads();
    if (fin && is_res) {
      const int Jz = Jf / 3;
      const int Jx = Jx0 + cjx, Jy = Jy0 + cjy;
      if (Jx >= 1 && Jx <= nc - 1 && Jy >= 1 && Jy <= nc - 1 && Jz >= 1 && Jz <= nc - 1) {
        const float rc = acc[Jz & 1];
        const float bt = p.omega * sX[cj];
        const long long ci = ((long long)Jz * ncp1 + Jy) * ncp1 + Jx;
        p.r_c[ci] = rc;
        if (p.variant == V_JAC) {
          p.bt_c[ci] = bt;
          p.g_c[ci] = p.c_invd * (p.omega * rc - p.omega_t * bt);
        } else {
          p.bt_c[ci] = 0.f;
          p.g_c[ci] = p.gscale * p.omega * p.c_invd * rc;
        }
      }
    }
  }
}

// FP64 residual of a uniform 3-D operator, z-marching with in-plane sums:
// rhs32 = (float)(b - A u) and per-block sums of h^3 r^2.
constexpr int RT_X = 32, RT_Y = 8;

__global__ void __launch_bounds__(RT_X* RT_Y) k_refine3(const Refine3Params p) {
  if (halted(p.ctl)) return;
  __shared__ double sU[2][(RT_X + 2) * (RT_Y + 2)];
  __shared__ double red[RT_X * RT_Y];
  const int n = p.n, np1 = n + 1;
  const int tx = threadIdx.x % RT_X, ty = threadIdx.x / RT_X;
  const int x = blockIdx.x * RT_X + tx, y = blockIdx.y * RT_Y + ty;
  const int zlo = blockIdx.z * p.zc + 1;
  const int zhi = min(zlo + p.zc, n);            // planes [zlo, zhi)
  constexpr int W = RT_X + 2;
  double Xs[3] = {0, 0, 0}, Ds[3] = {0, 0, 0}, Cs[3] = {0, 0, 0};
  double acc = 0.0;
  // planes zlo-1 .. zhi are loaded; residual at plane z uses planes z-1..z+1
  for (int z = zlo - 1; z <= zhi; ++z) {
    double* pl = sU[z & 1];
    for (int i = threadIdx.x; i < W * (RT_Y + 2); i += RT_X * RT_Y) {
      const int xx = blockIdx.x * RT_X - 1 + i % W, yy = blockIdx.y * RT_Y - 1 + i / W;
      double v = 0.0;
      if (xx >= 0 && xx <= n && yy >= 0 && yy <= n && z >= 0 && z <= n)
        v = p.u[((long long)z * np1 + yy) * np1 + xx];
      pl[i] = v;
    }
    __syncthreads();
    const int ai = (ty + 1) * W + tx + 1;
    Xs[0] = Xs[1];
    Xs[1] = Xs[2];
    Xs[2] = pl[ai - 1] + pl[ai + 1] + pl[ai - W] + pl[ai + W];
    Ds[0] = Ds[1];
    Ds[1] = Ds[2];
    Ds[2] = pl[ai - W - 1] + pl[ai - W + 1] + pl[ai + W - 1] + pl[ai + W + 1];
    Cs[0] = Cs[1];
    Cs[1] = Cs[2];
    Cs[2] = pl[ai];
    __syncthreads();
    const int zz = z - 1;  // residual plane
    if (zz >= zlo && zz < zhi && x >= 1 && x <= n - 1 && y >= 1 && y <= n - 1) {
      const double Au = p.a_c * Cs[1] + p.a_f * (Xs[1] + Cs[0] + Cs[2]) +
                        p.a_e * (Ds[1] + Xs[0] + Xs[2]) + p.a_k * (Ds[0] + Ds[2]);
      const long long gi = ((long long)zz * np1 + y) * np1 + x;
      const double r = p.b[gi] - Au;
      p.rhs32[gi] = (float)r;
      acc += r * r;
    }
  }
  red[threadIdx.x] = acc * p.hD;
  __syncthreads();
  for (int w = RT_X * RT_Y / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    p.partials[b] = red[0];
  }
}

}  // namespace

void sweep3_grid(int nc, int bjx, int bjy, int zc, dim3* grid) {
  const int ncp1 = nc + 1;
  *grid = dim3((ncp1 + bjx - 1) / bjx, (ncp1 + bjy - 1) / bjy, (ncp1 + zc - 1) / zc);
}

void launch_sweep3(const Sweep3Params& p, int mode, cudaStream_t s) {
  dim3 grid;
  sweep3_grid(p.nc, kSweepBJX, kSweepBJY, p.zc, &grid);
  if (mode == SWEEP_FULL)
    k_sweep3<kSweepBJX, kSweepBJY, SWEEP_FULL><<<grid, NT, 0, s>>>(p);
  else if (mode == SWEEP_UP)
    k_sweep3<kSweepBJX, kSweepBJY, SWEEP_UP><<<grid, NT, 0, s>>>(p);
  else
    k_sweep3<kSweepBJX, kSweepBJY, SWEEP_DOWNU><<<grid, NT, 0, s>>>(p);
}

int refine3_blocks(int n, int zc) {
  const int gx = (n + 1 + RT_X - 1) / RT_X, gy = (n + 1 + RT_Y - 1) / RT_Y;
  const int gz = (n - 1 + zc - 1) / zc;
  return gx * gy * gz;
}

void launch_refine3(const Refine3Params& p, cudaStream_t s) {
  const int n = p.n;
  dim3 grid((n + 1 + RT_X - 1) / RT_X, (n + 1 + RT_Y - 1) / RT_Y, (n - 1 + p.zc - 1) / p.zc);
  k_refine3<<<grid, RT_X * RT_Y, 0, s>>>(p);
}

}  // namespace adafac
