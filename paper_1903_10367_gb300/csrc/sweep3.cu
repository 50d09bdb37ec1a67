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
// UP is the first up-pass of a refinement step (rho = rhs, restriction only);
// DOWNU is the last down-pass, which adds e to the FP64 iterate u.
//
// Blocking.  A block owns BJX x BJY coarse columns of level L-1 and zc coarse
// planes, i.e. the fine vertices whose nearest coarse vertex lies in that box
// (3 per coarse vertex and direction), and marches through its fine planes in
// z.  A ring of NSTAGE shared-memory slots is filled by the tensor memory
// accelerator PREF planes ahead of use: one slot holds a 68 x 30 box of e_{k-2}
// (owned box + 3, the x origin on a 16-byte boundary) and of rhs; the
// elected thread arms the slot's mbarrier with the byte count and issues both
// copies; out-of-domain parts are zero-filled.  Stage B forms e_{k-1} on the
// owned box + 2, stage C rho_k on the owned box + 1 (the restriction
// support); the restriction and the damping right-hand side of the block's
// coarse columns accumulate as planes pass.  Every thread keeps one column
// and a strip of rows for stages B and C; a 27-point stencil is split into an
// in-plane part W_p and an off-plane part Y_p per plane,
// A e(s) = W_s + Y_{s-1} + Y_{s+1}, both kept in registers as planes roll by.
#include "common.cuh"
#include "sweep3.cuh"

namespace adafac {

namespace {

constexpr int NT = 256;
constexpr int BJX = kSweepBJX, BJY = kSweepBJY;
constexpr int OW = 3 * BJX, OH = 3 * BJY;   // owned fine box (x, y)
constexpr int NCOL = 64;                    // thread columns
constexpr int NSTRIP = NT / NCOL;           // thread strips
constexpr int BOXW = kBoxW, BOXH = kBoxH;   // staged box of a plane
constexpr int PLANE_F = 2048;               // floats per staged plane (128-byte multiple)
constexpr int NSTAGE = 4, PREF = 2;         // ring slots, planes staged ahead
constexpr int QH = BJY + 4;                 // coarse rows of the q window (origin J0y - 2)
constexpr int NQX = QH * NCOL;              // x-interpolated coarse values per plane
constexpr int NJ = BJX * BJY;               // coarse columns of a block
constexpr int SB_F = 64 * 28, SR_F = 62 * 26 + 4;
constexpr long kWaitLimit = 1L << 24;       // polls before a wait gives up
static_assert(BOXW * BOXH <= PLANE_F, "staged box fits its slot");
static_assert(NJ <= NT && NQX % NT == 0, "thread counts");
static_assert((BOXW * 4) % 16 == 0, "box rows are 16-byte multiples");

// smem layout (floats): ring slots (e, rhs), sB, sR, sQX[2]; then mbarriers
constexpr int OFF_SB = NSTAGE * 2 * PLANE_F;
constexpr int OFF_SR = OFF_SB + SB_F;
constexpr int OFF_QX = OFF_SR + SR_F;
constexpr int OFF_BAR = OFF_QX + 2 * NQX;   // 8-byte aligned (even float index)
constexpr size_t SMEM_BYTES = (size_t)OFF_BAR * 4 + NSTAGE * 8 + 16;

template <int MODE>
struct Geo {
  // stage B (new e) and stage C (new residual) relative to the staged box
  static constexpr int BX0 = MODE == SWEEP_FULL ? 1 : 3;
  static constexpr int BW = MODE == SWEEP_FULL ? 64 : 60;
  static constexpr int BH = MODE == SWEEP_FULL ? 28 : 24;
  static constexpr int RB = BH / NSTRIP;
  static constexpr int CW = 62, CH = 26, RC = (CH + NSTRIP - 1) / NSTRIP;
  static_assert(RB * NSTRIP == BH, "stage B strips tile the region");
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on a phase of an mbarrier
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long i = 0; i < kWaitLimit; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* tm, int x, int y, int z,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(NT, 2)
    k_sweep3(const __grid_constant__ Sweep3Params p, const __grid_constant__ CUtensorMap tm_e,
             const __grid_constant__ CUtensorMap tm_rhs) {
  using G = Geo<MODE>;
  constexpr bool HAS_B = MODE != SWEEP_UP;
  constexpr bool FULL = MODE == SWEEP_FULL;
  constexpr int RB = G::RB, RC = G::RC;
  extern __shared__ __align__(1024) float smem[];
  __shared__ int s_fail;
  if (halted(p.ctl)) return;
  if (MODE != SWEEP_UP && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 &&
      threadIdx.x == 0 && p.applied)
    atomicAdd(p.applied, 1);  // one down-pass (a cycle's update) per launch

  float* sB = smem + OFF_SB;
  float* sR = smem + OFF_SR;
  float* sQX = smem + OFF_QX;
  const uint32_t bar0 = smem_addr(smem + OFF_BAR);

  const int n = p.n, nc = p.nc, ncp1 = nc + 1, ldx = p.ldx;
  const long long fplane = (long long)ldx * (n + 1);
  const int tid = threadIdx.x;
  const int col = tid % NCOL, strip = tid / NCOL;
  const int Jx0 = blockIdx.x * BJX, Jy0 = blockIdx.y * BJY;
  const int Jz0 = blockIdx.z * p.zc;
  const int Jz1 = min(Jz0 + p.zc, ncp1);
  const int xA = 3 * Jx0 - 4, yA = 3 * Jy0 - 4;            // staged box origin
  const int oz0 = 3 * Jz0 - 1, oz1 = 3 * Jz1 - 1;          // owned planes [oz0, oz1)
  const int zB0 = FULL ? oz0 - 2 : oz0, zB1 = FULL ? oz1 + 2 : oz1;
  const int zC0 = oz0 - 1, zC1 = oz1 + 1;
  int t0, t1;
  if (FULL) {
    t0 = zB0 - 1;
    t1 = zC1 + 2;
  } else if (MODE == SWEEP_DOWNU) {
    t0 = zB0 - 1;
    t1 = zB1 + 1;
  } else {
    t0 = zC0;
    t1 = zC1;
  }
  constexpr uint32_t kBytes = (HAS_B ? 2 : 1) * BOXW * BOXH * 4;
  // the copies of step t: e plane t and rhs plane t-1 (UP: rhs plane t)
  auto issue = [&](int t) {
    const int k = (t - t0) % NSTAGE;
    const uint32_t bar = bar0 + 8 * k;
    float* slot = smem + k * 2 * PLANE_F;
    mbar_expect(bar, kBytes);
    if (HAS_B) {
      tma_load(smem_addr(slot), &tm_e, xA, yA, t, bar);
      tma_load(smem_addr(slot + PLANE_F), &tm_rhs, xA, yA, t - 1, bar);
    } else {
      tma_load(smem_addr(slot + PLANE_F), &tm_rhs, xA, yA, t, bar);
    }
  };
  if (tid == 0) {
    s_fail = 0;
    for (int k = 0; k < NSTAGE; ++k) mbar_init(bar0 + 8 * k);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int t = t0; t < t0 + PREF && t < t1; ++t) issue(t);

  // ---- per-thread geometry, fixed for the whole z march -------------------
  // stage B: column col, rows strip RB + i of the stage-B region
  const int xb = xA + G::BX0 + col;
  const bool inxB = HAS_B && col < G::BW && xb >= 1 && xb <= n - 1;
  float mB[RB];
  int qkB[RB];
  float tyB[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int y = yA + G::BX0 + strip * RB + i;
    mB[i] = (inxB && y >= 1 && y <= n - 1) ? 1.f : 0.f;
    const int Oy = min(max(y, 0) / 3, nc - 1);
    qkB[i] = (Oy - (Jy0 - 2)) * NCOL + col;
    tyB[i] = (float)(y - 3 * Oy) * (1.f / 3.f);
  }
  // stage C (FULL): column col, rows strip RC + i of the stage-C region
  const int xc = xA + 2 + col;
  const bool inxC = FULL && col < G::CW && xc >= 1 && xc <= n - 1;
  const int ncrows = max(0, min(RC, G::CH - strip * RC));
  float mC[RC];
  unsigned ownC = 0;
#pragma unroll
  for (int i = 0; i < RC; ++i) {
    const int y = yA + 2 + strip * RC + i;
    mC[i] = (inxC && i < ncrows && y >= 1 && y <= n - 1) ? 1.f : 0.f;
    const int cy = strip * RC + i;
    if (col >= 1 && col <= OW && cy >= 1 && cy <= OH && mC[i] != 0.f) ownC |= 1u << i;
  }
  // x-interpolated coarse values: three (coarse row, B column) entries a thread
  int qoff[NQX / NT];
  float qtx[NQX / NT];
  bool qok[NQX / NT];
#pragma unroll
  for (int k = 0; k < NQX / NT; ++k) {
    const int e = tid + k * NT;
    const int ky = e / NCOL, c = e % NCOL;
    const int x = xA + G::BX0 + c, Jy = Jy0 - 2 + ky;
    const int Ox = min(max(x, 0) / 3, nc - 1);
    qok[k] = HAS_B && x >= 1 && x <= n - 1 && Jy >= 0 && Jy <= nc;
    qoff[k] = qok[k] ? Jy * ncp1 + Ox : 0;
    qtx[k] = (float)(x - 3 * Ox) * (1.f / 3.f);
  }
  float qa[NQX / NT][2], qb[NQX / NT][2];
  int qOz = -1;
  // z-interpolated, x-interpolated coarse row values of fine plane s -> sQX[buf]
  auto make_qx = [&](int s, int buf) {
    const int Oz = min(max(s, 0) / 3, nc - 1);
    if (Oz != qOz) {
      const float* q0 = p.q + (long long)Oz * ncp1 * ncp1;
      const float* q1 = q0 + ncp1 * ncp1;
#pragma unroll
      for (int k = 0; k < NQX / NT; ++k) {
        qa[k][0] = qok[k] ? q0[qoff[k]] : 0.f;
        qa[k][1] = qok[k] ? q0[qoff[k] + 1] : 0.f;
        qb[k][0] = qok[k] ? q1[qoff[k]] : 0.f;
        qb[k][1] = qok[k] ? q1[qoff[k] + 1] : 0.f;
      }
      qOz = Oz;
    }
    const float tz = (float)(s - 3 * Oz) * (1.f / 3.f);
#pragma unroll
    for (int k = 0; k < NQX / NT; ++k) {
      const float v0 = fmaf(tz, qb[k][0] - qa[k][0], qa[k][0]);
      const float v1 = fmaf(tz, qb[k][1] - qa[k][1], qa[k][1]);
      sQX[buf * NQX + tid + k * NT] = fmaf(qtx[k], v1 - v0, v0);
    }
  };
  if (HAS_B) make_qx(t0 - 1, (t0 - 1) & 1);

  // restriction: one thread per coarse column
  const bool resT = MODE != SWEEP_DOWNU && tid < NJ;
  const int cjx = tid % BJX, cjy = tid / BJX;
  const float a_c = p.a_c, a_f = p.a_f, a_e = p.a_e, a_k = p.a_k, w_invd = p.w_invd;
  // rolling per-plane parts of the stencils: centre value and W of plane t-1,
  // Y of planes t-1 and t-2
  float eB1[RB], WB1[RB], YB1[RB], YB2[RB];
  float eC1[RC], WC1[RC], YC1[RC], YC2[RC];
#pragma unroll
  for (int i = 0; i < RB; ++i) eB1[i] = WB1[i] = YB1[i] = YB2[i] = 0.f;
#pragma unroll
  for (int i = 0; i < RC; ++i) eC1[i] = WC1[i] = YC1[i] = YC2[i] = 0.f;
  float accR[2] = {0.f, 0.f}, accB[2] = {0.f, 0.f};

  for (int t = t0; t < t1; ++t) {
    __syncthreads();
    if (s_fail) break;
    if (tid == 0 && t + PREF < t1) issue(t + PREF);
    const int k = (t - t0) % NSTAGE;
    if (!mbar_wait(bar0 + 8 * k, ((t - t0) / NSTAGE) & 1)) {
      s_fail = 1;
      if (atomicCAS(p.fault, 0, 1) == 0) {  // first failure records where
        p.fault_info[0] = MODE;
        p.fault_info[1] = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        p.fault_info[2] = t - t0;
        p.fault_info[3] = k;
        p.fault_info[4] = ((t - t0) / NSTAGE) & 1;
        p.fault_info[5] = t;
        p.fault_info[6] = tid;
        p.fault_info[7] = t1 - t0;
      }
    }
    const float* sE = smem + k * 2 * PLANE_F;
    const float* sRhs = sE + PLANE_F;
    const int s = t - 1;                                    // stage B plane
    const int r = FULL ? t - 2 : t;                         // stage C plane
    // ---- stage B: new e at plane s ----------------------------------------
    if (HAS_B) {
      const bool doB = s >= zB0 && s < zB1;
      const float zm = (s >= 1 && s <= n - 1) ? 1.f : 0.f;
      const float* E = sE + (strip * RB + G::BX0 - 1) * BOXW + col + G::BX0 - 1;
      const float* Rh = sRhs + (strip * RB + G::BX0) * BOXW + col + G::BX0;
      const float* qx = sQX + (s & 1) * NQX;
      double uo[RB];
      if (MODE == SWEEP_DOWNU && doB && zm != 0.f) {
#pragma unroll
        for (int i = 0; i < RB; ++i)
          if (mB[i] != 0.f)
            uo[i] = p.u[((long long)s * (n + 1) + yA + G::BX0 + strip * RB + i) * (n + 1) + xb];
      }
      float hm = E[0] + E[2], mm = E[1];
      float hc = E[BOXW] + E[BOXW + 2], mc = E[BOXW + 1];
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const float* rb = E + (i + 2) * BOXW;
        const float hb = rb[0] + rb[2], mb = rb[1];
        const float X = hc + mm + mb;
        const float Dd = hm + hb;
        const float W = fmaf(a_c, mc, fmaf(a_f, X, a_e * Dd));
        const float Y = fmaf(a_f, mc, fmaf(a_e, X, a_k * Dd));
        if (doB && col < G::BW) {
          const float Ae = WB1[i] + YB2[i] + Y;
          const float rho = Rh[i * BOXW] - Ae;
          const float q0 = qx[qkB[i]], q1 = qx[qkB[i] + NCOL];
          const float pq = fmaf(tyB[i], q1 - q0, q0);
          const float ek = zm * mB[i] * (fmaf(w_invd, rho, eB1[i]) + pq);
          if (FULL) {
            sB[(strip * RB + i) * 64 + col] = ek;
          } else if (mB[i] != 0.f && zm != 0.f) {
            const long long row = (long long)s * (n + 1) + yA + G::BX0 + strip * RB + i;
            p.u[row * (n + 1) + xb] = uo[i] + (double)ek;
            p.e_out[s * fplane + (long long)(yA + G::BX0 + strip * RB + i) * ldx + xb] = 0.f;
          }
        }
        YB2[i] = YB1[i];
        YB1[i] = Y;
        WB1[i] = W;
        eB1[i] = mc;
        hm = hc;
        mm = mc;
        hc = hb;
        mc = mb;
      }
    }
    // ---- stage C: residual of the new e at plane r --------------------------
    if (FULL) {
      __syncthreads();
      if (col < G::CW && s >= zB0) {
        const bool doC = r >= zC0 && r < zC1;
        const float zm = (r >= 1 && r <= n - 1) ? 1.f : 0.f;
        // owned planes of the last chunk run past the domain: store interior only
        const bool ownZ = r >= oz0 && r < oz1 && r >= 1 && r <= n - 1;
        // rhs of plane r is in the previous slot
        const float* sRhsPrev = smem + ((t - 1 - t0 + NSTAGE) % NSTAGE) * 2 * PLANE_F + PLANE_F;
        const float* Rh = sRhsPrev + (strip * RC + 2) * BOXW + col + 2;
        const float* Bp = sB + (strip * RC) * 64 + col;
        float* eo = p.e_out + (long long)r * fplane + (long long)(yA + 2 + strip * RC) * ldx + xc;
        float hm = Bp[0] + Bp[2], mm = Bp[1];
        float hc = Bp[64] + Bp[66], mc = Bp[65];
#pragma unroll
        for (int i = 0; i < RC; ++i) {
          if (i >= ncrows) break;
          const float* rb = Bp + (i + 2) * 64;
          const float hb = rb[0] + rb[2], mb = rb[1];
          const float X = hc + mm + mb;
          const float Dd = hm + hb;
          const float W = fmaf(a_c, mc, fmaf(a_f, X, a_e * Dd));
          const float Y = fmaf(a_f, mc, fmaf(a_e, X, a_k * Dd));
          if (doC) {
            const float Ae = WC1[i] + YC2[i] + Y;
            const float rho = zm * mC[i] * (Rh[i * BOXW] - Ae);
            if (ownZ && ((ownC >> i) & 1u)) eo[(long long)i * ldx] = eC1[i];
            sR[(strip * RC + i) * 62 + col] = rho;
          }
          YC2[i] = YC1[i];
          YC1[i] = Y;
          WC1[i] = W;
          eC1[i] = mc;
          hm = hc;
          mm = mc;
          hc = hb;
          mc = mb;
        }
      }
      __syncthreads();
    }
    // ---- restriction and damping right-hand side of plane r -----------------
    if (resT && r >= zC0 && r < zC1) {
      // the 5x5 window of the coarse column, summed per class of distances
      // (|ox|, |oy|) from its centre: (0,0) (1,0) (2,0) (1,1) (1,2) (2,2)
      const float* w0;
      int pitch;
      if (FULL) {
        w0 = sR + (3 * cjy) * 62 + 3 * cjx;
        pitch = 62;
      } else {
        w0 = sRhs + (3 * cjy + 2) * BOXW + 3 * cjx + 2;
        pitch = BOXW;
      }
      float c0 = 0.f, l1 = 0.f, l2 = 0.f, p11 = 0.f, p12 = 0.f, p22 = 0.f;
#pragma unroll
      for (int oy = 0; oy < 5; ++oy) {
        const float* row = w0 + oy * pitch;
        const float v0 = row[0], v1 = row[1], v2 = row[2], v3 = row[3], v4 = row[4];
        if (oy == 2) {
          c0 = v2;
          l1 += v1 + v3;
          l2 += v0 + v4;
        } else if (oy == 1 || oy == 3) {
          l1 += v2;
          p11 += v1 + v3;
          p12 += v0 + v4;
        } else {
          l2 += v2;
          p12 += v1 + v3;
          p22 += v0 + v4;
        }
      }
      const float rin = c0 + (2.f / 3.f) * l1 + (1.f / 3.f) * l2 + (4.f / 9.f) * p11 +
                        (2.f / 9.f) * p12 + (1.f / 9.f) * p22;
      const int jtop = (r + 2) / 3;  // r >= -2
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const int Jz = jtop - 1 + d;
        const int oz = r - 3 * Jz;
        if (oz < -2 || oz > 2 || Jz < Jz0 || Jz >= Jz1) continue;
        const int az = oz < 0 ? -oz : oz;
        const int slot = Jz & 1;
        if (oz == -2) {
          accR[slot] = 0.f;
          accB[slot] = 0.f;
        }
        // d-linear restriction: weight (1 - |o|/3) per direction
        accR[slot] = fmaf(1.f - (float)az * (1.f / 3.f), rin, accR[slot]);
        const float* dz = p.dcls + 6 * az;
        accB[slot] += dz[0] * c0 + dz[1] * l1 + dz[2] * l2 + dz[3] * p11 + dz[4] * p12 +
                      dz[5] * p22;
        if (oz == 2) {
          const int Jx = Jx0 + cjx, Jy = Jy0 + cjy;
          if (Jx >= 1 && Jx <= nc - 1 && Jy >= 1 && Jy <= nc - 1 && Jz >= 1 && Jz <= nc - 1) {
            const float rc = accR[slot];
            const float bt = p.omega * accB[slot];
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
    // ---- coarse values for the next stage-B plane ---------------------------
    if (HAS_B && t + 1 < t1) make_qx(s + 1, (s + 1) & 1);
  }
  __syncthreads();
  if (s_fail && tid == 0) {
    atomicExch(p.fault, 1);
    // let the copies still in flight land before the block's memory is reused
    for (int k = 0; k < NSTAGE; ++k) {
      for (long i = 0; i < kWaitLimit / 64; ++i)
        if (mbar_try(bar0 + 8 * k, 0) || mbar_try(bar0 + 8 * k, 1)) break;
    }
  }
}

// FP64 residual of a uniform 3-D operator, z-marching with in-plane sums:
// rhs32 = (float)(b - A u) and per-block sums of h^3 r^2.
constexpr int RT_X = 32, RT_Y = 8;

__global__ void __launch_bounds__(RT_X* RT_Y) k_refine3(const Refine3Params p) {
  if (halted(p.ctl)) return;
  __shared__ double sU[(RT_X + 2) * (RT_Y + 2)];
  __shared__ double red[RT_X * RT_Y];
  const int n = p.n, np1 = n + 1;
  const int tx = threadIdx.x % RT_X, ty = threadIdx.x / RT_X;
  const int x = blockIdx.x * RT_X + tx, y = blockIdx.y * RT_Y + ty;
  const int zlo = blockIdx.z * p.zc + 1;
  const int zhi = min(zlo + p.zc, n);            // planes [zlo, zhi)
  constexpr int W = RT_X + 2;
  double Xs[3] = {0, 0, 0}, Ds[3] = {0, 0, 0}, Cs[3] = {0, 0, 0};
  double acc = 0.0;
  for (int z = zlo - 1; z <= zhi; ++z) {
    for (int i = threadIdx.x; i < W * (RT_Y + 2); i += RT_X * RT_Y) {
      const int xx = blockIdx.x * RT_X - 1 + i % W, yy = blockIdx.y * RT_Y - 1 + i / W;
      double v = 0.0;
      if (xx >= 0 && xx <= n && yy >= 0 && yy <= n && z >= 0 && z <= n)
        v = p.u[((long long)z * np1 + yy) * np1 + xx];
      sU[i] = v;
    }
    __syncthreads();
    const int ai = (ty + 1) * W + tx + 1;
    Xs[0] = Xs[1];
    Xs[1] = Xs[2];
    Xs[2] = sU[ai - 1] + sU[ai + 1] + sU[ai - W] + sU[ai + W];
    Ds[0] = Ds[1];
    Ds[1] = Ds[2];
    Ds[2] = sU[ai - W - 1] + sU[ai - W + 1] + sU[ai + W - 1] + sU[ai + W + 1];
    Cs[0] = Cs[1];
    Cs[1] = Cs[2];
    Cs[2] = sU[ai];
    __syncthreads();
    const int zz = z - 1;  // residual plane
    if (zz >= zlo && zz < zhi && x >= 1 && x <= n - 1 && y >= 1 && y <= n - 1) {
      const double Au = p.a_c * Cs[1] + p.a_f * (Xs[1] + Cs[0] + Cs[2]) +
                        p.a_e * (Ds[1] + Xs[0] + Xs[2]) + p.a_k * (Ds[0] + Ds[2]);
      const long long gi = ((long long)zz * np1 + y) * np1 + x;
      const double r = p.b[gi] - Au;
      p.rhs32[((long long)zz * np1 + y) * p.ldx + x] = (float)r;
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

size_t sweep3_smem_bytes() { return SMEM_BYTES; }

bool sweep3_make_maps(float* e0, float* e1, float* rhs, int n, int ldx, Sweep3Maps* maps) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  Encode encode = reinterpret_cast<Encode>(fn);
  const cuuint64_t np1 = (cuuint64_t)n + 1;
  const cuuint64_t dims[3] = {np1, np1, np1};
  const cuuint64_t strides[2] = {(cuuint64_t)ldx * 4, (cuuint64_t)ldx * np1 * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)kBoxH, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  float* bases[3] = {e0, e1, rhs};
  CUtensorMap* outs[3] = {&maps->e[0], &maps->e[1], &maps->rhs};
  for (int i = 0; i < 3; ++i) {
    if (encode(outs[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, bases[i], dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

void sweep3_grid(int nc, int zc, dim3* grid) {
  const int ncp1 = nc + 1;
  *grid = dim3((ncp1 + BJX - 1) / BJX, (ncp1 + BJY - 1) / BJY, (ncp1 + zc - 1) / zc);
}

bool sweep3_prepare() {
  return cudaFuncSetAttribute(k_sweep3<SWEEP_FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES) == cudaSuccess &&
         cudaFuncSetAttribute(k_sweep3<SWEEP_UP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES) == cudaSuccess &&
         cudaFuncSetAttribute(k_sweep3<SWEEP_DOWNU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES) == cudaSuccess;
}

template <int MODE>
static void launch_mode(const Sweep3Params& p, const Sweep3Maps& maps, int ein, cudaStream_t s) {
  dim3 grid;
  sweep3_grid(p.nc, p.zc, &grid);
  k_sweep3<MODE><<<grid, NT, SMEM_BYTES, s>>>(p, maps.e[ein], maps.rhs);
}

void launch_sweep3(const Sweep3Params& p, const Sweep3Maps& maps, int ein, int mode,
                   cudaStream_t s) {
  if (mode == SWEEP_FULL)
    launch_mode<SWEEP_FULL>(p, maps, ein, s);
  else if (mode == SWEEP_UP)
    launch_mode<SWEEP_UP>(p, maps, ein, s);
  else
    launch_mode<SWEEP_DOWNU>(p, maps, ein, s);
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
