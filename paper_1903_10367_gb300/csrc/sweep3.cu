// Fine-level sweeps for 3-D trees whose finest operator is uniform (scalar
// eps) and whose transfers are d-linear: the hot path of the mixed precision
// cycle.  Each FP32 cycle visits the finest level in two sweeps:
//
//   DOWN   down-pass of cycle j-1 (the fine-level part of the update of
//          Algorithm 1 / Eq. 9, with c_L = omega M^-1 rho):
//            e_{j-1} = e_{j-2} + omega M^-1 (rhs - A e_{j-2}) + P q_{j-1}
//          where q is the prolonged coarse part of the cycle;
//   UPE    up-pass of cycle j:  rho = rhs - A e_{j-1},
//            r_{L-1} = P^T rho,  b~_{L-1} = omega S~^T rho   (Eq. 8),
//            g_{L-1} = M^-1 (omega r_{L-1} - omega~ b~_{L-1});
//   UP     the first up-pass of a refinement step (e = 0, so rho = rhs);
//   DOWNU  the last down-pass, which adds e to the FP64 iterate u and clears
//          the other correction buffer for the next refinement step.
// The down-pass recomputes the residual it needs instead of reading a stored
// one: DOWN reads e and rhs and writes e (12 bytes per unknown), UPE reads e
// and rhs (8 bytes per unknown).
//
// Both sweeps march through the planes of their block in z.  A ring of
// NSTAGE shared-memory slots is filled by the tensor memory accelerator PREF
// planes ahead of use: a slot holds a box of e and of rhs around the block's
// columns (its x origin on a 16-byte boundary); one thread arms the slot's
// mbarrier with the byte count and issues the copies; parts outside the domain
// are zero-filled.  A thread owns a pair of adjacent columns and a strip of
// rows and works on the pair with packed FP32x2 arithmetic.  The 27-point
// stencil is split into an in-plane part W_p and an off-plane part Y_p per
// plane, A e(s) = W_s + Y_{s-1} + Y_{s+1}; the partial sum W_s + Y_{s-1} and
// Y_s roll along in registers.
//   * Down-passes own 64 fine columns (the 32 lane pairs of a warp) and 22
//     rows from row 1; they prolong q with the d-linear weights in three
//     interpolation stages (z per plane, x per plane into shared memory, y
//     per thread).
//   * Up-passes own 20 x 8 interior coarse columns (their restriction
//     targets; four x-tiles and ten y-tiles cover the 80 x 80 interior coarse
//     columns of a 243-cell grid exactly), form rho on the owned box + 1 (the
//     support of the restriction) in shared memory, and accumulate the
//     restriction and the damping right-hand side of their coarse columns as
//     the planes pass.
//   * Both split their planes into balanced slabs along z (grid z).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "mbarrier.cuh"
#include "sweep3.cuh"

namespace adafac {

namespace {

// down-pass tiles: 64 fine columns x OH rows; the coarse window of the
// prolongation is QW x QH coarse columns
constexpr int OH = kDownRows;               // owned fine rows per block: 22
constexpr int NPAIR = 32;                   // thread column pairs
constexpr int BOXW = kBoxW, BOXH = kBoxH;   // staged box of a plane: 68 x 24
constexpr int PLANE_F = 1632;               // floats per staged plane (128-byte multiple)
constexpr int NSTAGE = 3, PREF = 2;         // ring slots, planes staged ahead
// the rows y0 .. y0 + OH - 1 interpolate between the coarse rows floor(y0 / 3)
// .. floor((y0 + OH - 1) / 3) + 1: at most (OH + 1) / 3 + 2 of them
constexpr int QW = 24, QH = 10;             // coarse q window
constexpr int NQX = QH * 64;                // x-interpolated coarse values per plane
static_assert(QH >= (OH + 1) / 3 + 2, "the q window covers the rows' coarse rows");

static_assert(BOXW * BOXH <= PLANE_F && (PLANE_F * 4) % 128 == 0, "staged box fits its slot");
static_assert((BOXW * 4) % 16 == 0, "box rows are 16-byte multiples");
static_assert(BOXW >= 68 && BOXH >= OH + 2, "the box covers 64 columns and the rows + halo");

// the slot refilled at step t (that of t + PREF) was last read at step
// t + PREF - NSTAGE <= t - 1, before the block barrier that opens step t
static_assert(PREF < NSTAGE, "prefetch distance");

// down-pass smem layout (floats): ring slots (e, rhs), the coarse windows
// sQ[3], sQX[2], mbarriers.  The extra buffers let one block barrier per plane
// order all hand-overs between threads.
constexpr int OFF_Q = NSTAGE * 2 * PLANE_F;
constexpr int OFF_QX = OFF_Q + 3 * QW * QH + 2;  // (+2: 8-byte alignment)
constexpr int OFF_BAR = OFF_QX + 2 * NQX;
constexpr size_t SMEM_BYTES = (size_t)OFF_BAR * 4 + NSTAGE * 8 + 16;
static_assert(OFF_QX % 2 == 0 && OFF_BAR % 2 == 0, "8-byte alignment");

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* tm, int x, int y, int z,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// in-plane sums of a row at a column pair whose first column is odd: the
// aligned pairs a = (c-1, c), b = (c+1, c+2) give the centre pair (a.y, b.x)
// and the sum of the x-neighbours h = a + b
struct RowPair {
  float2 h, c;
};
__device__ __forceinline__ RowPair row_pair(const float* p) {
  const float2 a = ld2(p), b = ld2(p + 2);
  RowPair r;
  r.h = add2(a, b);
  r.c = make_float2(a.y, b.x);
  return r;
}

// in-plane part W and off-plane part Y of the stencil at a row pair, from the
// rows above (up), at (ce) and below (dn): with X the face neighbours in the
// plane and D the in-plane diagonal ones,
//   W = a_c e + a_e D,  Y = a_e (e + X) + a_k D   (a_f = 0 in 3-D)
struct Parts {
  float2 W, Y;
};
__device__ __forceinline__ Parts parts(const RowPair& up, const RowPair& ce, const RowPair& dn,
                                       float2 ac2, float2 ae2, float2 ak2) {
  const float2 X = add2(add2(ce.h, up.c), dn.c);
  const float2 D = add2(up.h, dn.h);
  Parts q;
  q.W = fma2(ac2, ce.c, mul2(ae2, D));
  q.Y = fma2(ae2, X, mul2(ak2, D));
  return q;
}

// ---- down-passes ----------------------------------------------------------------
// A block owns 64 fine columns in x from column 64 bx + 1 (all 32 lane pairs
// busy; no coarse alignment is needed), OH rows from row OH by + 1 and one of
// gridDim.z balanced slabs of the interior planes 1 .. n - 1 (no coarse
// alignment is needed in z either).  NT threads are 32 column pairs x NT/32
// row strips; MINB blocks per SM.
template <int MODE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_down3(const __grid_constant__ Sweep3Params p, const __grid_constant__ CUtensorMap tm_e,
            const __grid_constant__ CUtensorMap tm_rhs) {
  static_assert(MODE == SWEEP_DOWN || MODE == SWEEP_DOWNU, "down-pass modes");
  constexpr int NSTRIP = NT / NPAIR;
  constexpr int RBB = OH / NSTRIP, RBX = OH % NSTRIP;
  constexpr int RB = RBB + (RBX ? 1 : 0);                // rows of the longest strip
  static_assert(NQX % NT == 0, "thread tiling");
  extern __shared__ __align__(128) float smem[];
  __shared__ int s_fail;
  if (halted(p.ctl)) return;
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && p.applied)
    atomicAdd(p.applied, 1);  // one down-pass (a cycle's update) per launch

  float* sQ = smem + OFF_Q;
  float* sQX = smem + OFF_QX;
  const uint32_t bar0 = smem_addr(smem + OFF_BAR);

  const int n = p.n, nc = p.nc, ncp1 = nc + 1, ldx = p.ldx;
  const long long fplane = (long long)ldx * (n + 1);
  const int tid = threadIdx.x;
  const int pc = tid % NPAIR, strip = tid / NPAIR;
  const int Y0 = 1 + blockIdx.y * OH;                     // first owned row
  const int xs = 64 * (int)blockIdx.x + 1;                // first owned column
  const int xA = xs - 1, yA = Y0 - 1;                      // staged box origin
  const int oz0 = 1 + (int)((long long)blockIdx.z * (n - 1) / gridDim.z);  // owned planes
  const int oz1 = 1 + (int)((long long)(blockIdx.z + 1) * (n - 1) / gridDim.z);  // [oz0, oz1)
  // step t stages e plane t and rhs plane t-1 and updates plane s = t-1
  // (W + Y of planes s-1 .. s+1 are known at step t)
  const int t0 = oz0 - 1, t1 = oz1 + 1;
  constexpr uint32_t kBytes = 2 * BOXW * BOXH * 4;
  auto issue = [&](int t) {
    const int k = (t - t0) % NSTAGE;
    const uint32_t bar = bar0 + 8 * k;
    float* slot = smem + k * 2 * PLANE_F;
    mbar_expect(bar, kBytes);
    tma_load(smem_addr(slot), &tm_e, xA, yA, t, bar);
    tma_load(smem_addr(slot + PLANE_F), &tm_rhs, xA, yA, t - 1, bar);
  };
  if (tid == 0) {
    s_fail = 0;
    for (int k = 0; k < NSTAGE; ++k) mbar_init(bar0 + 8 * k);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int t = t0; t < t0 + PREF && t < t1; ++t) issue(t);

  // the pair (2 pc, 2 pc + 1) of the owned box is box columns 1 + 2 pc (+1);
  // the strip's owned rows rs0 + i (i < nr) are box rows rs0 + i + 1
  const int rs0 = strip * RBB + min(strip, RBX);
  const int nr = RBB + (strip < RBX ? 1 : 0);
  const int xb = xs + 2 * pc;                              // odd
  const float2 mxB = make_float2(xb >= 1 && xb <= n - 1 ? 1.f : 0.f,
                                 xb + 1 >= 1 && xb + 1 <= n - 1 ? 1.f : 0.f);
  const int y0 = Y0 + rs0;
  const int qy0 = min(Y0 / 3, nc - 1);                     // first coarse row of the window
  float myB[RB];
  int qrB[RB];
  float tyB[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int y = y0 + i;
    myB[i] = i < nr && y >= 1 && y <= n - 1 ? 1.f : 0.f;
    const int Oy = min(max(y, 0) / 3, nc - 1);
    qrB[i] = i < nr ? (Oy - qy0) * 64 + 2 * pc : 0;
    tyB[i] = (float)(y - 3 * Oy) * (1.f / 3.f);
  }
  // prolongation of q: per plane the z-interpolated coarse window sQ (QW x QH,
  // origin (qx0, qy0)), then the x-interpolated values sQX at the owned
  // columns; each thread interpolates in y itself.  The owned columns x in
  // [xs, xs + 64) interpolate between coarse columns floor(x / 3) and + 1.
  constexpr int NQ = (QW * QH + NT - 1) / NT, NX = NQX / NT;
  const int qx0 = xs / 3 - 1;
  int qoff[NQ];
  bool qok[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const int e = tid + k * NT;
    const int Jx = qx0 + e % QW, Jy = qy0 + e / QW;
    qok[k] = e < QW * QH && Jx >= 0 && Jx <= nc && Jy >= 0 && Jy <= nc;
    qoff[k] = qok[k] ? Jy * ncp1 + Jx : 0;
  }
  int xq[NX];
  float xt[NX];
#pragma unroll
  for (int k = 0; k < NX; ++k) {
    const int e = tid + k * NT;
    const int ky = e / 64, c = e % 64;
    const int x = xs + c;
    const int Ox = min(max(x, 0) / 3, nc - 1);
    xq[k] = ky * QW + Ox - qx0;
    xt[k] = (float)(x - 3 * Ox) * (1.f / 3.f);
  }
  float qa[NQ], qb[NQ];
  int qOz = -1;
  auto make_q = [&](int s, int buf) {  // sQ of plane s, from cached coarse values
    const int Oz = min(max(s, 0) / 3, nc - 1);
    if (Oz != qOz) {
      const float* q0 = p.q + (long long)Oz * ncp1 * ncp1;
      const float* q1 = q0 + ncp1 * ncp1;
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        qa[k] = qok[k] ? q0[qoff[k]] : 0.f;
        qb[k] = qok[k] ? q1[qoff[k]] : 0.f;
      }
      qOz = Oz;
    }
    const float tz = (float)(s - 3 * Oz) * (1.f / 3.f);
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const int e = tid + k * NT;
      if (e < QW * QH) sQ[buf * QW * QH + e] = fmaf(tz, qb[k] - qa[k], qa[k]);
    }
  };
  auto make_qx = [&](int qbuf, int buf) {  // sQX of a plane from its sQ
    const float* q = sQ + qbuf * QW * QH;
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      const float v0 = q[xq[k]], v1 = q[xq[k] + 1];
      sQX[buf * NQX + tid + k * NT] = fmaf(xt[k], v1 - v0, v0);
    }
  };
  // step t (plane s = t - 1) reads sQX[s & 1], forms sQX of plane s + 1 from
  // sQ[mod3(s + 1)] and sQ of plane s + 2: one block barrier per plane orders
  // every hand-over
  auto mod3 = [](int v) { return ((v % 3) + 3) % 3; };
  make_q(t0 - 1, mod3(t0 - 1));
  make_q(t0, mod3(t0));
  __syncthreads();
  make_qx(mod3(t0 - 1), (t0 - 1) & 1);

  // the block's columns and rows reach the boundary (or beyond): only then
  // are its stores masked
  const bool edge = xs + 63 > n - 1 || Y0 + OH - 1 > n - 1;
  const float2 ac2 = f2(p.a_c), ae2 = f2(p.a_e), ak2 = f2(p.a_k), w2 = f2(p.w_invd);
  const float2 neg1 = f2(-1.f);
  // rolling stencil parts per row: centre of the last plane, PR = W_s + Y_{s-1}
  // of the last plane s, YR = Y_s
  float2 eR[RB], PR[RB], YR[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) eR[i] = PR[i] = YR[i] = f2(0.f);
  // DOWNU: the largest biased exponent of the u this thread writes (the
  // scale of the next refinement step's fixed-point residual)
  unsigned uexp_max = 0;
  // DOWNU: the FP64 iterate at the thread's columns of an owned plane
  double un[RB][2];
  auto fetch_u = [&](int sp) {
    const bool own = sp >= oz0 && sp < oz1 && sp >= 1 && sp <= n - 1;
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const long long urow = ((long long)sp * (n + 1) + y0 + i) * (n + 1);
      un[i][0] = (own && myB[i] != 0.f && mxB.x != 0.f) ? p.u[urow + xb] : 0.0;
      un[i][1] = (own && myB[i] != 0.f && mxB.y != 0.f) ? p.u[urow + xb + 1] : 0.0;
    }
  };
  if (MODE == SWEEP_DOWNU) fetch_u(t0 - 1);
  auto expo = [](double v) {
    return (unsigned)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
  };

  for (int t = t0; t < t1; ++t) {
    __syncthreads();
    if (s_fail) break;
    if (tid == 0 && t + PREF < t1) issue(t + PREF);
    const int k = (t - t0) % NSTAGE;
    if (!mbar_wait(bar0 + 8 * k, ((t - t0) / NSTAGE) & 1, p.wait_polls)) {
      // the slot's data may not have landed: nothing of this step is stored,
      // and the block leaves at the next barrier
      s_fail = t - t0 + 1;
      if (atomicCAS(p.fault, 0, 1) == 0) {  // the first failure records where
        p.fault_info[0] = MODE;
        p.fault_info[1] = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        p.fault_info[2] = t - t0;
        p.fault_info[3] = k;
        p.fault_info[4] = ((t - t0) / NSTAGE) & 1;
        p.fault_info[5] = t;
        p.fault_info[6] = tid;
        p.fault_info[7] = t1 - t0;
      }
      continue;
    }
    const float* sE = smem + k * 2 * PLANE_F;
    const float* sRhs = sE + PLANE_F;
    const int s = t - 1;
    const bool doB = s >= oz0 && s < oz1 && s >= 1 && s <= n - 1;
    const float* E = sE + rs0 * BOXW + 2 * pc;
    const float* Rh = sRhs + (rs0 + 1) * BOXW + 1 + 2 * pc;
    const float* qx = sQX + (s & 1) * NQX;
    // DOWNU: the FP64 iterate of plane s came in during the previous step;
    // the loads of plane s + 1 go out now (their latency overlaps this step)
    double uo[RB][2];
    if (MODE == SWEEP_DOWNU) {
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        uo[i][0] = un[i][0];
        uo[i][1] = un[i][1];
      }
      fetch_u(s + 1);
    }
    // the same rows with and without the boundary masks: the down-pass
    // blocks whose columns and rows are all interior store unconditionally
    auto rows = [&](auto masked) {
      constexpr bool M = decltype(masked)::value;
      RowPair up = row_pair(E), ce = row_pair(E + BOXW);
  #pragma unroll
      for (int i = 0; i < RB; ++i) {
        if (i >= nr) break;
        const RowPair dn = row_pair(E + (i + 2) * BOXW);
        const Parts q = parts(up, ce, dn, ac2, ae2, ak2);
        if (doB && (!M || myB[i] != 0.f)) {
          const float2 Ae = add2(PR[i], q.Y);
          const float2 rhs = make_float2(Rh[i * BOXW], Rh[i * BOXW + 1]);
          const float2 rho = fma2(Ae, neg1, rhs);
          const float2 q0 = ld2(qx + qrB[i]), q1 = ld2(qx + qrB[i] + 64);
          const float2 pq = fma2(f2(tyB[i]), fma2(q0, neg1, q1), q0);
          const float2 ek = add2(fma2(w2, rho, eR[i]), pq);
          float* eo = p.e_out + s * fplane + (long long)(y0 + i) * ldx + xb;
          if (MODE == SWEEP_DOWN) {
            if (!M || mxB.x != 0.f) eo[0] = ek.x;
            if (!M || mxB.y != 0.f) eo[1] = ek.y;
          } else {
            const long long urow = ((long long)s * (n + 1) + y0 + i) * (n + 1);
            if (mxB.x != 0.f) {
              const double un = uo[i][0] + (double)ek.x;
              p.u[urow + xb] = un;
              uexp_max = max(uexp_max, expo(un));
              eo[0] = 0.f;  // the zero buffer of the next refinement step
            }
            if (mxB.y != 0.f) {
              const double un = uo[i][1] + (double)ek.y;
              p.u[urow + xb + 1] = un;
              uexp_max = max(uexp_max, expo(un));
              eo[1] = 0.f;
            }
          }
        }
        PR[i] = add2(q.W, YR[i]);
        YR[i] = q.Y;
        eR[i] = ce.c;
        up = ce;
        ce = dn;
      }
    };
    if (MODE == SWEEP_DOWN && !edge) rows(std::false_type());
    else rows(std::true_type());
    if (t + 1 < t1) {
      make_qx(mod3(s + 1), (s + 1) & 1);
      if (t + 2 < t1) make_q(s + 2, mod3(s + 2));
    }
  }
  if (MODE == SWEEP_DOWNU && p.uexp) {
    uexp_max = __reduce_max_sync(0xffffffffu, uexp_max);
    if ((tid & 31) == 0 && uexp_max > 0) atomicMax(p.uexp, (int)uexp_max);
  }
  __syncthreads();
  if (s_fail && tid == 0) {
    atomicExch(p.fault, 1);
    // let the copies still in flight (steps tf .. tf + PREF) land before the
    // block's shared memory is released
    const int tf = t0 + s_fail - 1;
    for (int tt = tf; tt <= tf + PREF && tt < t1; ++tt) {
      const uint32_t bar = bar0 + 8 * ((tt - t0) % NSTAGE);
      const uint32_t par = ((tt - t0) / NSTAGE) & 1;
      for (long i = 0; i < kWaitLimit / 16 && !mbar_try(bar, par); ++i) {
      }
    }
  }
}

// ---- up-passes on wide tiles -------------------------------------------------
// A block owns UBJX x UBJY interior coarse columns (20 x 8, from column and row
// 1: four x-tiles and ten y-tiles cover the 80 x 80 interior coarse columns of
// a 243-cell grid exactly, and the 160 restriction targets are five full
// warps) and one of gridDim.z balanced slabs of the interior coarse planes
// 1 .. nc - 1.  Its 256 threads are 32 column pairs (one warp per row) x 8 row
// strips.  The residual region is the owned fine box + 1 (62 x 26 fine
// columns), computed by the first UNACT pairs, whose first column is odd,
// starting at cstart = 3 J0x - 2 (J0x odd) or 3 J0x - 3 (J0x even); the staged
// box starts at the 16-byte boundary at or below cstart - 1 and is 64 x 28
// floats.  Strips 0 and 1 take 4 residual rows, the others 3; warps 2 .. 6
// also restrict.
constexpr int UBJX = kUpBJX, UBJY = kUpBJY;
constexpr int UNT = 256, UNPAIR = 32, UNSTRIP = UNT / UNPAIR;
constexpr int kUpMinB = 3;                              // blocks per SM
constexpr int UNACT = (3 * UBJX + 3) / 2;               // pairs of the residual region (31)
constexpr int UBOXW = kUpBoxW, UBOXH = kUpBoxH;
constexpr int UPLANE_F = UBOXW * UBOXH;                 // 1792 floats: 128-byte multiple
constexpr int UCH = 3 * UBJY + 2;                       // residual rows (26)
constexpr int URCB = UCH / UNSTRIP, URCX = UCH % UNSTRIP;
constexpr int URC = URCB + (URCX ? 1 : 0);
// residual-plane pitch: 84 = 20 mod 32 keeps the restriction's loads free of
// bank conflicts (a warp's targets span up to three coarse rows)
constexpr int USR_P = 84;
constexpr int USR_F = USR_P * UCH;
constexpr int UNJ = UBJX * UBJY;                        // 160 coarse columns
constexpr int UJ0 = URCX * UNPAIR;                      // first restricting thread
constexpr int UOFF_SR = NSTAGE * 2 * UPLANE_F;
constexpr int UOFF_BAR = UOFF_SR + 2 * USR_F;
constexpr size_t USMEM_BYTES = (size_t)UOFF_BAR * 4 + NSTAGE * 8 + 16;
static_assert((UPLANE_F * 4) % 128 == 0 && UOFF_SR % 2 == 0 && UOFF_BAR % 2 == 0, "alignment");
static_assert(UJ0 + UNJ <= UNT && UNACT <= UNPAIR && 2 * UNACT >= 3 * UBJX + 2, "thread counts");
static_assert(2 * UNACT <= USR_P && UBOXW >= 2 * UNACT + 2, "the residual region fits its planes");

template <int MODE>
__global__ void __launch_bounds__(UNT, kUpMinB)
    k_up3(const __grid_constant__ Sweep3Params p, const __grid_constant__ CUtensorMap tm_e,
          const __grid_constant__ CUtensorMap tm_rhs) {
  static_assert(MODE == SWEEP_UP || MODE == SWEEP_UPE, "up-pass modes");
  extern __shared__ __align__(128) float smem[];
  __shared__ int s_fail;
  if (halted(p.ctl)) return;
  // the step's refinement residual has read the exponent of u: start the
  // maximum over the u the step's last down-pass writes (boundary values
  // stay; they enter through bdexp)
  if (MODE == SWEEP_UP && p.uexp && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 &&
      threadIdx.x == 0)
    *p.uexp = *p.bdexp;
  float* sR = smem + UOFF_SR;
  const uint32_t bar0 = smem_addr(smem + UOFF_BAR);
  const int n = p.n, nc = p.nc, ncp1 = nc + 1;
  const int tid = threadIdx.x;
  const int pc = tid % UNPAIR, strip = tid / UNPAIR;
  const int Jx0 = 1 + blockIdx.x * UBJX, Jy0 = 1 + blockIdx.y * UBJY;
  const int Jz0 = 1 + (int)((long long)blockIdx.z * (nc - 1) / gridDim.z);  // coarse planes
  const int Jz1 = 1 + (int)((long long)(blockIdx.z + 1) * (nc - 1) / gridDim.z);  // [Jz0, Jz1)
  const int soff = (Jx0 & 1) ? 0 : 1;                   // restriction column offset in sR
  const int cstart = 3 * Jx0 - 2 - soff;                // odd
  const int xA = ((cstart - 1) >> 2) << 2;              // floor to a multiple of 4
  const int yA = 3 * Jy0 - 3;                           // box row i + 1 = residual row i
  const int zC0 = 3 * Jz0 - 2, zC1 = 3 * Jz1;          // residual planes [zC0, zC1)
  constexpr bool UPE = MODE == SWEEP_UPE;
  const int t0 = UPE ? zC0 - 1 : zC0, t1 = UPE ? zC1 + 1 : zC1;
  constexpr uint32_t kBytes = (UPE ? 2 : 1) * UBOXW * UBOXH * 4;
  auto issue = [&](int t) {
    const int k = (t - t0) % NSTAGE;
    const uint32_t bar = bar0 + 8 * k;
    float* slot = smem + k * 2 * UPLANE_F;
    mbar_expect(bar, kBytes);
    if (UPE) {
      tma_load(smem_addr(slot), &tm_e, xA, yA, t, bar);
      tma_load(smem_addr(slot + UPLANE_F), &tm_rhs, xA, yA, t - 1, bar);
    } else {
      tma_load(smem_addr(slot + UPLANE_F), &tm_rhs, xA, yA, t, bar);
    }
  };
  if (tid == 0) {
    s_fail = 0;
    for (int k = 0; k < NSTAGE; ++k) mbar_init(bar0 + 8 * k);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int t = t0; t < t0 + PREF && t < t1; ++t) issue(t);

  // residual geometry: pair pc = columns c, c + 1 (c = cstart + 2 pc, odd);
  // the last pair has no columns
  const bool active = pc < UNACT;
  const int c = cstart + 2 * pc;
  const float2 mxC = make_float2(active && c >= 1 && c <= n - 1 ? 1.f : 0.f,
                                 active && c + 1 >= 1 && c + 1 <= n - 1 ? 1.f : 0.f);
  const int rc0 = strip * URCB + min(strip, URCX);
  const int ncrows = URCB + (strip < URCX ? 1 : 0);
  float myC[URC];
#pragma unroll
  for (int i = 0; i < URC; ++i) {
    const int y = 3 * Jy0 - 2 + rc0 + i;
    myC[i] = (i < ncrows && y >= 1 && y <= n - 1) ? 1.f : 0.f;
  }
  // the residual region reaches the boundary (rows or columns 0 or n and
  // beyond) only in blocks at the end of a grid whose interior the tiles do
  // not divide: only there does the residual need its masks
  const bool edge = 3 * Jy0 - 2 < 1 || 3 * Jy0 - 2 + UCH - 1 > n - 1 || cstart < 1 ||
                    cstart + 2 * UNACT - 1 > n - 1;
  const float2 ac2 = f2(p.a_c), ae2 = f2(p.a_e), ak2 = f2(p.a_k);
  const float2 neg1 = f2(-1.f);
  float2 PR[URC], YR[URC];
#pragma unroll
  for (int i = 0; i < URC; ++i) PR[i] = YR[i] = f2(0.f);
  // restriction and damping sums of the coarse plane being completed (cur)
  // and of the next one (nxt); the class weights of S~ by |oz| in registers
  float curR = 0.f, curB = 0.f, nxtR = 0.f, nxtB = 0.f;
  float dz0[6], dz1[6], dz2[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    dz0[k] = p.dcls[k];
    dz1[k] = p.dcls[6 + k];
    dz2[k] = p.dcls[12 + k];
  }
  // restriction geometry: coarse column tid - UJ0 (the strips with fewer rows)
  const int jt = tid - UJ0;
  const bool hasJ = jt >= 0 && jt < UNJ;
  const int cjx = hasJ ? jt % UBJX : 0, cjy = hasJ ? jt / UBJX : 0;
  const int Jx = Jx0 + cjx, Jy = Jy0 + cjy;
  const bool outJ = hasJ && Jx >= 1 && Jx <= nc - 1 && Jy >= 1 && Jy <= nc - 1;

  const int tEnd = UPE ? t1 + 1 : t1;
  for (int t = t0; t < tEnd; ++t) {
    __syncthreads();
    if (s_fail) break;
    if (tid == 0 && t + PREF < t1) issue(t + PREF);
    const int k = (t - t0) % NSTAGE;
    if (t < t1 && !mbar_wait(bar0 + 8 * k, ((t - t0) / NSTAGE) & 1, p.wait_polls)) {
      // as in the down-pass: no store of this step, leave at the next barrier
      s_fail = t - t0 + 1;
      if (atomicCAS(p.fault, 0, 1) == 0) {
        p.fault_info[0] = 10 + MODE;
        p.fault_info[1] = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        p.fault_info[2] = t - t0;
        p.fault_info[3] = k;
        p.fault_info[4] = ((t - t0) / NSTAGE) & 1;
        p.fault_info[5] = t;
        p.fault_info[6] = tid;
        p.fault_info[7] = t1 - t0;
      }
      continue;
    }
    const float* sE = smem + k * 2 * UPLANE_F;
    const float* sRhs = sE + UPLANE_F;
    const int r = UPE ? t - 2 : t;                      // plane restricted in this step
    const float* wbase;
    int pitch;
    if (UPE) {
      // residual of plane t - 1 into sR[(t - 1) & 1]
      const int rn = t - 1;
      if (t < t1 && active) {
        const bool store = rn >= zC0 && rn < zC1;
        const float zm = (rn >= 1 && rn <= n - 1) ? 1.f : 0.f;
        const float* E = sE + rc0 * UBOXW + (c - 1 - xA);
        const float* Rh = sRhs + (rc0 + 1) * UBOXW + (c - xA);
        float* sRn = sR + (rn & 1) * USR_F;
        // the same rows with and without the boundary masks (multiplying by
        // 1 changes nothing, so both give the same values)
        auto rows = [&](auto masked) {
          RowPair up = row_pair(E), ce = row_pair(E + UBOXW);
#pragma unroll
          for (int i = 0; i < URC; ++i) {
            if (i >= ncrows) break;
            const RowPair dn = row_pair(E + (i + 2) * UBOXW);
            const Parts q = parts(up, ce, dn, ac2, ae2, ak2);
            if (store) {
              const float2 Ae = add2(PR[i], q.Y);
              const float2 rhs = make_float2(Rh[i * UBOXW], Rh[i * UBOXW + 1]);
              float2 rho = fma2(Ae, neg1, rhs);
              if constexpr (decltype(masked)::value) rho = mul2(rho, mul2(mxC, f2(zm * myC[i])));
              st2(sRn + (rc0 + i) * USR_P + 2 * pc, rho);
            }
            PR[i] = add2(q.W, YR[i]);
            YR[i] = q.Y;
            up = ce;
            ce = dn;
          }
        };
        if (edge) rows(std::true_type());
        else rows(std::false_type());
      }
      // sR column j = absolute column cstart + j, row j = residual row j
      wbase = sR + (r & 1) * USR_F + soff;
      pitch = USR_P;
    } else {
      // UP: rho = rhs (zero outside the interior), read from the staged box
      wbase = sRhs + UBOXW + (3 * Jx0 - 2 - xA);
      pitch = UBOXW;
    }
    // ---- restriction and damping right-hand side of plane r -----------------
    if (hasJ && r >= zC0 && r < zC1) {
      const float* w0 = wbase + (3 * cjy) * pitch + 3 * cjx;
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
      // fine plane r = 3 m + ph lies at oz = ph from coarse plane m and at
      // oz = ph - 3 from m + 1: ph 0 adds to m only; ph 1 adds oz = 1 to m and
      // opens m + 1 with oz = -2; ph 2 completes m (oz = 2) and adds oz = -1 to
      // m + 1.  The phase is the same for the whole block, so the branches do
      // not diverge and the weights of |oz| are compile-time indices.
      const int ph = (r + 3) % 3;  // r >= -2
      const int m = (r + 3) / 3 - 1;
      if (ph == 0) {
        curR += rin;
        curB += dz0[0] * c0 + dz0[1] * l1 + dz0[2] * l2 + dz0[3] * p11 + dz0[4] * p12 +
                dz0[5] * p22;
      } else {
        const float b1 = dz1[0] * c0 + dz1[1] * l1 + dz1[2] * l2 + dz1[3] * p11 +
                         dz1[4] * p12 + dz1[5] * p22;
        const float b2 = dz2[0] * c0 + dz2[1] * l1 + dz2[2] * l2 + dz2[3] * p11 +
                         dz2[4] * p12 + dz2[5] * p22;
        if (ph == 1) {
          curR = fmaf(2.f / 3.f, rin, curR);
          curB += b1;
          nxtR = (1.f / 3.f) * rin;
          nxtB = b2;
        } else {
          const float aR = fmaf(1.f / 3.f, rin, curR);
          const float aB = curB + b2;
          if (outJ && m >= Jz0 && m >= 1 && m <= nc - 1) {
            const float bt = p.omega * aB;
            const long long ci = ((long long)m * ncp1 + Jy) * ncp1 + Jx;
            p.r_c[ci] = aR;
            if (p.variant == V_JAC) {
              p.bt_c[ci] = bt;
              p.g_c[ci] = p.c_invd * (p.omega * aR - p.omega_t * bt);
            } else {
              p.bt_c[ci] = 0.f;
              p.g_c[ci] = p.gscale * p.omega * p.c_invd * aR;
            }
          }
          curR = fmaf(2.f / 3.f, rin, nxtR);
          curB = nxtB + b1;
        }
      }
    }
  }
  __syncthreads();
  if (s_fail && tid == 0) {
    atomicExch(p.fault, 1);
    const int tf = t0 + s_fail - 1;
    for (int tt = tf; tt <= tf + PREF && tt < t1; ++tt) {
      const uint32_t bar = bar0 + 8 * ((tt - t0) % NSTAGE);
      const uint32_t par = ((tt - t0) / NSTAGE) & 1;
      for (long i = 0; i < kWaitLimit / 16 && !mbar_try(bar, par); ++i) {
      }
    }
  }
}

// Refinement residual of the uniform 3-D operator, z-marching with in-plane
// sums: rhs32 = (float)(b - A u) and per-block sums of h^3 r^2.
//
// The d-linear stencil in 3-D is alpha [32, 0, -2, -1] (centre, faces, edges,
// corners; alpha = eps h / 12), so A u = alpha S u with integer weights.  u and
// b / alpha are taken to 64-bit fixed point with a common scale 2^F that keeps
// every value below 2^56, and S u and b / alpha - S u are summed exactly in
// integers: the only rounding is the conversion of each value (below 2^-F,
// i.e. 2^-55 of the largest magnitude) and of the result to FP32.  This is at
// least as accurate as FP64 arithmetic and runs on the integer units; the
// GPU's FP64 rate (about 1/64 of FP32) would otherwise bound the kernel.
// b / alpha is stored in fixed point at setup (scale 2^(1078 - bexp)) and only
// shifted to the step's scale here.
//
// A block owns 32 columns x 16 rows and zc planes; a warp owns a strip of 4
// rows, a lane one column.  Per plane the block converts the plane's 34 x 18
// box of u (the tile and its ring) to fixed point into one of two shared
// buffers; one barrier per plane orders the hand-over.  The values of plane
// z + 1 and b of plane z are loaded into registers while plane z is worked on,
// so the global loads of one plane overlap the arithmetic of the previous.
// Per plane p, W_p = 32 u - 2 D_p and Y_p = -(2 X_p + D_p), with X_p / D_p
// the sums of the 4 in-plane face / diagonal neighbours; (S u)_s = W_s +
// Y_{s-1} + Y_{s+1}.  In a row, with h = u(x-1) + u(x+1) and m = u(x):
// X = h + m(y-1) + m(y+1) and D = h(y-1) + h(y+1).
constexpr int RT_X = 32, RT_Y = 16, RT_RB = 4;
constexpr int RT_NT = RT_X * (RT_Y / RT_RB);                  // 128 threads
constexpr int RT_W = RT_X + 2, RT_H = RT_Y + 2;               // staged box 34 x 18
constexpr int RT_NH = (RT_W * RT_H + RT_NT - 1) / RT_NT;      // box values per thread
constexpr int RT_MINB = 6;                                    // resident blocks per SM
static_assert(RT_Y % RT_RB == 0 && RT_NT % 32 == 0, "refinement tiling");

// x 2^F as an integer, F = 1078 - emax (emax >= the biased exponent of x);
// values below 2^-1022 count as zero.  (m << 3) >> (emax - e) is m 2^(e - emax
// + 3): exact when e >= emax - 3, truncated towards zero below.
__device__ __forceinline__ long long to_fixed(double x, int emax) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  const long long m = ((bits & 0xfffffffffffffLL) | 0x10000000000000LL) << 3;  // < 2^56
  const int k = emax - e;
  const long long v = (e != 0 && k >= 0 && k < 64) ? (m >> k) : 0;
  return bits < 0 ? -v : v;
}

// |R| < 2^63 as a float, without cancellation
__device__ __forceinline__ float fixed_to_float(long long R) {
  const unsigned long long a = (unsigned long long)(R < 0 ? -R : R);
  const float f = fmaf(__uint2float_rn((unsigned)(a >> 32)), 4294967296.f,
                       __uint2float_rn((unsigned)(a & 0xffffffffu)));
  return R < 0 ? -f : f;
}

__global__ void __launch_bounds__(RT_NT, RT_MINB) k_refine3(const Refine3Params p) {
  if (halted(p.ctl)) return;
  __shared__ long long sU[2][RT_W * RT_H];
  __shared__ double red[RT_NT / 32];
  const int bexp = max(p.ctl->bexp, 1);
  const int emax = max(p.ctl->uexp, bexp);
  const int F = 1078 - emax;
  const int bsh = min(emax - bexp, 63);                // b / alpha: scale 2^(1078 - bexp)
  // rhs = alpha R 2^-F = (R malpha) 2^ks; one multiplication when 2^ks is a
  // normal float (the same rounded value as ldexpf)
  const int ks = p.ealpha - F;
  const bool one_mul = ks >= -126 && ks <= 127;
  const float sc = one_mul ? ldexpf(p.malpha, ks) : 0.f;
  const int n = p.n, np1 = n + 1;
  const long long plane = (long long)np1 * np1;
  const int tx = threadIdx.x & 31, strip = threadIdx.x >> 5;
  const int x = blockIdx.x * RT_X + tx;
  const int y0 = blockIdx.y * RT_Y + strip * RT_RB;
  const int zlo = blockIdx.z * p.zc + 1;
  const int zhi = min(zlo + p.zc, n);                  // residual planes [zlo, zhi)
  const bool xin = x >= 1 && x <= n - 1;
  // the box values this thread converts: box index i = tid + k NT, at plane
  // offset hoff (-1: outside the box or the grid)
  int hoff[RT_NH];
#pragma unroll
  for (int k = 0; k < RT_NH; ++k) {
    const int i = threadIdx.x + k * RT_NT;
    const int xx = blockIdx.x * RT_X - 1 + i % RT_W, yy = blockIdx.y * RT_Y - 1 + i / RT_W;
    const bool ok = i < RT_W * RT_H && xx >= 0 && xx <= n && yy >= 0 && yy <= n;
    hoff[k] = ok ? yy * np1 + xx : -1;
  }
  bool yin[RT_RB];
#pragma unroll
  for (int i = 0; i < RT_RB; ++i) yin[i] = xin && y0 + i >= 1 && y0 + i <= n - 1;
  double un[RT_NH];
  long long bn[RT_RB];
  auto fetch_u = [&](int z) {  // z in [0, n]
    const double* up = p.u + (long long)z * plane;
#pragma unroll
    for (int k = 0; k < RT_NH; ++k) un[k] = hoff[k] >= 0 ? up[hoff[k]] : 0.0;
  };
  auto fetch_b = [&](int z) {
    const bool zin = z >= zlo && z < zhi;
    const long long* bp = p.bq + (long long)z * plane + (long long)y0 * np1 + x;
#pragma unroll
    for (int i = 0; i < RT_RB; ++i) bn[i] = zin && yin[i] ? bp[(long long)i * np1] : 0;
  };
  fetch_u(zlo - 1);
#pragma unroll
  for (int i = 0; i < RT_RB; ++i) bn[i] = 0;
  long long P[RT_RB], Ym[RT_RB];  // W_{z-1} + Y_{z-2} and Y_{z-1} per row
#pragma unroll
  for (int i = 0; i < RT_RB; ++i) P[i] = Ym[i] = 0;
  float acc = 0.f;                // sum of (R 2^-32)^2
  int buf = 0;
  for (int z = zlo - 1; z <= zhi; ++z, buf ^= 1) {
    // plane z (loaded during the previous plane) into the shared buffer, then
    // the loads of plane z + 1 and of b of plane z go out
    long long* S = sU[buf];
#pragma unroll
    for (int k = 0; k < RT_NH; ++k) {
      const int i = threadIdx.x + k * RT_NT;
      if (i < RT_W * RT_H) S[i] = to_fixed(un[k], emax);
    }
    if (z + 1 <= zhi) fetch_u(z + 1);
    long long bc[RT_RB];          // b of plane z - 1
#pragma unroll
    for (int i = 0; i < RT_RB; ++i) bc[i] = bn[i];
    fetch_b(z);
    __syncthreads();
    const int zr = z - 1;  // residual plane
    const bool zout = zr >= zlo && zr < zhi;
    const long long* c = S + strip * RT_RB * RT_W + tx;  // box row of y0 - 1, column x - 1
    long long hU = c[0] + c[2], mU = c[1];
    long long hC = c[RT_W] + c[RT_W + 2], mC = c[RT_W + 1];
    float* rrow = p.rhs32 + ((long long)zr * np1 + y0) * p.ldx + x;
#pragma unroll
    for (int i = 0; i < RT_RB; ++i) {
      const long long* d = c + (i + 2) * RT_W;
      const long long hD = d[0] + d[2], mD = d[1];
      const long long X = hC + (mU + mD);
      const long long D = hU + hD;
      const long long W = mC * 32 - D * 2;
      const long long Y = -(X * 2 + D);
      if (zout && yin[i]) {
        const long long R = (bc[i] >> bsh) - (P[i] + Y);
        const float Rf = fixed_to_float(R);
        rrow[(long long)i * p.ldx] = one_mul ? Rf * sc : ldexpf(Rf * p.malpha, ks);
        const float Rs = Rf * 2.3283064365386963e-10f;  // 2^-32
        acc = fmaf(Rs, Rs, acc);
      }
      P[i] = W + Ym[i];
      Ym[i] = Y;
      hU = hC;
      mU = mC;
      hC = hD;
      mC = mD;
    }
  }
  // block sum: warp shuffles, then the warps' partial sums
  double dacc = (double)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = dacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RT_NT / 32; ++w) t += red[w];
    const double scd = ldexp(p.alpha, 32 - F);  // r = scd R 2^-32
    const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    p.partials[b] = t * scd * scd * p.hD;
  }
}

// b / alpha in place as 64-bit fixed point with scale 2^(1078 - max(bexp, 1))
__global__ void k_fix_scaled(long long* __restrict__ bq, long long V, const Control* ctl) {
  const int emax = max(ctl->bexp, 1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V;
       i += (long long)gridDim.x * blockDim.x)
    bq[i] = to_fixed(__longlong_as_double(bq[i]), emax);
}

__global__ void k_max_exponent(const double* __restrict__ x, long long V, int* out,
                               const Control* ctl) {
  if (halted(ctl)) return;
  unsigned m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned e =
        (unsigned)(((unsigned long long)__double_as_longlong(x[i]) >> 52) & 0x7ff);
    m = e > m ? e : m;
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, (int)m);
}

__global__ void k_scale(const double* __restrict__ b, double* __restrict__ bq, long long V,
                        double inv_alpha) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V;
       i += (long long)gridDim.x * blockDim.x)
    bq[i] = b[i] * inv_alpha;
}

}  // namespace


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
  const cuuint32_t box_down[3] = {(cuuint32_t)kBoxW, (cuuint32_t)kBoxH, 1};
  const cuuint32_t box_up[3] = {(cuuint32_t)kUpBoxW, (cuuint32_t)kUpBoxH, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  float* bases[6] = {e0, e1, rhs, e0, e1, rhs};
  CUtensorMap* outs[6] = {&maps->e[0],    &maps->e[1],    &maps->rhs,
                          &maps->e_up[0], &maps->e_up[1], &maps->rhs_up};
  for (int i = 0; i < 6; ++i) {
    const cuuint32_t* box = i < 3 ? box_down : box_up;
    if (encode(outs[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, bases[i], dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

void sweep3_grid(int nc, int nz, dim3* grid) {
  const int ni = std::max(1, nc - 1);  // interior coarse columns
  *grid = dim3((ni + UBJX - 1) / UBJX, (ni + UBJY - 1) / UBJY, std::min(std::max(nz, 1), ni));
}

void sweep3_grid_down(int nc, int nz, dim3* grid) {
  const int ni = std::max(1, 3 * nc - 1);  // interior fine rows and planes
  *grid = dim3((ni + 63) / 64, (ni + OH - 1) / OH, std::min(std::max(nz, 1), ni));
}
// threads and blocks per SM of the down-passes
constexpr int kDownNT = 128, kDownMinB = 4;
// the last down-pass holds the next plane's FP64 iterate in registers: three
// blocks per SM
constexpr int kDownUMinB = 3;

int sweep3_default_nz(int nc, int nsm) {
  dim3 g;
  sweep3_grid(nc, 1, &g);
  return std::min(std::max(1, (kUpMinB * nsm) / (int)(g.x * g.y)), std::max(1, nc - 1));
}

int sweep3_default_nz_down(int nc, int nsm) {
  dim3 g;
  sweep3_grid_down(nc, 1, &g);
  return std::min(std::max(1, (kDownMinB * nsm) / (int)(g.x * g.y)), std::max(1, 3 * nc - 1));
}

int sweep3_default_nz_downu(int nc, int nsm) {
  dim3 g;
  sweep3_grid_down(nc, 1, &g);
  return std::min(std::max(1, (kDownUMinB * nsm) / (int)(g.x * g.y)), std::max(1, 3 * nc - 1));
}

bool sweep3_prepare() {
  return cudaFuncSetAttribute(k_up3<SWEEP_UP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)USMEM_BYTES) == cudaSuccess &&
         cudaFuncSetAttribute(k_up3<SWEEP_UPE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)USMEM_BYTES) == cudaSuccess &&
         cudaFuncSetAttribute(k_down3<SWEEP_DOWN, kDownNT, kDownMinB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES) == cudaSuccess &&
         cudaFuncSetAttribute(k_down3<SWEEP_DOWNU, kDownNT, kDownUMinB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES) == cudaSuccess;
}

void launch_sweep3(const Sweep3Params& p, const Sweep3Maps& maps, int ein, int mode,
                   cudaStream_t s) {
  dim3 grid;
  if (mode == SWEEP_DOWN || mode == SWEEP_DOWNU)
    sweep3_grid_down(p.nc, mode == SWEEP_DOWNU ? p.nz_downu : p.nz_down, &grid);
  else
    sweep3_grid(p.nc, p.nz, &grid);
  switch (mode) {
    case SWEEP_UP:
      k_up3<SWEEP_UP><<<grid, UNT, USMEM_BYTES, s>>>(p, maps.e_up[ein], maps.rhs_up);
      break;
    case SWEEP_UPE:
      k_up3<SWEEP_UPE><<<grid, UNT, USMEM_BYTES, s>>>(p, maps.e_up[ein], maps.rhs_up);
      break;
    case SWEEP_DOWN:
      k_down3<SWEEP_DOWN, kDownNT, kDownMinB>
          <<<grid, kDownNT, SMEM_BYTES, s>>>(p, maps.e[ein], maps.rhs);
      break;
    default:
      k_down3<SWEEP_DOWNU, kDownNT, kDownUMinB>
          <<<grid, kDownNT, SMEM_BYTES, s>>>(p, maps.e[ein], maps.rhs);
      break;
  }
}

void refine3_grid(int n, int zc, dim3* grid) {
  // columns and rows 1 .. n - 1 carry residuals
  *grid = dim3((n + RT_X - 1) / RT_X, (n + RT_Y - 1) / RT_Y, (n - 1 + zc - 1) / zc);
}

int refine3_blocks(int n, int zc) {
  dim3 g;
  refine3_grid(n, zc, &g);
  return (int)(g.x * g.y * g.z);
}

int refine3_zc(int n) {
  // one wave of RT_MINB resident blocks on each of the 152 SMs of a GB300: the
  // planes split into as many slabs as that allows.  The rule does not query
  // the device, so the workspace layout (one norm partial per block) is the
  // same wherever it is computed.
  constexpr long long kSlots = 152 * RT_MINB;
  dim3 g;
  refine3_grid(n, 1, &g);
  const long long tiles = (long long)g.x * g.y;
  const long long slabs = std::max(1LL, kSlots / tiles);
  return (int)std::max(1LL, (n - 1 + slabs - 1) / slabs);
}

void launch_fix_scaled(long long* bq, long long V, const Control* ctl, cudaStream_t s) {
  k_fix_scaled<<<152 * 8, 256, 0, s>>>(bq, V, ctl);
}

void launch_max_exponent(const double* x, long long V, int* out, const Control* ctl,
                         cudaStream_t s) {
  k_max_exponent<<<152 * 8, 256, 0, s>>>(x, V, out, ctl);
}

void launch_scale(const double* b, double* bq, long long V, double inv_alpha, cudaStream_t s) {
  k_scale<<<152 * 8, 256, 0, s>>>(b, bq, V, inv_alpha);
}

void launch_refine3(const Refine3Params& p, cudaStream_t s) {
  dim3 grid;
  refine3_grid(p.n, p.zc, &grid);
  k_refine3<<<grid, RT_NT, 0, s>>>(p);
}

}  // namespace adafac
