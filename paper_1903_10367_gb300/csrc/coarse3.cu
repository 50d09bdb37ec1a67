// The small coarse levels of the 3-D uniform path (levels lmin .. T, T <= 3,
// at most 28^3 vertices) in one launch of one block.
//
// Below the finest level, every cycle restricts level by level down to lmin
// and prolongs back up (the nested form of Eq. 9):
//   r_l = P^T r_{l+1},  b~_l = omega S~^T r_{l+1},
//   g_l = M_l^-1 (omega r_l - omega~ b~_l)            [adAFAC-Jac]
//       = gscale_l omega M_l^-1 r_l                   [additive, exponential]
//   t_lmin = g_lmin,  t_l = g_l + P t_{l-1}.
// On levels this small each step is one short dependent phase, and as separate
// launches the chain is bound by launch latency.  Here one block of 1024
// threads runs every phase with a block barrier between them and works out of
// shared memory: r of the top level T and then its g arrive by bulk copies,
// the lower levels' r, g and t stay in shared memory, and r, b~, g and t of
// every level are written to global memory as the level-by-level kernels do.
//   * restriction: one thread per interior coarse vertex over its 5^3 window
//     of the staged fine r, with the d-linear weights and S~ as immediates;
//   * prolongation: the d-linear P is a tensor product, applied in x, then y,
//     then z through two shared-memory scratch arrays; lanes run along x and
//     each warp takes whole planes or rows, so no index is divided in a loop.
// The transfers are d-linear and the coarse operators uniform (the 3-D path's
// preconditions), so P needs no stored weights.
#include <algorithm>

#include "common.cuh"
#include "mbarrier.cuh"
#include "sweep3.cuh"

namespace adafac {

namespace {

constexpr int CNT = 1024;

__device__ __forceinline__ int pow3(int l) {
  int n = 1;
  for (int i = 0; i < l; ++i) n *= 3;
  return n;
}

// one restriction, level l + 1 -> l, from the staged r of level l + 1; g_l
// goes to its shared-memory slot, r_l too when a restriction follows
__device__ void restrict_level(const Coarse3Params& p, int l, float* sm) {
  const int nc = pow3(l), ncp1 = nc + 1, nf = 3 * nc, nfp1 = nf + 1;
  const int Vc = ncp1 * ncp1 * ncp1;
  const float* sRf = sm + p.off_r[l + 1];
  float* sR = sm + p.off_r[l];
  float* sG = sm + p.off_t[l];
  float* r = p.r[l];
  float* bt = p.bt[l];
  float* g = p.g[l];
  const float* invd = p.invd[l];
  const bool keep_r = l > p.lmin;
  // boundary vertices carry nothing
  for (int v = threadIdx.x; v < Vc; v += CNT) {
    const int x = v % ncp1, y = (v / ncp1) % ncp1, z = v / (ncp1 * ncp1);
    if (x > 0 && x < nc && y > 0 && y < nc && z > 0 && z < nc) continue;
    r[v] = 0.f;
    bt[v] = 0.f;
    g[v] = 0.f;
    if (keep_r) sR[v] = 0.f;
    sG[v] = 0.f;
  }
  const int ni = nc - 1, Vi = ni * ni * ni;
  constexpr float kW[5] = {1.f / 3.f, 2.f / 3.f, 1.f, 2.f / 3.f, 1.f / 3.f};
  for (int i = threadIdx.x; i < Vi; i += CNT) {
    const int x = 1 + i % ni, y = 1 + (i / ni) % ni, z = 1 + i / (ni * ni);
    const int v = (z * ncp1 + y) * ncp1 + x;
    const float id = invd[v];
    const float* w0 = sRf + ((3 * z - 2) * nfp1 + (3 * y - 2)) * nfp1 + (3 * x - 2);
    // a plane of the window at a time: its 25 loads are issued before the
    // arithmetic, and two accumulator pairs shorten the dependent chains
    float rc = 0.f, b = 0.f;
#pragma unroll
    for (int oz = 0; oz < 5; ++oz) {
      float val[25];
#pragma unroll
      for (int k = 0; k < 25; ++k) val[k] = w0[(oz * nfp1 + k / 5) * nfp1 + k % 5];
      float r0 = 0.f, r1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
      for (int k = 0; k < 25; ++k) {
        const float wr = kW[k % 5] * kW[k / 5] * kW[oz];
        const float ws = p.stilde[oz * 25 + k];
        if (k & 1) {
          r1 = fmaf(wr, val[k], r1);
          b1 = fmaf(ws, val[k], b1);
        } else {
          r0 = fmaf(wr, val[k], r0);
          b0 = fmaf(ws, val[k], b0);
        }
      }
      rc += r0 + r1;
      b += b0 + b1;
    }
    float gv;
    if (p.variant == V_JAC) {
      b *= p.omega;
      gv = id * (p.omega * rc - p.omega_t * b);
    } else {
      b = 0.f;
      gv = p.gscale[l] * p.omega * id * rc;
    }
    r[v] = rc;
    bt[v] = b;
    g[v] = gv;
    if (keep_r) sR[v] = rc;
    sG[v] = gv;
  }
}

// weights of fine index i towards coarse I = min(i / 3, nc - 1) and I + 1
__device__ __forceinline__ void lerp_at(int i, int nc, int* I, float* t) {
  int c = i / 3;
  c = c < nc - 1 ? c : nc - 1;
  *I = c;
  *t = (float)(i - 3 * c) * (1.f / 3.f);
}

// x and y stages of one prolongation, level l - 1 -> l, into B[Z][yf][xf]
// (lanes along xf; a warp takes whole coarse planes Z in x, then one fine
// row yf over all Z in y, so no index is divided inside the loops)
__device__ void prolong_xy(const Coarse3Params& p, int l, float* sm) {
  const int nf = pow3(l), nfp1 = nf + 1, nc = nf / 3, ncp1 = nc + 1;
  const float* tc = sm + p.off_t[l - 1];
  float* A = sm + p.off_a;  // [Z][Y][xf]
  float* B = sm + p.off_b;  // [Z][yf][xf]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < nfp1) {
    int X;
    float tx;
    lerp_at(lane, nc, &X, &tx);
    for (int Z = warp; Z < ncp1; Z += CNT / 32) {
      const float* src = tc + Z * ncp1 * ncp1 + X;
      float* dst = A + Z * ncp1 * nfp1 + lane;
#pragma unroll 5
      for (int Y = 0; Y < ncp1; ++Y, src += ncp1, dst += nfp1)
        *dst = (1.f - tx) * src[0] + tx * src[1];
    }
  }
  __syncthreads();
  if (lane < nfp1) {
    for (int yf = warp; yf < nfp1; yf += CNT / 32) {
      int Y;
      float ty;
      lerp_at(yf, nc, &Y, &ty);
      const float* a = A + Y * nfp1 + lane;
      float* dst = B + yf * nfp1 + lane;
#pragma unroll 5
      for (int Z = 0; Z < ncp1; ++Z, a += ncp1 * nfp1, dst += nfp1 * nfp1)
        *dst = (1.f - ty) * a[0] + ty * a[nfp1];
    }
  }
  __syncthreads();
}

// z stage: t_l = g_l + (P t_{l-1}), zero on the boundary; g_l is read from
// gsrc, and t_l replaces it there when a prolongation follows.  A warp takes
// whole fine planes zf.
__device__ void prolong_z(const Coarse3Params& p, int l, float* sm, float* gsrc) {
  const int nf = pow3(l), nfp1 = nf + 1, nc = nf / 3;
  const float* B = sm + p.off_b;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* t = p.t[l];
  const bool keep = l < p.T;
  if (lane >= nfp1) return;
  const bool in_x = lane > 0 && lane < nf;
  for (int zf = warp; zf < nfp1; zf += CNT / 32) {
    int Z;
    float tz;
    lerp_at(zf, nc, &Z, &tz);
    const bool in_xz = in_x && zf > 0 && zf < nf;
    const float* b = B + Z * nfp1 * nfp1 + lane;
    int v = zf * nfp1 * nfp1 + lane;
#pragma unroll 4
    for (int yf = 0; yf < nfp1; ++yf, b += nfp1, v += nfp1) {
      const bool interior = in_xz && yf > 0 && yf < nf;
      const float val = interior ? gsrc[v] + ((1.f - tz) * b[0] + tz * b[nfp1 * nfp1]) : 0.f;
      t[v] = val;
      if (keep) gsrc[v] = val;
    }
  }
}

// a bulk copy split into pieces of at most 16 KB (bytes a multiple of 16), so
// that the copy engine works on several at once
__device__ void bulk_load_chunked(float* dst, const float* src, uint32_t bytes, uint32_t bar) {
  constexpr uint32_t kChunk = 16384;
  for (uint32_t off = 0; off < bytes; off += kChunk) {
    const uint32_t n = bytes - off < kChunk ? bytes - off : kChunk;
    bulk_load(smem_addr(dst) + off, reinterpret_cast<const char*>(src) + off, n, bar);
  }
}

// every thread waits (bounded) on phase 0 of the mbarrier; false in all threads
// when any of them gave up, after recording the fault
__device__ bool block_wait(const Coarse3Params& p, uint32_t bar, int where) {
  const bool ok = mbar_wait(bar, 0);
  if (!ok && atomicCAS(p.fault, 0, 1) == 0) {
    p.fault_info[0] = 20;
    p.fault_info[1] = where;
    p.fault_info[6] = threadIdx.x;
  }
  return __syncthreads_and(ok) != 0;
}

__global__ void __launch_bounds__(CNT, 1) k_coarse3(const __grid_constant__ Coarse3Params p) {
  if (halted(p.ctl)) return;
  extern __shared__ __align__(16) float sm[];
  __shared__ __align__(8) uint64_t s_bar[2];
  const int T = p.T;
  const int nT = pow3(T);
  const uint32_t bytesT = 4u * (uint32_t)((nT + 1) * (nT + 1) * (nT + 1));
  float* sRT = sm + p.off_r[T];  // r of level T, later its g
  const uint32_t bar0 = smem_addr(&s_bar[0]), bar1 = smem_addr(&s_bar[1]);
  if (threadIdx.x == 0) {
    mbar_init(bar0);
    mbar_init(bar1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect(bar0, bytesT);
    bulk_load_chunked(sRT, p.r[T], bytesT, bar0);
  }
  if (!block_wait(p, bar0, 0)) return;
  restrict_level(p, T - 1, sm);
  __syncthreads();
  // r of level T is consumed: fetch its g into the same slot meanwhile
  if (threadIdx.x == 0) {
    mbar_expect(bar1, bytesT);
    bulk_load_chunked(sRT, p.g[T], bytesT, bar1);
  }
  for (int l = T - 2; l >= p.lmin; --l) {
    restrict_level(p, l, sm);
    __syncthreads();
  }
  for (int l = p.lmin + 1; l < T; ++l) {
    prolong_xy(p, l, sm);
    prolong_z(p, l, sm, sm + p.off_t[l]);
    __syncthreads();
  }
  prolong_xy(p, T, sm);
  if (!block_wait(p, bar1, 1)) return;
  prolong_z(p, T, sm, sRT);
}

}  // namespace

void coarse3_layout(Coarse3Params* p, size_t* bytes) {
  auto V = [](int l) {
    int n = 1;
    for (int i = 0; i < l; ++i) n *= 3;
    return (n + 1) * (n + 1) * (n + 1);
  };
  for (int l = 0; l <= kCoarse3Top; ++l) p->off_r[l] = p->off_t[l] = 0;
  // r of the levels restricted from (lmin + 1 .. T; the slot of T later
  // holds its g); g, then t, of the levels lmin .. T - 1; the two scratch
  // arrays of the largest prolongation
  int off = 0;
  for (int l = p->lmin + 1; l <= p->T; ++l) {
    p->off_r[l] = off;
    off += (V(l) + 3) & ~3;
  }
  for (int l = p->lmin; l < p->T; ++l) {
    p->off_t[l] = off;
    off += (V(l) + 3) & ~3;
  }
  int na = 0, nb = 0;
  for (int l = p->lmin + 1; l <= p->T; ++l) {
    int nf = 1;
    for (int i = 0; i < l; ++i) nf *= 3;
    const int ncp1 = nf / 3 + 1, nfp1 = nf + 1;
    na = std::max(na, ncp1 * ncp1 * nfp1);
    nb = std::max(nb, ncp1 * nfp1 * nfp1);
  }
  p->off_a = off;
  off += (na + 3) & ~3;
  p->off_b = off;
  off += (nb + 3) & ~3;
  *bytes = sizeof(float) * (size_t)off;
}

bool coarse3_prepare() {
  Coarse3Params p;
  p.T = kCoarse3Top;
  p.lmin = 1;
  size_t bytes = 0;
  coarse3_layout(&p, &bytes);
  return cudaFuncSetAttribute(k_coarse3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes) == cudaSuccess;
}

void launch_coarse3(const Coarse3Params& p, size_t smem_bytes, cudaStream_t s) {
  k_coarse3<<<1, CNT, smem_bytes, s>>>(p);
}

}  // namespace adafac
