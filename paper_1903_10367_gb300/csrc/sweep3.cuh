// Parameters of the 3-D fine-level sweeps (uniform finest operator, d-linear
// transfers) and of the z-marching FP64 refinement residual.
#pragma once

#include <cuda.h>

#include "engine.h"

namespace adafac {

// UP: first up-pass of a refinement step (e = 0); UPE: up-pass of e;
// DOWN: down-pass; DOWNU: last down-pass (u += e, the other buffer zeroed)
enum SweepMode { SWEEP_UP = 0, SWEEP_UPE = 1, SWEEP_DOWN = 2, SWEEP_DOWNU = 3 };

// down-passes: 64 fine columns x kDownRows rows per block (tiles from column
// and row 1: eleven tiles cover the 242 interior rows of a 243-cell grid
// exactly), staged box 68 x (kDownRows + 2) floats (x origin 64 bx, a 16-byte
// boundary)
constexpr int kDownRows = 22;
constexpr int kBoxW = 68, kBoxH = kDownRows + 2;
// up-passes: 20 x 8 interior coarse columns per block, staged box 64 x 28 floats
constexpr int kUpBJX = 20, kUpBJY = 8;
constexpr int kUpBoxW = 64, kUpBoxH = 3 * kUpBJY + 4;

struct Sweep3Params {
  int n = 0, nc = 0;               // fine cells, coarse cells
  int nz = 1;                      // up-passes: slabs of the interior coarse planes
  int nz_down = 1;                 // down-passes: slabs of the interior fine planes
  int nz_downu = 1;                // the last down-pass of a refinement step: the same
  int ldx = 0;                     // row stride of the FP32 fine arrays (multiple of 4)
  // uniform stencil: A e = a_c e + a_f (6 faces) + a_e (12 edges) + a_k (8 corners)
  float a_c = 0, a_f = 0, a_e = 0, a_k = 0;
  float w_invd = 0;                // omega / diag(A_L)
  float* e_out = nullptr;          // DOWN: new correction; DOWNU: zeroed
  const float* q = nullptr;        // level L-1 vector to prolong
  float* r_c = nullptr;            // level L-1 restricted residual
  float* bt_c = nullptr;           // level L-1 damping right-hand side
  float* g_c = nullptr;            // level L-1 combined correction
  float c_invd = 0;                // 1 / diag(A_{L-1}) (uniform)
  float omega = 0, omega_t = 0, gscale = 1;
  int variant = V_JAC;
  // truncated smoothed restriction S~ by class: for |oz| = 0, 1, 2 the weights of
  // the in-plane distance classes (0,0) (1,0) (2,0) (1,1) (1,2) (2,2)
  float dcls[18] = {};
  double* u = nullptr;             // DOWNU: u += e
  const Control* ctl = nullptr;
  int* applied = nullptr;          // &ctl->applied
  int* fault = nullptr;            // &ctl->fault: set when a bounded wait gives up
  int* fault_info = nullptr;       // &ctl->fault_info[0]
  long long wait_polls = 1LL << 22;  // polls of a staged-plane wait before it gives up
  int* uexp = nullptr;             // &ctl->uexp: UP resets it, DOWNU raises it
  const int* bdexp = nullptr;      // &ctl->bdexp
};

// The refinement residual of the uniform 3-D operator A = alpha [32, 0, -2, -1]
// (centre, faces, edges, corners): r = alpha (b / alpha - S u) with the integer
// stencil S evaluated exactly in 64-bit fixed point.
struct Refine3Params {
  int n = 0, zc = 0, ldx = 0;
  double alpha = 0;                // eps h / 12
  float malpha = 0;                // alpha = malpha 2^ealpha, malpha in [0.5, 1)
  int ealpha = 0;
  double hD = 0;
  const double* u = nullptr;
  const long long* bq = nullptr;   // b / alpha in fixed point, scale 2^(1078 - max(bexp, 1))
  float* rhs32 = nullptr;          // padded FP32 layout (row stride ldx)
  double* partials = nullptr;
  const Control* ctl = nullptr;    // uexp, bexp: exponents fixing the scale
};

// Tensor maps of the FP32 fine arrays for the staged loads.
struct Sweep3Maps {
  CUtensorMap e[2];      // down-pass boxes (kBoxW x kBoxH)
  CUtensorMap rhs;
  CUtensorMap e_up[2];   // up-pass boxes (kUpBoxW x kUpBoxH)
  CUtensorMap rhs_up;
};

// Encodes the tensor maps (host; false when the driver entry point is missing).
bool sweep3_make_maps(float* e0, float* e1, float* rhs, int n, int ldx, Sweep3Maps* maps);
// Allows the sweeps' dynamic shared memory (once per process and device).
bool sweep3_prepare();
void launch_sweep3(const Sweep3Params& p, const Sweep3Maps& maps, int ein, int mode,
                   cudaStream_t s);
void sweep3_grid(int nc, int nz, dim3* grid);       // up-passes (20 x 8 coarse columns, nz slabs)
void sweep3_grid_down(int nc, int nz, dim3* grid);  // down-passes (64-column tiles, nz slabs)
// default slab counts: as many as one wave of resident blocks on nsm SMs allows
int sweep3_default_nz(int nc, int nsm);
int sweep3_default_nz_down(int nc, int nsm);
int sweep3_default_nz_downu(int nc, int nsm);
int refine3_blocks(int n, int zc);
// planes per block of the refinement residual (one wave of resident blocks)
int refine3_zc(int n);
void launch_refine3(const Refine3Params& p, cudaStream_t s);
// b / alpha (FP64, in place) to the fixed point of Refine3Params::bq, after
// the largest exponent ctl->bexp has been found
void launch_fix_scaled(long long* bq, long long V, const Control* ctl, cudaStream_t s);
// One restriction (level l + 1 -> l) or prolongation (l - 1 -> l) of the 3-D
// uniform path's coarse levels, with the d-linear weights as constants: n_c /
// n_f are the coarse / fine cell counts.
struct Level3Params {
  int nc = 0, nf = 0;
  int variant = V_JAC;
  float omega = 0.6f, omega_t = 0.6f, gscale = 1.0f;
  float stilde[125] = {};
  const float* r_f = nullptr;   // restriction: fine r
  float* r_c = nullptr;         //   coarse r, b~, g
  float* bt_c = nullptr;
  float* g_c = nullptr;
  const float* invd_c = nullptr;
  const float* t_c = nullptr;   // prolongation: coarse t (or g on level lmin)
  const float* g_f = nullptr;   //   fine g
  float* t_f = nullptr;         //   fine t
  const Control* ctl = nullptr;
};
void launch_restrict3u(const Level3Params& p, cudaStream_t s);
void launch_prolong3u(const Level3Params& p, cudaStream_t s);

// *out = max(*out, largest biased exponent of x[0 .. V)); skipped once halted
void launch_max_exponent(const double* x, long long V, int* out, const Control* ctl,
                         cudaStream_t s);
// bq = b * inv_alpha
void launch_scale(const double* b, double* bq, long long V, double inv_alpha, cudaStream_t s);

}  // namespace adafac
