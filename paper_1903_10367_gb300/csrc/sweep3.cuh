// Parameters of the fused 3-D sweeps (uniform finest operator, d-linear
// transfers) and of the z-marching FP64 refinement residual.
#pragma once

#include "engine.h"

namespace adafac {

enum SweepMode { SWEEP_UP = 0, SWEEP_FULL = 1, SWEEP_DOWNU = 2 };

// coarse columns per block (x, y); the z extent is a launch parameter
constexpr int kSweepBJX = 16, kSweepBJY = 8;

struct Sweep3Params {
  int n = 0, nc = 0, zc = 0;       // fine cells, coarse cells, coarse planes per block
  // uniform stencil: A e = a_c e + a_f (6 faces) + a_e (12 edges) + a_k (8 corners)
  float a_c = 0, a_f = 0, a_e = 0, a_k = 0;
  float w_invd = 0;                // omega / diag(A_L)
  const float* e_in = nullptr;     // previous correction (zero buffer for UP)
  float* e_out = nullptr;          // FULL: new correction; DOWNU: zeroed
  const float* rhs = nullptr;      // right-hand side of the correction equation
  const float* q = nullptr;        // level L-1 vector to prolong
  float* r_c = nullptr;            // level L-1 restricted residual
  float* bt_c = nullptr;           // level L-1 damping right-hand side
  float* g_c = nullptr;            // level L-1 combined correction
  float c_invd = 0;                // 1 / diag(A_{L-1}) (uniform)
  float omega = 0, omega_t = 0, gscale = 1;
  int variant = V_JAC;
  float wres[125] = {};            // restriction weights w(ox) w(oy) w(oz)
  float wdamp[125] = {};           // truncated smoothed restriction (omega applied later)
  double* u = nullptr;             // DOWNU: u += e
  const Control* ctl = nullptr;
  int* applied = nullptr;          // &ctl->applied
};

struct Refine3Params {
  int n = 0, zc = 0;
  double a_c = 0, a_f = 0, a_e = 0, a_k = 0;
  double hD = 0;
  const double* u = nullptr;
  const double* b = nullptr;
  float* rhs32 = nullptr;
  double* partials = nullptr;
  const Control* ctl = nullptr;
};

void launch_sweep3(const Sweep3Params& p, int mode, cudaStream_t s);
void sweep3_grid(int nc, int bjx, int bjy, int zc, dim3* grid);
int refine3_blocks(int n, int zc);
void launch_refine3(const Refine3Params& p, cudaStream_t s);

}  // namespace adafac
