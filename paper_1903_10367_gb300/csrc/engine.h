// Internal header of the adAFAC CUDA library: level views passed to kernels
// by value, and the host-side launch wrappers the engine calls.
//
// Geometry: a level with n cells per dimension has np1 = n+1 vertices per
// dimension, V = np1^D vertices in total, linear index x + np1 (y + np1 z).
// Cells (n^D) use the same order.  Corner c of a cell has offset bit
// (c >> j) & 1 along dimension j (x = 0); stencil entry s has offset
// o_j = (s / 3^j) % 3 - 1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adafac.h"

namespace adafac {

constexpr int kMaxLevels = 16;

enum OpKind { OP_EPS = 0, OP_STORED = 1, OP_UNIFORM = 2 };
enum Variant { V_ADDITIVE = 0, V_JAC = 1, V_PI = 2, V_EXP = 3 };

// The operator, inverse diagonal and incoming prolongation of one level, in
// element type T (double for FP64 work, float for the FP32 cycles).
template <typename T>
struct LevelView {
  int n = 0, np1 = 0;
  long long V = 0;
  int opkind = OP_UNIFORM;
  const T* st = nullptr;     // OP_STORED: 3^D entries per vertex, entry-major
  const T* eps = nullptr;    // OP_EPS: per-cell eps (n^D)
  T hfac = 0;                // h^(D-2) of the level
  T eps0 = 0;                // fine level with scalar eps: the value
  T cst[27] = {};            // OP_UNIFORM: the stencil
  const T* invd = nullptr;   // 1/diag per vertex, or nullptr -> invd0
  T invd0 = 0;
  int boxmg = 0;             // prolongation from level l-1: 0 d-linear, 1 stored
  const T* P = nullptr;      // BoxMG: 2^D weights per vertex, entry-major
};

// Cycle parameters shared by the kernels.
template <typename T>
struct CycleParams {
  int variant = V_JAC;
  int rtilde_exact = 0;
  T omega = T(0.6), omega_tilde = T(0.6);
  T stilde[125] = {};        // truncated smoothed-restriction stencil (5^D)
};

// Device-side control block (one per handle).
struct Control {
  double r0sq;        // ||r_0||_h^2
  double lastsq;      // last evaluated ||r||_h^2 (cycle evaluations)
  double rel;         // last normalised residual (cycle evaluations)
  double tol;         // convergence threshold on rel (solve), or -1
  double qsq;         // ||r||_h^2 of the last explicit query
  double qrel;        // its normalised value
  int done;           // 1 once rel <= tol: later kernels of the batch return
  int diverged;       // 1 once rel is non-finite or > 1e6
  int nhist;          // entries written to the history
  int applied;        // cycles applied (one per update kernel that ran)
  int set_r0;         // 1: the next norm evaluation defines r_0
  int fault;          // 1: a bounded device-side wait gave up (reported as TIMEOUT)
  int fault_info[8];  // where it gave up: mode, block, step index, slot, parity, z
  int uexp;           // largest biased binary exponent of the fine iterate u (3-D uniform
                      // path: exact at the start of a refinement step; the step's first
                      // up-pass resets it to bdexp, its last down-pass raises it to the
                      // exponents of the u it writes)
  int bexp;           // largest biased binary exponent of b / alpha (3-D uniform path)
  int bdexp;          // largest biased binary exponent of the Dirichlet values of u
};

// ---- batched refinement steps (batch.cu) -------------------------------------
// One instance of the batched path: everything a refinement step of a mixed
// solve touches, on the device (the handle's workspace holds it).  Level l =
// 1 .. L; P of level l weights level l's vertices towards the corners of
// their level-(l-1) cell (BoxMG), null for d-linear weights.
struct BatchLevel {
  int n = 0;                   // cells per axis
  int pad = 0;
  long long V = 0;             // vertices (n + 1)^D
  const float* invd = nullptr; // 1/diag per vertex, or null -> invd0
  const float* P = nullptr;
  float* r = nullptr;          // r_l (level L: the FP32 residual)
  float* bt = nullptr;         // b~_l
  float* g = nullptr;          // g_l = c_l - c~_l
  float* t = nullptr;          // t_l = g_l + P q_{l-1}
  float invd0 = 0.f;
  float gscale = 1.f;          // EXP: omega_exp^(L - l)
};

struct BatchItem {
  int L = 0, lmin = 1, variant = V_JAC, nunits = 0;
  float omega = 0.6f, omega_t = 0.6f;
  float hfac32 = 1.f, eps0f = 0.f;   // FP32 fine operator: h^(D-2), scalar eps
  double hfac = 1.0, eps0 = 0.0;     // FP64 fine operator
  double hD = 0.0;                   // h^D of the finest level (Eq. 10)
  const double* eps = nullptr;       // per-cell eps (null: scalar eps0)
  const float* eps32 = nullptr;
  double* u = nullptr;
  const double* b = nullptr;
  float* e = nullptr;                // correction of the FP32 cycles
  float* rhs = nullptr;              // FP32 right-hand side (the FP64 residual)
  double* partials = nullptr;        // one norm partial per unit of vertices
  Control* ctl = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  int pad = 0;
  float stilde[125] = {};            // truncated smoothed restriction (5^D)
  BatchLevel lev[kMaxLevels + 1];
};

constexpr int kBatchThreads = 512;   // threads per CTA; a unit is this many vertices
constexpr int kBatchMax = 64;        // instances per launch

struct BatchLaunch {
  const BatchItem* item[kBatchMax];
  int k[kBatchMax];                  // FP32 cycles of the step, per instance
  Control* mirror = nullptr;         // optional: mirror[i] = control block of item i at the end
  int count = 0;
  int dyn_bytes = 0;                 // one-CTA instances: shared memory for their vectors
};

// Shared memory a one-CTA instance may take for its FP32 vectors.
constexpr int kBatchOnchipBytes = 100 << 10;
// Bytes of the FP32 vectors an instance keeps on chip when it runs on one
// CTA, or 0 when they exceed kBatchOnchipBytes.
int batch_onchip_bytes(const BatchItem& host_item);

// CTAs per instance (a power of two, at most 16) for a fine grid of V
// vertices: one when the vectors fit on chip (onchip_bytes > 0).
int batch_cluster_size(long long V, int onchip_bytes);
// The largest cluster the device places (16, else 8).
int batch_max_cluster();
// Norm partials the batched step writes for a fine grid of V vertices.
inline long long batch_units(long long V) { return (V + kBatchThreads - 1) / kBatchThreads; }
// One launch: a cluster of C CTAs per item, every item of dimension D and
// cluster size C.  Returns the launch's error.
cudaError_t launch_batch_step(int D, int C, const BatchLaunch& bl, cudaStream_t s);

// ---- handle internals used by the request server ---------------------------
// The batched path's instance of a handle (null unless the handle runs the
// batched path), its dimension, cluster size and on-chip bytes
// (batch_onchip_bytes).
const BatchItem* handle_batch_item(adafac_handle h, int* D, int* C, int* onchip_bytes);
Control* handle_control(adafac_handle h);
// ctl->tol = rel_tol, ctl->done = 0 (synchronises the handle's stream)
adafac_status handle_arm(adafac_handle h, double rel_tol);

// ---- setup launches (FP64) -------------------------------------------------
template <int D>
void launch_rhs(const double* f, double* b, int n, cudaStream_t s);
template <int D>
void launch_fine_invdiag(const LevelView<double>& fine, double* invd, cudaStream_t s);
template <int D>
void launch_boxmg(const LevelView<double>& fine, double* P, int n_c, cudaStream_t s);
// Rediscretised coarse element matrices: eps of a coarse cell = mean of the
// eps of its 3^D children (from eps on the finest level, from the stored
// element matrices below it).
template <int D>
void launch_rediscretise(const LevelView<double>& fine, const double* Kc_fine, double* Kc,
                         int n_c, cudaStream_t s);
template <int D>
void launch_galerkin(const LevelView<double>& fine, const double* Kc_fine,
                     double* Kc_coarse, int n_c, cudaStream_t s);
template <int D>
void launch_assemble(const double* Kc, double* st, double* invd, int n, cudaStream_t s);
void launch_to_float(const double* src, float* dst, long long count, cudaStream_t s);
void launch_fill(double* dst, double value, long long count, cudaStream_t s);

// ---- cycle launches --------------------------------------------------------
// r = b - A x at the interior vertices of level `lv` (b may be null = 0);
// optional FP32 copy r32; optional per-block sums of h^D r^2 into partials.
template <int D, typename T, typename TX>
void launch_residual(const LevelView<T>& lv, const TX* x, const TX* b, TX* r,
                     float* r32, double* partials, int nblocks, double hD,
                     const Control* ctl, cudaStream_t s);
// Restriction from fine level lf to coarse level lc and the per-level
// correction: r_c = P^T r_f (unless given), b~_c, g_c.
template <int D, typename T>
void launch_restrict(const LevelView<T>& lf, const LevelView<T>& lc,
                     const CycleParams<T>& cp, const T* r_f, const T* y_f,
                     T* r_c, int rc_given, T* bt_c, T* g_c, T gscale,
                     const Control* ctl, cudaStream_t s);
// y = A (invd .* r) on level lv (exact smoothed restriction).
template <int D, typename T>
void launch_apply_scaled(const LevelView<T>& lv, const T* r, T* y,
                         const Control* ctl, cudaStream_t s);
// Prolongation chain on a coarse level l >= 2: t_l = g_l + P q_{l-1} with
// q = t_{l-1} (- I g_l for adAFAC-PI).
template <int D, typename T>
void launch_prolong(const LevelView<T>& lf, const LevelView<T>& lc,
                    const CycleParams<T>& cp, const T* t_c, const T* g_f, T* t_f,
                    const Control* ctl, cudaStream_t s);
// Fine update x += c_L + P q_{L-1}, c_L = omega invd r_L.
template <int D, typename T, typename TX>
void launch_update(const LevelView<T>& lf, const LevelView<T>& lc,
                   const CycleParams<T>& cp, const T* r_f, const T* t_c, TX* x,
                   const Control* ctl, cudaStream_t s);
// FAS: hierarchical u^_f = u_f - P I u_f (u_f given on level lf; the injected
// coarse values are read at stride 3).
template <int D>
void launch_hierarchical(const LevelView<double>& lf, const LevelView<double>& lc,
                         const double* u_f, const double* u_c, double* uhat,
                         const Control* ctl, cudaStream_t s);
template <int D>
void launch_inject(const double* u_f, int n_f, double* u_c, const Control* ctl,
                   cudaStream_t s);
template <int D>
void launch_restrict_plain(const LevelView<double>& lf, const LevelView<double>& lc,
                           const double* r_f, double* b_c, const Control* ctl,
                           cudaStream_t s);
// ---- grid-shaped level launches of the mixed-precision cycles (level.cu) ----
// Launch shape of a vertex-grid kernel: bx x by threads (whole warps, at most
// 256), zr planes per thread column of the 3-D residual (0: a size rule);
// bx = by = 0 takes 32 x 8.  The arithmetic of every vertex is the same for
// every shape.
struct GridShape {
  int bx = 0, by = 0, zr = 0;
};
// Blocks of the residual on a level with n cells (one norm partial per block).
template <int D>
int residual_g_blocks(int n);
// r = b - A x on the finest level (OP_EPS or OP_UNIFORM), r zero on the
// boundary; with partials: per-block sums of h^D r^2 in a fixed order.
template <int D, typename T, typename TO>
void launch_residual_g(const LevelView<T>& lv, const T* x, const T* b, TO* r,
                       double* partials, double hD, const Control* ctl, cudaStream_t s,
                       GridShape shape = GridShape());
// r_c = P^T r_f, b~_c (truncated R~, JAC), g_c: one thread per coarse vertex.
template <int D>
void launch_restrict_g(const LevelView<float>& lf, const LevelView<float>& lc,
                       const CycleParams<float>& cp, const float* r_f, float* r_c,
                       float* bt_c, float* g_c, float gscale, const Control* ctl,
                       cudaStream_t s);
// UPDATE: x += omega M^-1 r_f + P q (finest level; counts the cycle);
// else x = g_f + P q (coarse level t, zero on the boundary).
template <int D, bool UPDATE>
void launch_prolong_g(const LevelView<float>& lf, const LevelView<float>& lc,
                      const CycleParams<float>& cp, const float* r_f, const float* g_f,
                      const float* t_c, float* x, Control* ctl, cudaStream_t s,
                      GridShape shape = GridShape());
// Sums the partials of one norm evaluation (fixed order), records history,
// sets done / diverged.
// query != 0: only qsq/qrel (and r_0 when set_r0) are written, regardless of
// done/diverged.
void launch_norm_finalize(const double* partials, int nblocks, Control* ctl,
                          double* hist, int hist_cap, int query, cudaStream_t s);
// Resets the control block (r_0 taken at the next evaluation, empty history).
void launch_reset_control(Control* ctl, cudaStream_t s);
// MIXED: u += e, e = 0.
void launch_refine_update(double* u, float* e, long long V, const Control* ctl,
                          cudaStream_t s);

}  // namespace adafac
