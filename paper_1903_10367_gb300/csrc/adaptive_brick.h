// Brick engine of the adaptive-tree cycles (adaptive_brick.cu): the
// generating-system cycle of adaptive.cu on per-level full grids.
//
// Level l holds its full (3^l + 1)^D vertex grid and 3^(l D) cell grid.  With
// W_l the residual contributions of level l's leaf cells (their lumped load
// minus their element matrices applied to the level's copy U_l of the
// iterate), the residual level l sees is
//   r_l = Phi_l^T (b - K u) = sum_{m >= l} (P^T)^(m - l) W_m,
// i.e. the chain rho_L = W_L, rho_l = P^T rho_{l+1} + W_l with the d-linear
// P: a level-m contribution at a position reaches a level-l pagoda with the
// pagoda's value there, and contributions of coarser leaf cells vanish at
// every active vertex of level l.  The corrections go back by the chain
// T_lmin = g_lmin, T_l = g_l + P T_{l-1}, and U_l += T_l: at the corners of
// level l's leaf cells the pagodas of finer levels vanish, so U_l keeps the
// iterate's values there (the only values of U_l that are read).  M_l =
// diag(Phi_l^T K Phi_l) comes from the Galerkin element matrices collapsed
// bottom-up, E_l(Q) = sum over the children c of Q of W_c^T E_{l+1}(c) W_c
// (E of a leaf cell: its element matrix).  No index arrays: every step is a
// stencil on a regular grid, restricted to the tiles of the grid that meet
// an existing cell of the level.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "adafac.h"

namespace adafac {
namespace brick {

constexpr int kMaxL = 16;
constexpr int kTX = 32, kTY = 8;   // vertex tile (one z plane in 3-D), one thread per vertex

struct Ctl {
  double r0;        // norm of the residual that defines rel
  double tol;       // solve: stop when rel <= tol (< 0: never)
  double abs;       // last evaluated norm
  double rel;
  int done;         // rel <= tol reached: the rest of the batch returns at entry
  int diverged;     // rel non-finite or > 1e6
  int applied;      // cycles applied
  int pad;
};

struct Level {
  int n = 0, s = 0;                  // cells per axis; fine cells per level cell
  long long V = 0, C = 0;            // vertices, cells
  double *U = nullptr, *R = nullptr, *G = nullptr, *T = nullptr;
  double *IM = nullptr;              // 1 / M_l at active vertices, else 0
  double *B = nullptr;               // lumped load of the level's leaf cells
  double *BT = nullptr;              // b~_l of the last cycle (levels < L)
  double *EL = nullptr;              // eps of the level's leaf cells, else 0
  uint8_t *nodal = nullptr;          // the position's finest active level is l
  uint8_t *leaf = nullptr;           // leaf cells
  // mixed solves: the FP32 correction E_l, its chains, and the FP32 copies
  // of 1 / M_l, eps and of the step's FP64 rho_l (RHS32)
  float *E32 = nullptr, *R32 = nullptr, *G32 = nullptr, *T32 = nullptr;
  float *IM32 = nullptr, *EL32 = nullptr, *RHS32 = nullptr;
  int2* tiles = nullptr;             // tiles meeting an existing cell (column | row << 16, plane)
  int ntiles = 0;
  int part_off = 0;                  // first norm partial of the level
};

struct System {
  int D = 0, L = 0;
  bool mixed = false;                // FP32 cycles with FP64 refinement steps
  Level lev[kMaxL + 1];
  double* part = nullptr;            // one norm partial per tile of every level
  int npart = 0;
  Ctl* ctl = nullptr;
  double stilde[125] = {};
  std::vector<void*> allocs;
};

// The tree as the host holds it: exists[l] / cut[l] per level-l cell (x fastest).
struct Tree {
  std::vector<std::vector<uint8_t>> exists, cut;   // index 1 .. L
};

// Builds the system on the device: eps (scalar or per fine cell) and f (at
// the fine positions) are host arrays.  Synchronises the stream.
adafac_status build(System& S, int D, int L, const Tree& tree, const double* eps, int eps_scalar,
                    const double* f, bool mixed, cudaStream_t s, std::string* err);
void release(System& S);
// One cycle (Eq. 9 on the generating system) of the given variant over
// levels lmin .. L.  with_norm: its residual norm is evaluated first, and
// once rel <= ctl->tol (a solve) the cycle and the rest of the batch return
// at entry.
void enqueue_cycle(System& S, const adafac_options& o, bool with_norm, cudaStream_t s);
// Mixed solves: one refinement step -- the FP64 level residuals rho_l (their
// norm first when with_norm), rounded to FP32, k FP32 cycles on the
// correction equation, U_l += E_l.
void enqueue_step(System& S, const adafac_options& o, int k, bool with_norm, cudaStream_t s);
// The residual chain of every level and the norm of Eq. 10 into ctl->abs / rel.
void enqueue_norm(System& S, cudaStream_t s);
// Leaf-node vectors (fine-grid indices nodes[0 .. nn)) <-> the level copies.
void gather_nodes(System& S, const long long* nodes, int nn, double* u, cudaStream_t s);
void scatter_nodes(System& S, const long long* nodes, int nn, const double* u, cudaStream_t s);
// The function of this grid's space that takes the values v (at the leaf
// nodes; node_map: fine position -> node) at its nodal-space vertices.
void from_node_values(System& S, const int* node_map, const double* v, cudaStream_t s);

}  // namespace brick
}  // namespace adafac
