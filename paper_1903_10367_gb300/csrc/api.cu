// C ABI of the adAFAC library (declared in include/adafac.h): handle
// lifetime, workspace layout, setup orchestration and the per-cycle launch
// sequences.  Every numerical step runs in the kernels of setup.cu and
// cycle.cu on the handle's stream.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/adafac.h"
#include "engine.h"
#include "coarse3.cuh"
#include "sweep3.cuh"

using namespace adafac;

namespace {

constexpr int kHistCap = 8192;
constexpr int kNormBlocks = 152 * 8;
// coarse grids up to this many vertices take the warp-per-vertex restriction
// in the mixed cycles: there a thread per coarse vertex leaves most of the
// GPU idle and each thread's 5^d window is a long dependent chain
constexpr long long kWarpRestrictMaxV = 4096;

struct Graph {
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
};

thread_local std::string g_setup_error;

struct LevelData {
  int n = 0;
  long long V = 0;
  double *st = nullptr, *invd = nullptr, *P = nullptr, *Kc = nullptr;
  double *r = nullptr, *bt = nullptr, *g = nullptr, *t = nullptr, *y = nullptr;
  double *ul = nullptr, *bl = nullptr, *uhat = nullptr;
  float *st32 = nullptr, *invd32 = nullptr, *P32 = nullptr;
  float *r32 = nullptr, *bt32 = nullptr, *g32 = nullptr, *t32 = nullptr, *y32 = nullptr;
  LevelView<double> v64;
  LevelView<float> v32;
};

// Bump allocator over the workspace; with base == nullptr it only measures.
struct Carver {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(long long count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * (size_t)(count > 0 ? count : 0);
    return p;
  }
};

long long ipow_ll(long long b, int e) {
  long long r = 1;
  while (e-- > 0) r *= b;
  return r;
}

}  // namespace

struct adafac_handle_s {
  int D = 0, L = 0;
  adafac_options opt{};
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  bool uniform = false;    // scalar eps and d-linear: every level's stencil is uniform
  int eps_scalar = 0;
  double eps0 = 0.0;
  LevelData lev[kMaxLevels + 1];
  double *u = nullptr, *b = nullptr, *eps = nullptr;
  float *eps32 = nullptr, *e32 = nullptr, *rhs32 = nullptr;
  double* partials = nullptr;
  Control* ctl = nullptr;
  double* hist = nullptr;
  CycleParams<double> cp64;
  CycleParams<float> cp32;
  std::string err;
  uint64_t launches = 0;
  // per-kernel timing (adafac_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> marks[ADAFAC_KERNEL_KINDS];
  // fused 3-D path (uniform operator, d-linear transfers, mixed precision)
  bool fast3 = false;
  float* e32b = nullptr;     // second correction buffer (ping-pong)
  int ebase = 0;             // which of e32 / e32b holds zeros at a step start
  double* bq = nullptr;      // b / alpha (3-D uniform path; fixed point after setup)
  double* ub = nullptr;      // Dirichlet values on the boundary, zero inside
  long long e_elems = 0;     // floats of e32 / e32b / rhs32 (padded rows on the 3-D path)
  int npartials = 0;
  int ldx = 0;               // row stride of the padded FP32 fine arrays
  Sweep3Maps maps;
  Sweep3Params sw;
  Refine3Params rf;
  // launch shapes of the fine residual and update of the level path (autotuned)
  GridShape res_shape, upd_shape;
  // batched refinement steps (path BATCHED): the instance on the device, its
  // host image, the CTAs per instance
  bool batched = false;
  BatchItem* bitem = nullptr;
  BatchItem bitem_host;
  int bC = 1;
  int bonchip = 0;           // bytes of FP32 vectors kept on chip at one CTA (0: none)
  // CUDA graphs of whole cycle batches / refinement steps
  bool use_graphs = true;
  cudaStream_t cap = nullptr;
  std::map<long, Graph> graphs;
};

namespace {

adafac_status fail(adafac_handle h, adafac_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_setup_error = msg;
  return st;
}

adafac_status check_cuda(adafac_handle h, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(h, ADAFAC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return ADAFAC_OK;
}

cudaEvent_t next_event(adafac_handle h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// Runs `launch`, bracketed by timing events when timing is on.
template <typename F>
void timed(adafac_handle h, int kind, F&& launch) {
  if (!h->timing || kind >= ADAFAC_KERNEL_KINDS) {
    launch();
    return;
  }
  cudaEvent_t a = next_event(h), b = next_event(h);
  cudaEventRecord(a, h->stream);
  launch();
  cudaEventRecord(b, h->stream);
  h->marks[kind].emplace_back(a, b);
}

bool valid_options(const adafac_options* o, std::string* why) {
  if (o->variant < 0 || o->variant > 3) return *why = "variant out of range", false;
  if (o->transfer < 0 || o->transfer > 1) return *why = "transfer out of range", false;
  if (o->precision < 0 || o->precision > 1) return *why = "precision out of range", false;
  if (o->rtilde < 0 || o->rtilde > 1) return *why = "rtilde out of range", false;
  if (o->form < 0 || o->form > 1) return *why = "form out of range", false;
  if (o->form == ADAFAC_FORM_FAS && o->precision != ADAFAC_PRECISION_FP64)
    return *why = "FAS form requires FP64 precision", false;
  if (o->inner_cycles < 1) return *why = "inner_cycles must be >= 1", false;
  if (o->path < 0 || o->path > 3) return *why = "path out of range", false;
  if (o->path == ADAFAC_PATH_BATCHED &&
      (o->precision != ADAFAC_PRECISION_MIXED ||
       (o->variant == ADAFAC_VARIANT_JAC && o->rtilde == ADAFAC_RTILDE_EXACT)))
    return *why = "path BATCHED needs MIXED precision and the truncated R~ for JAC", false;
  if (o->coarse_op < 0 || o->coarse_op > 1) return *why = "coarse_op out of range", false;
  if (o->lmin < 1) return *why = "lmin must be >= 1", false;
  if (!(o->omega > 0.0) || !(o->omega_tilde >= 0.0) || !(o->omega_exp > 0.0))
    return *why = "damping factors must be positive", false;
  return true;
}

bool valid_tree(const adafac_tree* t, std::string* why) {
  if (t->dim != 2 && t->dim != 3) return *why = "dim must be 2 or 3", false;
  if (t->depth < 1 || t->depth > kMaxLevels) return *why = "depth must be in 1..16", false;
  const long long np1 = ipow_ll(3, t->depth) + 1;
  if ((double)ipow_ll(np1, t->dim) >= 2147483647.0)
    return *why = "tree too large: (3^depth+1)^dim must be < 2^31", false;
  return true;
}

// The fused 3-D sweeps cover the uniform (scalar eps, d-linear) mixed
// precision cycles of adAFAC-Jac with the truncated smoothed restriction and
// of plain / exponentially damped additive multigrid, in correction form.
bool fast3_eligible(const adafac_handle_s* h) {
  const adafac_options& o = h->opt;
  return o.path == ADAFAC_PATH_AUTO && h->D == 3 && h->L >= 2 && o.lmin < h->L && h->uniform &&
         o.precision == ADAFAC_PRECISION_MIXED &&
         o.form == ADAFAC_FORM_CS && o.rtilde == ADAFAC_RTILDE_TRUNCATED &&
         (o.variant == ADAFAC_VARIANT_JAC || o.variant == ADAFAC_VARIANT_ADDITIVE ||
          o.variant == ADAFAC_VARIANT_EXP);
}

// Path BATCHED, or AUTO on the smallest grids (at most kAutoBatchMaxV fine
// vertices: 2-D depth <= 3, 3-D depth <= 2) outside the fused 3-D path: there
// a refinement step in one launch on one CTA, with its vectors in shared
// memory, is faster than a graph of level kernels, and the request server
// batches such requests into shared launches.
constexpr long long kAutoBatchMaxV = 1024;

bool batched_choice(const adafac_handle_s* h) {
  const adafac_options& o = h->opt;
  if (o.path == ADAFAC_PATH_BATCHED) return true;
  const bool covered = o.precision == ADAFAC_PRECISION_MIXED && o.form == ADAFAC_FORM_CS &&
                       !(o.variant == ADAFAC_VARIANT_JAC && o.rtilde == ADAFAC_RTILDE_EXACT);
  return o.path == ADAFAC_PATH_AUTO && covered && !h->fast3 &&
         ipow_ll(ipow_ll(3, h->L) + 1, h->D) <= kAutoBatchMaxV;
}

// Carves every array of the handle (measure-only when base is null).
void carve(adafac_handle h, Carver& cv) {
  const int D = h->D, L = h->L;
  const bool mixed = h->opt.precision == ADAFAC_PRECISION_MIXED;
  const bool boxmg = h->opt.transfer == ADAFAC_TRANSFER_BOXMG;
  const bool exact = h->opt.rtilde == ADAFAC_RTILDE_EXACT && h->opt.variant == ADAFAC_VARIANT_JAC;
  const bool fas = h->opt.form == ADAFAC_FORM_FAS;
  const int NC = 1 << D, NS = D == 2 ? 9 : 27;
  for (int l = 1; l <= L; ++l) {
    LevelData& lv = h->lev[l];
    lv.n = (int)ipow_ll(3, l);
    lv.V = ipow_ll(lv.n + 1, D);
    const long long ncell = ipow_ll(lv.n, D);
    // decisions depend on the configuration only, never on pointers: the
    // measuring pass (base == nullptr) must carve exactly what the real one does
    const bool stored = l < L && !h->uniform;
    const bool has_p = l >= 2 && boxmg;
    lv.invd = cv.take<double>(lv.V);
    if (stored) {
      lv.st = cv.take<double>(NS * lv.V);
      lv.Kc = cv.take<double>((long long)NC * NC * ncell);
    }
    if (has_p) lv.P = cv.take<double>(NC * lv.V);
    lv.r = cv.take<double>(lv.V);  // fine level: FP64 residual / f staging
    if (!mixed) {
      if (l < L) {
        lv.bt = cv.take<double>(lv.V);
        lv.g = cv.take<double>(lv.V);
        lv.t = cv.take<double>(lv.V);
      }
      if ((exact || fas) && l >= 2) lv.y = cv.take<double>(lv.V);
      if (fas && l < L) {
        lv.ul = cv.take<double>(lv.V);
        lv.bl = cv.take<double>(lv.V);
      }
      if (fas && l >= 2) lv.uhat = cv.take<double>(lv.V);
    } else {
      lv.invd32 = cv.take<float>(lv.V);
      if (stored) lv.st32 = cv.take<float>(NS * lv.V);
      if (has_p) lv.P32 = cv.take<float>(NC * lv.V);
      lv.r32 = cv.take<float>(lv.V);
      if (l < L) {
        lv.bt32 = cv.take<float>(lv.V);
        lv.g32 = cv.take<float>(lv.V);
        lv.t32 = cv.take<float>(lv.V);
      }
      if (exact && l >= 2) lv.y32 = cv.take<float>(lv.V);
    }
  }
  const long long Vf = h->lev[L].V;
  h->u = cv.take<double>(Vf);
  h->ub = cv.take<double>(Vf);
  h->b = cv.take<double>(Vf);
  if (h->fast3) h->bq = cv.take<double>(Vf);
  if (h->batched) h->bitem = cv.take<BatchItem>(1);
  if (!h->eps_scalar) {
    h->eps = cv.take<double>(ipow_ll(h->lev[L].n, D));
    if (mixed) h->eps32 = cv.take<float>(ipow_ll(h->lev[L].n, D));
  }
  if (mixed) {
    // the fused path stages planes with the tensor memory accelerator, which
    // needs row strides that are multiples of 16 bytes: pad rows to 4 floats
    const long long np1 = h->lev[L].n + 1;
    h->ldx = h->fast3 ? (int)((np1 + 3) / 4 * 4) : (int)np1;
    const long long Vp = h->fast3 ? (long long)h->ldx * np1 * np1 : Vf;
    h->e_elems = Vp;
    h->e32 = cv.take<float>(Vp);
    h->rhs32 = cv.take<float>(Vp);
    if (h->fast3) h->e32b = cv.take<float>(Vp);
  }
  // one norm partial per block of the refinement residual in use (the fused
  // path may still fall back to the level kernels at setup)
  h->npartials = kNormBlocks;
  if (h->fast3)
    h->npartials =
        std::max(h->npartials, refine3_blocks(h->lev[L].n, refine3_zc(h->lev[L].n)));
  if (mixed)
    h->npartials = std::max(h->npartials, D == 2 ? residual_g_blocks<2>(h->lev[L].n)
                                                 : residual_g_blocks<3>(h->lev[L].n));
  if (h->batched) h->npartials = std::max<long long>(h->npartials, batch_units(Vf));
  h->partials = cv.take<double>(h->npartials);
  h->ctl = cv.take<Control>(1);
  h->hist = cv.take<double>(kHistCap);
}

// Reference stencil (eps = 1, without the h^(D-2) factor): the neighbour at
// offset o shares 2^(D-k) cells with the centre (k non-zero components of o),
// each contributing K_ref(k).
void ref_stencil(int D, double* st) {
  const double k2[3] = {2.0 / 3.0, -1.0 / 6.0, -1.0 / 3.0};
  const double k3[4] = {1.0 / 3.0, 0.0, -1.0 / 12.0, -1.0 / 12.0};
  const int NS = D == 2 ? 9 : 27;
  for (int s = 0; s < NS; ++s) {
    int t = s, k = 0;
    for (int j = 0; j < D; ++j) {
      k += (t % 3) != 1;
      t /= 3;
    }
    st[s] = (double)(1 << (D - k)) * (D == 2 ? k2[k] : k3[k]);
  }
}

// The truncated smoothed restriction stencil: (M^-1 A_{eps=1} P e_J) at the
// fine vertices 3J + o, o in [-2, 2]^D, for d-linear P (Sec. 3.2, option 1),
// ordered with x fastest.  The mesh width cancels between A and M.
void smoothed_stencil(int D, double* out) {
  double st[27];
  ref_stencil(D, st);
  const int NS = D == 2 ? 9 : 27;
  const int N5 = D == 2 ? 25 : 125;
  const double centre = st[(NS - 1) / 2];
  for (int k = 0; k < N5; ++k) {
    int o[3] = {0, 0, 0}, t = k;
    for (int j = 0; j < D; ++j) {
      o[j] = t % 5 - 2;
      t /= 5;
    }
    double acc = 0.0;
    for (int s = 0; s < NS; ++s) {
      int u = s;
      double hat = 1.0;
      for (int j = 0; j < D; ++j) {
        const int p = o[j] + (u % 3) - 1;
        u /= 3;
        const double w = 1.0 - std::fabs((double)p) / 3.0;
        hat *= w > 0.0 ? w : 0.0;
      }
      acc += st[s] * hat;
    }
    out[k] = acc / centre;
  }
}

template <typename T>
void fill_uniform_view(LevelView<T>& v, int D, double eps, int n) {
  double st[27];
  ref_stencil(D, st);
  const double hf = D == 2 ? 1.0 : 1.0 / n;
  v.opkind = OP_UNIFORM;
  for (int s = 0; s < (D == 2 ? 9 : 27); ++s) v.cst[s] = (T)(eps * hf * st[s]);
  v.invd0 = (T)(1.0 / (eps * hf * st[D == 2 ? 4 : 13]));
  v.eps0 = (T)eps;
}

template <int D>
adafac_status run_setup(adafac_handle h, const double* eps_in, const double* f_in, int on_dev) {
  const int L = h->L;
  cudaStream_t s = h->stream;
  const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  LevelData& fine = h->lev[L];
  const long long ncf = ipow_ll(fine.n, D);
  // eps
  if (!h->eps_scalar) {
    if (cudaMemcpyAsync(h->eps, eps_in, sizeof(double) * ncf, kind, s) != cudaSuccess)
      return check_cuda(h, "copy eps");
  }
  // right-hand side: f staged in the fine residual array, then b = h^D f
  if (f_in) {
    if (cudaMemcpyAsync(fine.r, f_in, sizeof(double) * fine.V, kind, s) != cudaSuccess)
      return check_cuda(h, "copy f");
    launch_rhs<D>(fine.r, h->b, fine.n, s);
  } else {
    cudaMemsetAsync(h->b, 0, sizeof(double) * fine.V, s);
  }
  // level views (FP64)
  for (int l = 1; l <= L; ++l) {
    LevelData& lv = h->lev[l];
    LevelView<double>& v = lv.v64;
    v = LevelView<double>();
    v.n = lv.n;
    v.np1 = lv.n + 1;
    v.V = lv.V;
    v.hfac = D == 2 ? 1.0 : 1.0 / lv.n;
    v.invd = lv.invd;
    v.boxmg = lv.P ? 1 : 0;
    v.P = lv.P;
    if (l == L) {
      if (h->eps_scalar) {
        fill_uniform_view(v, D, h->eps0, lv.n);
        v.invd = lv.invd;
      } else {
        v.opkind = OP_EPS;
        v.eps = h->eps;
      }
    } else if (h->uniform) {
      fill_uniform_view(v, D, h->eps0, lv.n);
      v.invd = lv.invd;
    } else {
      v.opkind = OP_STORED;
      v.st = lv.st;
    }
  }
  // fine inverse diagonal
  launch_fine_invdiag<D>(fine.v64, fine.invd, s);
  // hierarchy: P_l, Galerkin A_{l-1}, assembled stencils
  for (int l = L; l >= 2; --l) {
    LevelData& lf = h->lev[l];
    LevelData& lc = h->lev[l - 1];
    if (lf.P) {
      LevelView<double> vf = lf.v64;
      vf.boxmg = 0;
      launch_boxmg<D>(vf, lf.P, lc.n, s);
      if (check_cuda(h, "boxmg") != ADAFAC_OK) return ADAFAC_ERR_CUDA;
    }
    if (!h->uniform) {
      if (h->opt.coarse_op == ADAFAC_COARSE_REDISCRETISED)
        launch_rediscretise<D>(lf.v64, l == L ? nullptr : lf.Kc, lc.Kc, lc.n, s);
      else
        launch_galerkin<D>(lf.v64, l == L ? nullptr : lf.Kc, lc.Kc, lc.n, s);
      launch_assemble<D>(lc.Kc, lc.st, lc.invd, lc.n, s);
    } else {
      launch_fine_invdiag<D>(lc.v64, lc.invd, s);
    }
    if (check_cuda(h, "galerkin") != ADAFAC_OK) return ADAFAC_ERR_CUDA;
  }
  // cycle parameters
  double sd[125];
  smoothed_stencil(D, sd);
  h->cp64 = CycleParams<double>();
  h->cp64.variant = h->opt.variant;
  h->cp64.rtilde_exact = h->opt.rtilde == ADAFAC_RTILDE_EXACT;
  h->cp64.omega = h->opt.omega;
  h->cp64.omega_tilde = h->opt.omega_tilde;
  for (int k = 0; k < 125; ++k) h->cp64.stilde[k] = sd[k];
  h->cp32 = CycleParams<float>();
  h->cp32.variant = h->cp64.variant;
  h->cp32.rtilde_exact = h->cp64.rtilde_exact;
  h->cp32.omega = (float)h->opt.omega;
  h->cp32.omega_tilde = (float)h->opt.omega_tilde;
  for (int k = 0; k < 125; ++k) h->cp32.stilde[k] = (float)sd[k];
  // FP32 copies for the mixed mode
  if (h->opt.precision == ADAFAC_PRECISION_MIXED) {
    const int NC = 1 << D, NS = D == 2 ? 9 : 27;
    if (h->eps32) launch_to_float(h->eps, h->eps32, ncf, s);
    for (int l = 1; l <= L; ++l) {
      LevelData& lv = h->lev[l];
      launch_to_float(lv.invd, lv.invd32, lv.V, s);
      if (lv.st) launch_to_float(lv.st, lv.st32, NS * lv.V, s);
      if (lv.P) launch_to_float(lv.P, lv.P32, NC * lv.V, s);
      const LevelView<double>& a = lv.v64;
      LevelView<float>& v = lv.v32;
      v = LevelView<float>();
      v.n = a.n;
      v.np1 = a.np1;
      v.V = a.V;
      v.opkind = a.opkind;
      v.st = lv.st32;
      v.eps = h->eps32;
      v.hfac = (float)a.hfac;
      v.eps0 = (float)a.eps0;
      for (int k = 0; k < 27; ++k) v.cst[k] = (float)a.cst[k];
      v.invd = lv.invd32;
      v.invd0 = (float)a.invd0;
      v.boxmg = a.boxmg;
      v.P = lv.P32;
    }
    cudaMemsetAsync(h->e32, 0, sizeof(float) * (size_t)h->e_elems, s);
  }
  if (h->fast3) {
    // stencil classes of the uniform 27-point operator: centre, face, edge, corner
    const LevelView<double>& a = fine.v64;
    Sweep3Params& sw = h->sw;
    sw = Sweep3Params();
    sw.n = fine.n;
    sw.nc = h->lev[L - 1].n;
    {
      // slabs along z: as many as one wave of resident blocks allows
      int dev = 0, nsm = 152;
      if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      sw.nz = sweep3_default_nz(sw.nc, nsm);
      sw.nz_down = sweep3_default_nz_down(sw.nc, nsm);
      sw.nz_downu = sweep3_default_nz_downu(sw.nc, nsm);
    }
    sw.a_c = (float)a.cst[13];
    sw.a_f = (float)a.cst[12];
    sw.a_e = (float)a.cst[9];
    sw.a_k = (float)a.cst[0];
    sw.w_invd = (float)(h->opt.omega * a.invd0);
    sw.r_c = h->lev[L - 1].r32;
    sw.bt_c = h->lev[L - 1].bt32;
    sw.g_c = h->lev[L - 1].g32;
    sw.c_invd = (float)h->lev[L - 1].v64.invd0;
    sw.omega = (float)h->opt.omega;
    sw.omega_t = (float)h->opt.omega_tilde;
    sw.gscale = h->opt.variant == ADAFAC_VARIANT_EXP ? (float)h->opt.omega_exp : 1.0f;
    sw.variant = h->opt.variant;
    // S~ by class (|oz|; in-plane distances); the class form is exact because
    // S~ is symmetric under reflections and permutations of the axes -- checked
    const int cls_of[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    double dcls[18];
    bool filled[18] = {};
    bool symmetric = true;
    for (int k = 0; k < 125; ++k) {
      const int ax = std::abs(k % 5 - 2), ay = std::abs((k / 5) % 5 - 2), az = std::abs(k / 25 - 2);
      const int c = 6 * az + cls_of[ay][ax];
      if (!filled[c]) {
        dcls[c] = sd[k];
        filled[c] = true;
      } else if (std::fabs(dcls[c] - sd[k]) > 1e-14 * (1.0 + std::fabs(sd[k]))) {
        symmetric = false;
      }
    }
    if (!symmetric) return fail(h, ADAFAC_ERR_INVALID_ARG, "smoothed restriction not symmetric");
    for (int c = 0; c < 18; ++c) sw.dcls[c] = (float)dcls[c];
    sw.ldx = h->ldx;
    sw.u = h->u;
    sw.ctl = h->ctl;
    sw.applied = &h->ctl->applied;
    sw.fault = &h->ctl->fault;
    sw.fault_info = &h->ctl->fault_info[0];
    sw.uexp = &h->ctl->uexp;
    sw.bdexp = &h->ctl->bdexp;
    Refine3Params& rf = h->rf;
    rf = Refine3Params();
    rf.n = fine.n;
    rf.zc = refine3_zc(fine.n);
    rf.ldx = h->ldx;
    // A = alpha [32, 0, -2, -1]: the refinement residual sums the integer
    // stencil exactly (checked to the last bits of the assembled coefficients)
    rf.alpha = -a.cst[0];
    const bool integer_stencil =
        rf.alpha > 0.0 && std::fabs(a.cst[13] - 32.0 * rf.alpha) <= 1e-14 * a.cst[13] &&
        std::fabs(a.cst[9] + 2.0 * rf.alpha) <= 1e-14 * rf.alpha;
    int ealpha = 0;
    rf.malpha = (float)std::frexp(rf.alpha, &ealpha);
    rf.ealpha = ealpha;
    rf.hD = std::pow(1.0 / fine.n, 3);
    rf.u = h->u;
    rf.bq = reinterpret_cast<const long long*>(h->bq);
    rf.rhs32 = h->rhs32;
    rf.partials = h->partials;
    rf.ctl = h->ctl;
    h->ebase = 0;
    // the fused sweep evaluates the trilinear stencil without face terms,
    // which are exactly zero for the d-linear element in 3-D
    if (a.cst[12] != 0.0 || !integer_stencil || !sweep3_prepare() ||
        !sweep3_make_maps(h->e32, h->e32b, h->rhs32, fine.n, h->ldx, &h->maps)) {
      cudaGetLastError();
      h->fast3 = false;  // no tensor-map encoder: level-by-level kernels
    }
  }
  if (h->batched) {
    BatchItem& it = h->bitem_host;
    it = BatchItem();
    it.L = L;
    it.lmin = h->opt.lmin;
    it.variant = h->opt.variant;
    it.nunits = (int)batch_units(fine.V);
    it.omega = h->cp32.omega;
    it.omega_t = h->cp32.omega_tilde;
    it.hfac = fine.v64.hfac;
    it.hfac32 = (float)fine.v64.hfac;
    it.eps0 = h->eps0;
    it.eps0f = (float)h->eps0;
    it.hD = std::pow(1.0 / fine.n, D);
    it.eps = h->eps_scalar ? nullptr : h->eps;
    it.eps32 = h->eps_scalar ? nullptr : h->eps32;
    it.u = h->u;
    it.b = h->b;
    it.e = h->e32;
    it.rhs = h->rhs32;
    it.partials = h->partials;
    it.ctl = h->ctl;
    it.hist = h->hist;
    it.hist_cap = kHistCap;
    for (int k = 0; k < 125; ++k) it.stilde[k] = h->cp32.stilde[k];
    for (int l = 1; l <= L; ++l) {
      const LevelData& lv = h->lev[l];
      BatchLevel& bl = it.lev[l];
      bl.n = lv.n;
      bl.V = lv.V;
      bl.invd = lv.invd32;
      bl.invd0 = lv.v32.invd0;
      bl.P = lv.P32;
      bl.r = lv.r32;
      bl.bt = lv.bt32;
      bl.g = lv.g32;
      bl.t = lv.t32;
      bl.gscale =
          h->opt.variant == ADAFAC_VARIANT_EXP ? (float)std::pow(h->opt.omega_exp, (double)(L - l)) : 1.0f;
    }
    h->bonchip = batch_onchip_bytes(it);
    h->bC = batch_cluster_size(fine.V, h->bonchip);
    if (cudaMemcpyAsync(h->bitem, &it, sizeof(BatchItem), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return check_cuda(h, "copy batch item");
  }
  cudaMemsetAsync(h->u, 0, sizeof(double) * fine.V, s);
  Control c{};
  c.tol = -1.0;
  c.set_r0 = 1;
  cudaMemcpyAsync(h->ctl, &c, sizeof(Control), cudaMemcpyHostToDevice, s);
  if (h->fast3) {
    // b / alpha and its largest exponent, for the fixed-point refinement residual
    launch_scale(h->b, h->bq, fine.V, 1.0 / h->rf.alpha, s);
    launch_max_exponent(h->bq, fine.V, &h->ctl->bexp, nullptr, s);
    launch_fix_scaled(reinterpret_cast<long long*>(h->bq), fine.V, h->ctl, s);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return check_cuda(h, "setup");
  return check_cuda(h, "setup");
}

double hD_of(adafac_handle h) {
  return std::pow(1.0 / h->lev[h->L].n, h->D);
}

// One FP64 cycle (Algorithm 1 or a variant) on u.
template <int D>
void fp64_cycle(adafac_handle h) {
  const int L = h->L;
  const int lmin = h->opt.lmin;
  cudaStream_t s = h->stream;
  LevelData* lv = h->lev;
  const CycleParams<double>& cp = h->cp64;
  const bool exact = cp.rtilde_exact && cp.variant == V_JAC;
  timed(h, ADAFAC_KERNEL_FINE_RESIDUAL, [&] {
    launch_residual<D, double, double>(lv[L].v64, h->u, h->b, lv[L].r, nullptr, h->partials,
                                       kNormBlocks, hD_of(h), h->ctl, s);
  });
  launch_norm_finalize(h->partials, kNormBlocks, h->ctl, h->hist, kHistCap, 0, s);
  h->launches += 2;
  const bool fas = h->opt.form == ADAFAC_FORM_FAS;
  if (fas) {
    // Eq. 4: u_l = I u_{l+1}, u^_{l+1} = u_{l+1} - P u_l,
    // b_l = R (b_{l+1} - A_{l+1} u^_{l+1}), r_l = b_l - A_l u_l
    for (int l = L - 1; l >= lmin; --l) {
      const double* uf = l + 1 == L ? h->u : lv[l + 1].ul;
      const double* bf = l + 1 == L ? h->b : lv[l + 1].bl;
      launch_inject<D>(uf, lv[l + 1].n, lv[l].ul, h->ctl, s);
      launch_hierarchical<D>(lv[l + 1].v64, lv[l].v64, uf, lv[l].ul, lv[l + 1].uhat, h->ctl, s);
      launch_residual<D, double, double>(lv[l + 1].v64, lv[l + 1].uhat, bf, lv[l + 1].y, nullptr,
                                         nullptr, 0, 0.0, h->ctl, s);
      launch_restrict_plain<D>(lv[l + 1].v64, lv[l].v64, lv[l + 1].y, lv[l].bl, h->ctl, s);
      launch_residual<D, double, double>(lv[l].v64, lv[l].ul, lv[l].bl, lv[l].r, nullptr, nullptr,
                                         0, 0.0, h->ctl, s);
      h->launches += 5;
    }
  }
  for (int l = L - 1; l >= lmin; --l) {
    const double gscale =
        cp.variant == V_EXP ? std::pow(h->opt.omega_exp, (double)(L - l)) : 1.0;
    if (exact) {
      launch_apply_scaled<D, double>(lv[l + 1].v64, lv[l + 1].r, lv[l + 1].y, h->ctl, s);
      h->launches += 1;
    }
    timed(h, l + 1 == L ? ADAFAC_KERNEL_FINE_RESTRICT : ADAFAC_KERNEL_KINDS, [&] {
      launch_restrict<D, double>(lv[l + 1].v64, lv[l].v64, cp, lv[l + 1].r, lv[l + 1].y,
                                 lv[l].r, fas ? 1 : 0, lv[l].bt, lv[l].g, gscale, h->ctl, s);
    });
    h->launches += 1;
  }
  // t_1 = g_1; t_l = g_l + P q_{l-1}
  for (int l = lmin + 1; l <= L - 1; ++l) {
    const double* tc = l - 1 == lmin ? lv[lmin].g : lv[l - 1].t;
    launch_prolong<D, double>(lv[l].v64, lv[l - 1].v64, cp, tc, lv[l].g, lv[l].t, h->ctl, s);
    h->launches += 1;
  }
  LevelView<double> empty;
  const double* tc = L > lmin ? (L - 1 == lmin ? lv[lmin].g : lv[L - 1].t) : nullptr;
  timed(h, ADAFAC_KERNEL_FINE_UPDATE, [&] {
    launch_update<D, double, double>(lv[L].v64, L > lmin ? lv[L - 1].v64 : empty, cp, lv[L].r,
                                     tc, h->u, h->ctl, s);
  });
  h->launches += 1;
}

// One FP32 cycle on the correction equation A e = rhs32 (mixed mode): the
// grid-shaped level kernels (level.cu), or with path GENERIC the generic
// per-level kernels (cycle.cu).  The exact smoothed restriction, and the
// restriction to small coarse grids, take the generic restriction.
template <int D>
void fp32_cycle(adafac_handle h) {
  const int L = h->L;
  const int lmin = h->opt.lmin;
  cudaStream_t s = h->stream;
  LevelData* lv = h->lev;
  const CycleParams<float>& cp = h->cp32;
  const bool exact = cp.rtilde_exact && cp.variant == V_JAC;
  const bool grid = h->opt.path != ADAFAC_PATH_GENERIC;
  timed(h, ADAFAC_KERNEL_FINE_RESIDUAL, [&] {
    if (grid)
      launch_residual_g<D, float, float>(lv[L].v32, h->e32, h->rhs32, lv[L].r32, nullptr, 0.0,
                                         h->ctl, s, h->res_shape);
    else
      launch_residual<D, float, float>(lv[L].v32, h->e32, h->rhs32, lv[L].r32, nullptr, nullptr,
                                       0, 0.0, h->ctl, s);
  });
  h->launches += 1;
  for (int l = L - 1; l >= lmin; --l) {
    const float gscale =
        cp.variant == V_EXP ? (float)std::pow(h->opt.omega_exp, (double)(L - l)) : 1.0f;
    if (exact) {
      launch_apply_scaled<D, float>(lv[l + 1].v32, lv[l + 1].r32, lv[l + 1].y32, h->ctl, s);
      h->launches += 1;
    }
    timed(h, l + 1 == L ? ADAFAC_KERNEL_FINE_RESTRICT : ADAFAC_KERNEL_KINDS, [&] {
      // a thread per coarse vertex on large coarse grids; on small ones a warp
      // per coarse vertex (its 32 lanes share the window) keeps more threads busy
      if (grid && !exact && lv[l].V > kWarpRestrictMaxV)
        launch_restrict_g<D>(lv[l + 1].v32, lv[l].v32, cp, lv[l + 1].r32, lv[l].r32, lv[l].bt32,
                             lv[l].g32, gscale, h->ctl, s);
      else
        launch_restrict<D, float>(lv[l + 1].v32, lv[l].v32, cp, lv[l + 1].r32, lv[l + 1].y32,
                                  lv[l].r32, 0, lv[l].bt32, lv[l].g32, gscale, h->ctl, s);
    });
    h->launches += 1;
  }
  for (int l = lmin + 1; l <= L - 1; ++l) {
    const float* tc = l - 1 == lmin ? lv[lmin].g32 : lv[l - 1].t32;
    if (grid)
      launch_prolong_g<D, false>(lv[l].v32, lv[l - 1].v32, cp, nullptr, lv[l].g32, tc,
                                 lv[l].t32, h->ctl, s);
    else
      launch_prolong<D, float>(lv[l].v32, lv[l - 1].v32, cp, tc, lv[l].g32, lv[l].t32, h->ctl, s);
    h->launches += 1;
  }
  LevelView<float> empty;
  const float* tc = L > lmin ? (L - 1 == lmin ? lv[lmin].g32 : lv[L - 1].t32) : nullptr;
  timed(h, ADAFAC_KERNEL_FINE_UPDATE, [&] {
    if (grid)
      launch_prolong_g<D, true>(lv[L].v32, L > lmin ? lv[L - 1].v32 : empty, cp, lv[L].r32,
                                nullptr, tc, h->e32, h->ctl, s, h->upd_shape);
    else
      launch_update<D, float, float>(lv[L].v32, L > lmin ? lv[L - 1].v32 : empty, cp, lv[L].r32,
                                     tc, h->e32, h->ctl, s);
  });
  h->launches += 1;
}

// FP64 residual of u (norm recorded as a cycle evaluation) and its FP32 copy
// as the right-hand side of the correction equation.
template <int D>
void refine_residual(adafac_handle h) {
  const int L = h->L;
  const bool grid = h->opt.path != ADAFAC_PATH_GENERIC;
  const int nb = grid ? residual_g_blocks<D>(h->lev[L].n) : kNormBlocks;
  timed(h, ADAFAC_KERNEL_REFINE, [&] {
    if (grid)
      launch_residual_g<D, double, float>(h->lev[L].v64, h->u, h->b, h->rhs32, h->partials,
                                          hD_of(h), h->ctl, h->stream);
    else
      launch_residual<D, double, double>(h->lev[L].v64, h->u, h->b, nullptr, h->rhs32,
                                         h->partials, kNormBlocks, hD_of(h), h->ctl, h->stream);
  });
  launch_norm_finalize(h->partials, nb, h->ctl, h->hist, kHistCap, 0, h->stream);
  h->launches += 2;
}

// k FP32 cycles on the correction equation and u += e (the refinement step
// without its leading residual)
template <int D>
void mixed_body(adafac_handle h, int k) {
  for (int i = 0; i < k; ++i) fp32_cycle<D>(h);
  launch_refine_update(h->u, h->e32, h->lev[h->L].V, h->ctl, h->stream);
  h->launches += 1;
}

template <int D>
void mixed_step(adafac_handle h, int k) {
  refine_residual<D>(h);
  mixed_body<D>(h, k);
}

// Coarse levels L-1 .. 1 of an FP32 cycle whose level L-1 vectors came from a
// fused sweep: restrictions below L-1, then the prolongation chain up to L-1.
void coarse_chain32(adafac_handle h) {
  const int L = h->L;
  const int lmin = h->opt.lmin;
  cudaStream_t s = h->stream;
  LevelData* lv = h->lev;
  const CycleParams<float>& cp = h->cp32;
  // the chain runs on the 3-D uniform path only: constant d-linear weights
  Level3Params lp;
  lp.variant = cp.variant;
  lp.omega = cp.omega;
  lp.omega_t = cp.omega_tilde;
  for (int k = 0; k < 125; ++k) lp.stilde[k] = cp.stilde[k];
  lp.ctl = h->ctl;
  auto restrict_to = [&](int l) {  // level l + 1 -> l
    Level3Params q = lp;
    q.nc = lv[l].n;
    q.nf = lv[l + 1].n;
    q.gscale = cp.variant == V_EXP ? (float)std::pow(h->opt.omega_exp, (double)(L - l)) : 1.0f;
    q.r_f = lv[l + 1].r32;
    q.r_c = lv[l].r32;
    q.bt_c = lv[l].bt32;
    q.g_c = lv[l].g32;
    q.invd_c = lv[l].invd32;
    return q;
  };
  auto prolong_to = [&](int l) {  // level l - 1 -> l
    Level3Params q = lp;
    q.nc = lv[l - 1].n;
    q.nf = lv[l].n;
    q.t_c = l - 1 == lmin ? lv[lmin].g32 : lv[l - 1].t32;
    q.g_f = lv[l].g32;
    q.t_f = lv[l].t32;
    return q;
  };
  // lmin = 1 and level 3 below the finest: levels 2 -> 1 -> 2 -> 3 in one launch
  Bottom3Params bp;
  const bool bottom = lmin == 1 && L - 1 >= 3;
  if (bottom) {
    bp.r21 = restrict_to(1);
    bp.p12 = prolong_to(2);
    bp.p23 = prolong_to(3);
  }
  const bool fused = bottom && bottom3u_applies(bp);
  for (int l = L - 2; l >= (fused ? 2 : lmin); --l) {
    launch_restrict3u(restrict_to(l), s);
    h->launches += 1;
  }
  if (fused) {
    launch_bottom3u(bp, s);
    h->launches += 1;
  }
  for (int l = fused ? 4 : lmin + 1; l <= L - 1; ++l) {
    launch_prolong3u(prolong_to(l), s);
    h->launches += 1;
  }
}

// One refinement step of the 3-D uniform path with k >= 1 FP32 cycles:
//   r = b - A u (FP64), rhs = (float) r;  UP: restrict rhs (cycle 1's up-pass);
//   for cycles j = 2 .. k: DOWN (down-pass of cycle j-1, e into the other
//   buffer), UPE (up-pass of cycle j from that e), coarse levels;
//   DOWNU: down-pass of cycle k and u += e.  Returns the zero buffer of the
//   next step.
void fast3_refine(adafac_handle h) {
  const Refine3Params rf = h->rf;
  // the scale of the fixed-point residual follows the largest |u|: ctl->uexp
  // is exact here (set by the last down-pass before it, or by the call that
  // set u)
  timed(h, ADAFAC_KERNEL_REFINE, [&] { launch_refine3(rf, h->stream); });
  launch_norm_finalize(h->partials, refine3_blocks(h->lev[h->L].n, rf.zc), h->ctl, h->hist,
                       kHistCap, 0, h->stream);
  h->launches += 2;
}

// The cycles of a refinement step of the 3-D uniform path after its residual.
int fast3_body(adafac_handle h, int k, int ebase);

int fast3_step(adafac_handle h, int k, int ebase) {
  fast3_refine(h);
  return fast3_body(h, k, ebase);
}

int fast3_body(adafac_handle h, int k, int ebase) {
  const int L = h->L;
  cudaStream_t s = h->stream;
  Sweep3Params p = h->sw;
  const int lmin = h->opt.lmin;
  p.q = L - 1 == lmin ? h->lev[lmin].g32 : h->lev[L - 1].t32;
  float* E[2] = {h->e32, h->e32b};
  int cur = ebase;
  timed(h, ADAFAC_KERNEL_FINE_RESTRICT,
        [&] { launch_sweep3(p, h->maps, cur, SWEEP_UP, s); });
  h->launches += 1;
  coarse_chain32(h);
  for (int j = 2; j <= k; ++j) {
    p.e_out = E[1 - cur];
    timed(h, ADAFAC_KERNEL_FINE_DOWN, [&] { launch_sweep3(p, h->maps, cur, SWEEP_DOWN, s); });
    timed(h, ADAFAC_KERNEL_FINE_UP, [&] { launch_sweep3(p, h->maps, 1 - cur, SWEEP_UPE, s); });
    h->launches += 2;
    coarse_chain32(h);
    cur ^= 1;
  }
  p.e_out = E[1 - cur];
  timed(h, ADAFAC_KERNEL_FINE_DOWN_U,
        [&] { launch_sweep3(p, h->maps, cur, SWEEP_DOWNU, s); });
  h->launches += 1;
  return 1 - cur;
}

// Runs `enqueue` as a CUDA graph captured once per key (replayed afterwards);
// direct launches while kernel timing is on or when capture is unavailable.
template <typename F>
void run_graph(adafac_handle h, long key, F&& enqueue) {
  if (h->timing || !h->use_graphs) {
    enqueue();
    return;
  }
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      h->use_graphs = false;
      enqueue();
      return;
    }
    const uint64_t before = h->launches;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->use_graphs = false;
      enqueue();
      return;
    }
    cudaStream_t saved = h->stream;
    h->stream = h->cap;
    enqueue();
    h->stream = saved;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    const uint64_t kernels = h->launches - before;
    h->launches = before;
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->use_graphs = false;
      enqueue();
      return;
    }
    Graph gr;
    gr.exec = ex;
    gr.kernels = kernels;
    it = h->graphs.emplace(key, gr).first;
  }
  cudaGraphLaunch(it->second.exec, h->stream);
  h->launches += it->second.kernels;
}

// One refinement step of the batched path with k FP32 cycles (k = 0: only
// the FP64 residual and its norm), this handle alone in the launch.
void batch_step(adafac_handle h, int k) {
  BatchLaunch bl;
  bl.item[0] = h->bitem;
  bl.k[0] = k;
  bl.count = 1;
  bl.dyn_bytes = h->bC == 1 ? h->bonchip : 0;
  timed(h, ADAFAC_KERNEL_BATCH_STEP, [&] {
    const cudaError_t e = launch_batch_step(h->D, h->bC, bl, h->stream);
    if (e != cudaSuccess) h->err = std::string("batched step: ") + cudaGetErrorString(e);
  });
  h->launches += 1;
}

template <int D>
void enqueue_cycles(adafac_handle h, int n) {
  if (h->batched) {
    while (n > 0) {
      const int k = n < h->opt.inner_cycles ? n : h->opt.inner_cycles;
      batch_step(h, k);
      n -= k;
    }
    return;
  }
  if (h->opt.precision == ADAFAC_PRECISION_FP64) {
    while (n > 0) {
      const int b = n < 8 ? n : 8;
      run_graph(h, 1000 + b, [&] {
        for (int i = 0; i < b; ++i) fp64_cycle<D>(h);
      });
      n -= b;
    }
    return;
  }
  while (n > 0) {
    const int k = n < h->opt.inner_cycles ? n : h->opt.inner_cycles;
    if (h->fast3) {
      const int e0 = h->ebase;
      int e1 = e0;
      run_graph(h, 4000 + 2 * k + e0, [&] { e1 = fast3_step(h, k, e0); });
      h->ebase = e0 ^ (k & 1);
      (void)e1;
    } else {
      run_graph(h, 2000 + k, [&] { mixed_step<D>(h, k); });
    }
    n -= k;
  }
}

// The refinement residual of u and its norm alone: the start of a mixed
// solve on the fused or level kernels.
template <int D>
void enqueue_refine_only(adafac_handle h) {
  if (h->fast3) run_graph(h, 6000, [&] { fast3_refine(h); });
  else run_graph(h, 6001, [&] { refine_residual<D>(h); });
}

// k FP32 cycles, u += e, then the residual of the new u and its norm: the
// steps of a mixed solve after its first residual.  The norm that ends the
// solve is the last work enqueued, so no step runs (or returns at entry)
// after it.
template <int D>
void enqueue_solve_group(adafac_handle h, int k) {
  if (h->fast3) {
    const int e0 = h->ebase;
    run_graph(h, 5000 + 2 * k + e0, [&] {
      fast3_body(h, k, e0);
      fast3_refine(h);
    });
    h->ebase = e0 ^ (k & 1);
  } else {
    run_graph(h, 3000 + k, [&] {
      mixed_body<D>(h, k);
      refine_residual<D>(h);
    });
  }
}

template <int D>
void enqueue_query(adafac_handle h) {
  const int L = h->L;
  launch_residual<D, double, double>(h->lev[L].v64, h->u, h->b, nullptr, nullptr, h->partials,
                                     kNormBlocks, hD_of(h), nullptr, h->stream);
  launch_norm_finalize(h->partials, kNormBlocks, h->ctl, h->hist, kHistCap, 1, h->stream);
  h->launches += 2;
}

adafac_status read_ctl(adafac_handle h, Control* c) {
  if (cudaMemcpyAsync(c, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->stream) !=
      cudaSuccess)
    return check_cuda(h, "read control");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "synchronise");
  if (c->fault) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "a bounded device-side wait gave up (mode %d block %d step %d/%d slot %d "
             "parity %d plane %d thread %d)",
             c->fault_info[0], c->fault_info[1], c->fault_info[2], c->fault_info[7],
             c->fault_info[3], c->fault_info[4], c->fault_info[5], c->fault_info[6]);
    return fail(h, ADAFAC_ERR_TIMEOUT, buf);
  }
  return check_cuda(h, "control");
}

template <typename F>
adafac_status write_ctl_field(adafac_handle h, size_t offset, const F& value) {
  if (cudaMemcpyAsync(reinterpret_cast<char*>(h->ctl) + offset, &value, sizeof(F),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return check_cuda(h, "write control");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "synchronise");
  return ADAFAC_OK;
}

// Boundary vertices of u take the Dirichlet values of ub (interior ones keep
// theirs): interior = false.  Interior vertices are zeroed and boundary ones
// kept: interior = true (the masked copy of Dirichlet data).
__global__ void k_boundary(double* u, const double* ub, int n, int D, int interior) {
  const long long np1 = n + 1;
  const long long V = D == 2 ? np1 * np1 : np1 * np1 * np1;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(v % np1), y = (int)((v / np1) % np1);
    const int z = D == 2 ? 1 : (int)(v / (np1 * np1));
    const bool bnd = x == 0 || y == 0 || x == n || y == n || (D == 3 && (z == 0 || z == n));
    if (interior) {
      if (!bnd) u[v] = 0.0;
    } else if (bnd) {
      u[v] = ub ? ub[v] : 0.0;
    }
  }
}

adafac_status reset_control(adafac_handle h) {
  launch_reset_control(h->ctl, h->stream);
  const size_t ebytes = sizeof(float) * (size_t)h->e_elems;
  if (h->e32) cudaMemsetAsync(h->e32, 0, ebytes, h->stream);
  if (h->e32b) cudaMemsetAsync(h->e32b, 0, ebytes, h->stream);
  h->ebase = 0;
  return check_cuda(h, "reset");
}

}  // namespace

namespace adafac {

// The truncated smoothed-restriction stencil for other parts of the library
// (the adaptive-tree cycles).
void smoothed_restriction_stencil(int D, double* out) { smoothed_stencil(D, out); }

// Internal accessors for the request server (same library, not part of the
// C ABI).
Control* handle_control(adafac_handle h) { return h->ctl; }

const BatchItem* handle_batch_item(adafac_handle h, int* D, int* C, int* onchip_bytes) {
  if (!h || !h->batched) return nullptr;
  if (D) *D = h->D;
  if (C) *C = h->bC;
  if (onchip_bytes) *onchip_bytes = h->bonchip;
  return h->bitem;
}

adafac_status handle_arm(adafac_handle h, double rel_tol) {
  adafac_status st = write_ctl_field(h, offsetof(Control, tol), rel_tol);
  if (st != ADAFAC_OK) return st;
  int zero = 0;
  return write_ctl_field(h, offsetof(Control, done), zero);
}

}  // namespace adafac

// ---- autotuner helpers -----------------------------------------------------------
namespace {

// Tuned shapes of the process, by device and problem shape: a handle whose
// shape was tuned before takes the stored result without timing.
struct TuneKey {
  int dev, D, L, fast3, opkind, boxmg, variant, lmin;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, D, L, fast3, opkind, boxmg, variant, lmin) <
           std::tie(o.dev, o.D, o.L, o.fast3, o.opkind, o.boxmg, o.variant, o.lmin);
  }
};
std::mutex g_tune_lock;
std::map<TuneKey, adafac_tuning> g_tune_cache;

// Mean device time of `reps` launches (after one untimed launch), in us.
template <typename F>
double time_us(adafac_handle h, int reps, F&& launch) {
  cudaEvent_t a = next_event(h), b = next_event(h);
  launch();
  cudaEventRecord(a, h->stream);
  for (int i = 0; i < reps; ++i) launch();
  cudaEventRecord(b, h->stream);
  float ms = 0.0f;
  if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
    return -1.0;
  h->ev_used -= 2;
  return 1e3 * ms / reps;
}

// Slab counts along z of the fused sweeps worth timing: every count whose
// slabs are 3 to 24 coarse planes thick (planes: the interior planes of the
// sweep's level, 3 per coarse plane on the fine level), at least one.
std::vector<int> nz_candidates(int planes, int per_coarse) {
  const int lo = std::max(1, (planes + 24 * per_coarse - 1) / (24 * per_coarse));
  const int hi = std::max(lo, planes / (3 * per_coarse));
  std::vector<int> out;
  for (int nz = lo; nz <= hi; ++nz) out.push_back(nz);
  return out;
}

template <int D>
adafac_status tune_level(adafac_handle h, int reps, adafac_tuning* t) {
  const int L = h->L, lmin = h->opt.lmin;
  LevelData* lv = h->lev;
  cudaStream_t s = h->stream;
  const float* tc = L > lmin ? (L - 1 == lmin ? lv[lmin].g32 : lv[L - 1].t32) : nullptr;
  LevelView<float> empty;
  auto res = [&](GridShape g) {
    return time_us(h, reps, [&] {
      launch_residual_g<D, float, float>(lv[L].v32, h->e32, h->rhs32, lv[L].r32, nullptr, 0.0,
                                         h->ctl, s, g);
    });
  };
  auto upd = [&](GridShape g) {
    return time_us(h, reps, [&] {
      launch_prolong_g<D, true>(lv[L].v32, L > lmin ? lv[L - 1].v32 : empty, h->cp32, lv[L].r32,
                                nullptr, tc, h->e32, h->ctl, s, g);
    });
  };
  const int shapes[6][2] = {{32, 8}, {64, 4}, {32, 4}, {128, 2}, {64, 2}, {256, 1}};
  const int zrs[6] = {0, 2, 4, 8, 16, 32};
  const double res0 = res(GridShape()), upd0 = upd(GridShape());
  if (res0 < 0.0 || upd0 < 0.0) return check_cuda(h, "autotune timing");
  double best_res = res0, best_upd = upd0;
  GridShape g_res, g_upd;
  int timed = 2;
  for (const auto& sh : shapes) {
    for (int zr : zrs) {
      if (D == 2 && zr != 0) continue;
      if (zr > lv[L].n + 1) continue;
      GridShape g;
      g.bx = sh[0];
      g.by = sh[1];
      g.zr = zr;
      const double us = res(g);
      ++timed;
      if (us > 0.0 && us < best_res) best_res = us, g_res = g;
    }
    GridShape g;
    g.bx = sh[0];
    g.by = sh[1];
    const double us = upd(g);
    ++timed;
    if (us > 0.0 && us < best_upd) best_upd = us, g_upd = g;
  }
  // keep the default unless the gain is clear of the timing noise
  if (best_res > 0.98 * res0) g_res = GridShape(), best_res = res0;
  if (best_upd > 0.98 * upd0) g_upd = GridShape(), best_upd = upd0;
  h->res_shape = g_res;
  h->upd_shape = g_upd;
  t->path = 2;
  t->res_bx = g_res.bx ? g_res.bx : 32;
  t->res_by = g_res.by ? g_res.by : 8;
  t->res_zr = g_res.zr;
  t->upd_bx = g_upd.bx ? g_upd.bx : 32;
  t->upd_by = g_upd.by ? g_upd.by : 8;
  t->candidates = timed;
  t->us_default = res0 + upd0;
  t->us_tuned = best_res + best_upd;
  return check_cuda(h, "autotune");
}

adafac_status tune_fast3(adafac_handle h, int reps, adafac_tuning* t) {
  const int L = h->L, lmin = h->opt.lmin;
  cudaStream_t s = h->stream;
  Sweep3Params p = h->sw;
  p.q = L - 1 == lmin ? h->lev[lmin].g32 : h->lev[L - 1].t32;
  p.e_out = h->e32b;
  auto sweep = [&](int mode, int nz) {
    Sweep3Params q = p;
    if (mode == SWEEP_UPE) q.nz = nz;
    else q.nz_down = nz;
    return time_us(h, reps, [&] { launch_sweep3(q, h->maps, mode == SWEEP_UPE ? 1 : 0, mode, s); });
  };
  const int nc = h->lev[L - 1].n;
  const double up0 = sweep(SWEEP_UPE, p.nz), down0 = sweep(SWEEP_DOWN, p.nz_down);
  if (up0 < 0.0 || down0 < 0.0) return check_cuda(h, "autotune timing");
  double best_up = up0, best_down = down0;
  int nz = p.nz, nzd = p.nz_down, timed = 2;
  for (int c : nz_candidates(nc - 1, 1)) {
    const double u = sweep(SWEEP_UPE, c);
    timed += 1;
    if (u > 0.0 && u < best_up) best_up = u, nz = c;
  }
  for (int c : nz_candidates(3 * nc - 1, 3)) {
    const double d = sweep(SWEEP_DOWN, c);
    timed += 1;
    if (d > 0.0 && d < best_down) best_down = d, nzd = c;
  }
  if (best_up > 0.98 * up0) nz = p.nz, best_up = up0;
  if (best_down > 0.98 * down0) nzd = p.nz_down, best_down = down0;
  h->sw.nz = nz;
  h->sw.nz_down = nzd;
  t->path = 1;
  t->sweep_nz = nz;
  t->sweep_nz_down = nzd;
  t->candidates = timed;
  t->us_default = up0 + down0;
  t->us_tuned = best_up + best_down;
  return check_cuda(h, "autotune");
}

void apply_tuning(adafac_handle h, const adafac_tuning& t) {
  if (t.path == 1) {
    h->sw.nz = t.sweep_nz;
    h->sw.nz_down = t.sweep_nz_down;
  } else if (t.path == 2) {
    h->res_shape.bx = t.res_bx;
    h->res_shape.by = t.res_by;
    h->res_shape.zr = t.res_zr;
    h->upd_shape.bx = t.upd_bx;
    h->upd_shape.by = t.upd_by;
  }
}

}  // namespace

extern "C" {

adafac_status adafac_default_options(adafac_options* o) {
  if (!o) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null options");
  o->variant = ADAFAC_VARIANT_JAC;
  o->transfer = ADAFAC_TRANSFER_DLINEAR;
  o->precision = ADAFAC_PRECISION_FP64;
  o->rtilde = ADAFAC_RTILDE_TRUNCATED;
  o->form = ADAFAC_FORM_CS;
  o->inner_cycles = 24;
  o->omega = 0.6;
  o->omega_tilde = 0.6;
  o->omega_exp = 0.5;
  o->path = ADAFAC_PATH_AUTO;
  o->coarse_op = ADAFAC_COARSE_GALERKIN;
  o->lmin = 1;
  return ADAFAC_OK;
}

adafac_status adafac_workspace_size(const adafac_tree* tree, const adafac_options* opt,
                                    size_t* bytes) {
  std::string why;
  if (!tree || !opt || !bytes) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null argument");
  if (!valid_tree(tree, &why) || !valid_options(opt, &why))
    return fail(nullptr, ADAFAC_ERR_INVALID_ARG, why);
  // the size depends on whether eps is scalar: report the larger of both
  size_t most = 0;
  for (int scalar = 0; scalar <= 1; ++scalar) {
    adafac_handle_s tmp;
    tmp.D = tree->dim;
    tmp.L = tree->depth;
    tmp.opt = *opt;
    tmp.eps_scalar = scalar;
    tmp.uniform = scalar && opt->transfer == ADAFAC_TRANSFER_DLINEAR;
    tmp.fast3 = fast3_eligible(&tmp);
    tmp.batched = batched_choice(&tmp);
    Carver cv;
    carve(&tmp, cv);
    // lay the arrays out once more against a fake, never dereferenced base:
    // both passes must agree, or the size reported here would be wrong
    Carver check;
    check.base = reinterpret_cast<char*>(256);
    carve(&tmp, check);
    if (check.off != cv.off)
      return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "internal error: workspace layout mismatch");
    most = cv.off > most ? cv.off : most;
  }
  *bytes = most + 256;
  return ADAFAC_OK;
}

adafac_status adafac_setup(const adafac_tree* tree, const double* eps, int eps_is_scalar,
                           const double* f, int inputs_on_device, const adafac_options* opt,
                           void* workspace, size_t workspace_bytes, void* stream,
                           adafac_handle* out) {
  std::string why;
  if (!out) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  if (!tree || !opt || !eps) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null argument");
  if (!valid_tree(tree, &why) || !valid_options(opt, &why))
    return fail(nullptr, ADAFAC_ERR_INVALID_ARG, why);
  if (opt->lmin > tree->depth)
    return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "lmin must not exceed the depth");
  adafac_handle h = new (std::nothrow) adafac_handle_s();
  if (!h) return fail(nullptr, ADAFAC_ERR_OOM, "host allocation failed");
  h->D = tree->dim;
  h->L = tree->depth;
  h->opt = *opt;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->eps_scalar = eps_is_scalar ? 1 : 0;
  if (eps_is_scalar) {
    if (inputs_on_device) {
      if (cudaMemcpy(&h->eps0, eps, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        delete h;
        return fail(nullptr, ADAFAC_ERR_CUDA, "copy scalar eps");
      }
    } else {
      h->eps0 = eps[0];
    }
    if (!(h->eps0 > 0.0) || !std::isfinite(h->eps0)) {
      delete h;
      return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "eps must be positive and finite");
    }
  } else if (!inputs_on_device) {
    const long long nc = ipow_ll(ipow_ll(3, h->L), h->D);
    for (long long i = 0; i < nc; ++i)
      if (!(eps[i] > 0.0) || !std::isfinite(eps[i])) {
        delete h;
        return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "eps must be positive and finite");
      }
  }
  h->uniform = h->eps_scalar && opt->transfer == ADAFAC_TRANSFER_DLINEAR;
  h->fast3 = fast3_eligible(h);
  h->batched = batched_choice(h);
  Carver measure;
  carve(h, measure);
  const size_t need = measure.off + 256;
  if (workspace) {
    if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
      delete h;
      return fail(nullptr, ADAFAC_ERR_OOM,
                  "workspace too small or not 256-byte aligned: need " + std::to_string(need));
    }
    h->ws = static_cast<char*>(workspace);
    h->ws_bytes = workspace_bytes;
  } else {
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail(nullptr, ADAFAC_ERR_OOM, "cudaMalloc of " + std::to_string(need) + " bytes failed");
    }
    h->ws = static_cast<char*>(p);
    h->ws_bytes = need;
    h->own_ws = true;
  }
  Carver cv;
  cv.base = h->ws;
  carve(h, cv);
  if (cv.off != measure.off) {
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "internal error: workspace layout mismatch");
  }
  // FP64 levels need zeroed vectors (boundary rings stay zero)
  cudaMemsetAsync(h->ws, 0, need - 256, h->stream);
  adafac_status st = h->D == 2 ? run_setup<2>(h, eps, f, inputs_on_device)
                               : run_setup<3>(h, eps, f, inputs_on_device);
  if (st != ADAFAC_OK) {
    g_setup_error = h->err;
    // the memset and setup kernels may still run on the stream: a caller-owned
    // workspace (a server's pool range) must not be handed on before they end
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return st;
  }
  h->launches = 0;
  *out = h;
  return ADAFAC_OK;
}

adafac_status adafac_cycle(adafac_handle h, int n_cycles) {
  if (!h) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null handle");
  if (n_cycles < 0) return fail(h, ADAFAC_ERR_INVALID_ARG, "n_cycles must be >= 0");
  if (h->D == 2) enqueue_cycles<2>(h, n_cycles);
  else enqueue_cycles<3>(h, n_cycles);
  return check_cuda(h, "cycle");
}

adafac_status adafac_solve(adafac_handle h, double rel_tol, int max_cycles, int* cycles_done,
                           double* rel) {
  if (!h) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null handle");
  if (!(rel_tol >= 0.0) || max_cycles < 0)
    return fail(h, ADAFAC_ERR_INVALID_ARG, "rel_tol must be >= 0 and max_cycles >= 0");
  Control c;
  adafac_status st = read_ctl(h, &c);
  if (st != ADAFAC_OK) return st;
  const int applied0 = c.applied;
  int zero = 0;
  if ((st = write_ctl_field(h, offsetof(Control, done), zero)) != ADAFAC_OK) return st;
  if ((st = write_ctl_field(h, offsetof(Control, tol), rel_tol)) != ADAFAC_OK) return st;
  const bool mixed = h->opt.precision == ADAFAC_PRECISION_MIXED;
  const int batch = mixed ? h->opt.inner_cycles : 8;
  int enq = 0;
  bool done = false, diverged = false, evaluated = false;
  if (mixed && !h->batched) {
    // residual first, then [cycles, u += e, residual] per step: the host
    // reads each step's norm before it enqueues the next step
    if (h->D == 2) enqueue_refine_only<2>(h);
    else enqueue_refine_only<3>(h);
    if ((st = read_ctl(h, &c)) != ADAFAC_OK) return st;
    done = c.done != 0;
    diverged = c.diverged != 0;
    while (!done && !diverged && enq < max_cycles) {
      const int k = max_cycles - enq < batch ? max_cycles - enq : batch;
      if (h->D == 2) enqueue_solve_group<2>(h, k);
      else enqueue_solve_group<3>(h, k);
      enq += k;
      if ((st = read_ctl(h, &c)) != ADAFAC_OK) return st;
      done = c.done != 0;
      diverged = c.diverged != 0;
    }
    // the last group ended with the residual of the final iterate
    if (!done && !diverged) done = c.rel <= rel_tol;
    evaluated = true;
    enq = max_cycles;  // nothing below runs again
  }
  while (enq < max_cycles) {
    const int k = max_cycles - enq < batch ? max_cycles - enq : batch;
    if (h->D == 2) enqueue_cycles<2>(h, k);
    else enqueue_cycles<3>(h, k);
    enq += k;
    if ((st = read_ctl(h, &c)) != ADAFAC_OK) return st;
    done = c.done != 0;
    diverged = c.diverged != 0;
    if (done || diverged) break;
  }
  if (!done && !diverged && !evaluated) {
    // residual of the final iterate, recorded like a cycle evaluation
    if (h->batched) {
      batch_step(h, 0);
    } else if (mixed) {
      if (h->D == 2) refine_residual<2>(h);
      else refine_residual<3>(h);
    } else {
      // an FP64 cycle starts with the residual; evaluate it without updating
      if (h->D == 2) enqueue_query<2>(h);
      else enqueue_query<3>(h);
    }
    if ((st = read_ctl(h, &c)) != ADAFAC_OK) return st;
    if (!mixed) c.rel = c.qrel;
    done = c.rel <= rel_tol || c.done;
  }
  const double reached = c.rel;
  double minus = -1.0;
  if ((st = write_ctl_field(h, offsetof(Control, tol), minus)) != ADAFAC_OK) return st;
  if ((st = write_ctl_field(h, offsetof(Control, done), zero)) != ADAFAC_OK) return st;
  if (cycles_done) *cycles_done = c.applied - applied0;
  if (rel) *rel = reached;
  if (diverged) return fail(h, ADAFAC_ERR_DIVERGED, "residual diverged");
  if (!done) return fail(h, ADAFAC_ERR_NOT_CONVERGED, "max_cycles reached before rel_tol");
  return ADAFAC_OK;
}

adafac_status adafac_residual_norm(adafac_handle h, double* rel, double* abs) {
  if (!h) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null handle");
  if (h->D == 2) enqueue_query<2>(h);
  else enqueue_query<3>(h);
  Control c;
  adafac_status st = read_ctl(h, &c);
  if (st != ADAFAC_OK) return st;
  if (rel) *rel = c.qrel;
  if (abs) *abs = std::sqrt(c.qsq);
  return ADAFAC_OK;
}

adafac_status adafac_solution(adafac_handle h, double* dst, int dst_on_device) {
  if (!h || !dst) return fail(h, ADAFAC_ERR_INVALID_ARG, "null argument");
  const size_t bytes = sizeof(double) * h->lev[h->L].V;
  if (cudaMemcpyAsync(dst, h->u, bytes,
                      dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      h->stream) != cudaSuccess)
    return check_cuda(h, "copy solution");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "synchronise");
  return check_cuda(h, "solution");
}

adafac_status adafac_set_solution(adafac_handle h, const double* src, int src_on_device) {
  if (!h || !src) return fail(h, ADAFAC_ERR_INVALID_ARG, "null argument");
  const size_t bytes = sizeof(double) * h->lev[h->L].V;
  if (cudaMemcpyAsync(h->u, src, bytes,
                      src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess)
    return check_cuda(h, "copy iterate");
  k_boundary<<<1024, 256, 0, h->stream>>>(h->u, h->ub, h->lev[h->L].n, h->D, 0);
  adafac_status st = reset_control(h);
  // the exponent of the new iterate (the scale of the fixed-point residual)
  if (st == ADAFAC_OK && h->fast3)
    launch_max_exponent(h->u, h->lev[h->L].V, &h->ctl->uexp, nullptr, h->stream);
  return st == ADAFAC_OK ? check_cuda(h, "iterate exponent") : st;
}

adafac_status adafac_set_boundary(adafac_handle h, const double* g, int g_on_device) {
  if (!h || !g) return fail(h, ADAFAC_ERR_INVALID_ARG, "null argument");
  if (h->opt.form == ADAFAC_FORM_FAS)
    return fail(h, ADAFAC_ERR_INVALID_ARG,
                "non-zero Dirichlet values need the correction-scheme form");
  const size_t bytes = sizeof(double) * h->lev[h->L].V;
  if (cudaMemcpyAsync(h->ub, g, bytes,
                      g_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess)
    return check_cuda(h, "copy boundary values");
  const int n = h->lev[h->L].n;
  k_boundary<<<1024, 256, 0, h->stream>>>(h->ub, nullptr, n, h->D, 1);
  k_boundary<<<1024, 256, 0, h->stream>>>(h->u, h->ub, n, h->D, 0);
  // the exponents of the Dirichlet values and of the iterate
  cudaMemsetAsync(&h->ctl->bdexp, 0, sizeof(int), h->stream);
  launch_max_exponent(h->ub, h->lev[h->L].V, &h->ctl->bdexp, nullptr, h->stream);
  adafac_status st = reset_control(h);
  if (st == ADAFAC_OK && h->fast3)
    launch_max_exponent(h->u, h->lev[h->L].V, &h->ctl->uexp, nullptr, h->stream);
  return st == ADAFAC_OK ? check_cuda(h, "iterate exponent") : st;
}

adafac_status adafac_reset(adafac_handle h) {
  if (!h) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null handle");
  // u = 0 inside, the Dirichlet values on the boundary
  cudaMemcpyAsync(h->u, h->ub, sizeof(double) * h->lev[h->L].V, cudaMemcpyDeviceToDevice,
                  h->stream);
  return reset_control(h);
}

adafac_status adafac_get_field(adafac_handle h, int field, int level, double* dst,
                               int dst_on_device, size_t* count) {
  if (!h || !count) return fail(h, ADAFAC_ERR_INVALID_ARG, "null argument");
  if (level < 1 || level > h->L) return fail(h, ADAFAC_ERR_INVALID_ARG, "level out of range");
  LevelData& lv = h->lev[level];
  const bool mixed = h->opt.precision == ADAFAC_PRECISION_MIXED;
  const int NC = 1 << h->D, NS = h->D == 2 ? 9 : 27;
  const double* src64 = nullptr;
  const float* src32 = nullptr;
  long long n = lv.V;
  switch (field) {
    case ADAFAC_FIELD_U:
      if (level != h->L) return fail(h, ADAFAC_ERR_INVALID_ARG, "U lives on the finest level");
      src64 = h->u;
      break;
    case ADAFAC_FIELD_B:
      if (level != h->L) return fail(h, ADAFAC_ERR_INVALID_ARG, "B lives on the finest level");
      src64 = h->b;
      break;
    case ADAFAC_FIELD_R:
      if (mixed) src32 = lv.r32;
      else src64 = lv.r;
      break;
    case ADAFAC_FIELD_BT:
      if (level == h->L) return fail(h, ADAFAC_ERR_INVALID_ARG, "BT lives on levels < L");
      if (mixed) src32 = lv.bt32;
      else src64 = lv.bt;
      break;
    case ADAFAC_FIELD_G:
      if (level == h->L) return fail(h, ADAFAC_ERR_INVALID_ARG, "G lives on levels < L");
      if (mixed) src32 = lv.g32;
      else src64 = lv.g;
      break;
    case ADAFAC_FIELD_T:
      if (level == h->L) return fail(h, ADAFAC_ERR_INVALID_ARG, "T lives on levels < L");
      if (mixed) src32 = level == h->opt.lmin ? lv.g32 : lv.t32;
      else src64 = level == h->opt.lmin ? lv.g : lv.t;
      break;
    case ADAFAC_FIELD_P:
      if (!lv.P) return fail(h, ADAFAC_ERR_INVALID_ARG, "P is stored for BoxMG levels >= 2 only");
      src64 = lv.P;
      n = NC * lv.V;
      break;
    case ADAFAC_FIELD_STENCIL:
      if (!lv.st) return fail(h, ADAFAC_ERR_INVALID_ARG, "stencil is stored for non-uniform levels < L only");
      src64 = lv.st;
      n = NS * lv.V;
      break;
    case ADAFAC_FIELD_INVDIAG:
      src64 = lv.invd;
      break;
    default:
      return fail(h, ADAFAC_ERR_INVALID_ARG, "unknown field");
  }
  *count = (size_t)n;
  if (!dst) return ADAFAC_OK;
  if (!src64 && !src32) return fail(h, ADAFAC_ERR_INVALID_ARG, "field not allocated in this mode");
  if (src64) {
    if (cudaMemcpyAsync(dst, src64, sizeof(double) * n,
                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
      return check_cuda(h, "copy field");
  } else {
    std::vector<float> tmp((size_t)n);
    if (cudaMemcpyAsync(tmp.data(), src32, sizeof(float) * n, cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
      return check_cuda(h, "copy field");
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "synchronise");
    std::vector<double> wide(tmp.begin(), tmp.end());
    if (cudaMemcpy(dst, wide.data(), sizeof(double) * n,
                   dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost) != cudaSuccess)
      return check_cuda(h, "copy field");
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "synchronise");
  return check_cuda(h, "get_field");
}

adafac_status adafac_history(adafac_handle h, double* dst, int max_entries, int* count) {
  if (!h || !count) return fail(h, ADAFAC_ERR_INVALID_ARG, "null argument");
  Control c;
  adafac_status st = read_ctl(h, &c);
  if (st != ADAFAC_OK) return st;
  const int avail = c.nhist < kHistCap ? c.nhist : kHistCap;
  *count = avail;
  if (dst && max_entries > 0) {
    const int m = avail < max_entries ? avail : max_entries;
    if (cudaMemcpy(dst, h->hist, sizeof(double) * m, cudaMemcpyDeviceToHost) != cudaSuccess)
      return check_cuda(h, "copy history");
  }
  return ADAFAC_OK;
}

adafac_status adafac_set_wait_limit(adafac_handle h, long long polls) {
  if (!h) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null handle");
  if (polls < 0) return fail(h, ADAFAC_ERR_INVALID_ARG, "polls must be >= 0");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "synchronise");
  h->sw.wait_polls = polls;
  // captured batches hold the sweeps' parameters by value: capture again
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
  return ADAFAC_OK;
}

adafac_status adafac_set_batch_cluster(adafac_handle h, int ctas) {
  if (!h) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null handle");
  if (!h->batched) return fail(h, ADAFAC_ERR_INVALID_ARG, "handle does not run the batched path");
  if (ctas < 1 || (ctas & (ctas - 1)) || ctas > batch_max_cluster())
    return fail(h, ADAFAC_ERR_INVALID_ARG,
                "ctas must be a power of two in 1.." + std::to_string(batch_max_cluster()));
  h->bC = ctas;
  return ADAFAC_OK;
}

adafac_status adafac_batch_cluster(adafac_handle h, int* ctas) {
  if (!h || !ctas) return fail(h, ADAFAC_ERR_INVALID_ARG, "null argument");
  if (!h->batched) return fail(h, ADAFAC_ERR_INVALID_ARG, "handle does not run the batched path");
  *ctas = h->bC;
  return ADAFAC_OK;
}

adafac_status adafac_launch_count(adafac_handle h, uint64_t* count) {
  if (!h || !count) return fail(h, ADAFAC_ERR_INVALID_ARG, "null argument");
  *count = h->launches;
  return ADAFAC_OK;
}

adafac_status adafac_timing(adafac_handle h, int enable) {
  if (!h) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null handle");
  if (enable) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "synchronise");
    for (auto& m : h->marks) m.clear();
    h->ev_used = 0;
  }
  h->timing = enable != 0;
  return ADAFAC_OK;
}

adafac_status adafac_timing_read(adafac_handle h, int kind, double* total_ms, int* launches) {
  if (!h) return fail(nullptr, ADAFAC_ERR_INVALID_ARG, "null handle");
  if (kind < 0 || kind >= ADAFAC_KERNEL_KINDS)
    return fail(h, ADAFAC_ERR_INVALID_ARG, "kernel kind out of range");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "synchronise");
  double sum = 0.0;
  for (auto& pr : h->marks[kind]) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess)
      return check_cuda(h, "event time");
    sum += ms;
  }
  if (total_ms) *total_ms = sum;
  if (launches) *launches = (int)h->marks[kind].size();
  return ADAFAC_OK;
}

const char* adafac_last_error(adafac_handle h) {
  return h ? h->err.c_str() : g_setup_error.c_str();
}

adafac_status adafac_autotune(adafac_handle h, int repeats, adafac_tuning* out) {
  if (!h || !out) return fail(h, ADAFAC_ERR_INVALID_ARG, "null argument");
  if (repeats < 1 || repeats > 1000) return fail(h, ADAFAC_ERR_INVALID_ARG, "repeats must be in 1..1000");
  *out = adafac_tuning();
  const bool mixed = h->opt.precision == ADAFAC_PRECISION_MIXED;
  const bool level = mixed && !h->fast3 && !h->batched && h->opt.path != ADAFAC_PATH_GENERIC;
  if (!h->fast3 && !level) return ADAFAC_OK;  // nothing tunable: path 0
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_cuda(h, "autotune device");
  const TuneKey key{dev, h->D, h->L, h->fast3 ? 1 : 0, h->lev[h->L].v32.opkind,
                    h->opt.transfer, h->opt.variant, h->opt.lmin};
  {
    std::lock_guard<std::mutex> g(g_tune_lock);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *out = it->second;
      out->cached = 1;
      apply_tuning(h, *out);
      for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
      h->graphs.clear();
      return ADAFAC_OK;
    }
  }
  // the timed kernels must run: clear the converged / diverged flags first
  adafac_status st = reset_control(h);
  if (st != ADAFAC_OK) return st;
  if (h->fast3) st = tune_fast3(h, repeats, out);
  else st = h->D == 2 ? tune_level<2>(h, repeats, out) : tune_level<3>(h, repeats, out);
  if (st != ADAFAC_OK) return st;
  // graphs captured with the old shapes are dropped; the timed launches wrote
  // the correction buffers and counted cycles: start the cycle state afresh
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
  st = reset_control(h);
  if (st != ADAFAC_OK) return st;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return check_cuda(h, "autotune");
  std::lock_guard<std::mutex> g(g_tune_lock);
  g_tune_cache[key] = *out;
  return ADAFAC_OK;
}

adafac_status adafac_destroy(adafac_handle h) {
  if (!h) return ADAFAC_OK;
  cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->own_ws) cudaFree(h->ws);
  delete h;
  return ADAFAC_OK;
}

}  // extern "C"
