// C ABI of the hierarchical multicontinuum cell-problem solver (declared in include/mch.h).
//
// Per level n (Algorithm 1, lines 4-6) mch_solve_level enqueues on the handle's stream:
//   setup     per point: targets G, centroids, S = Ct M^-1 Ct^T and S^-1 (FP64)
//   [n > 1]   I = sum_t c_t Phi_t on the level-1 grid (Eq. phiXiI_all), y = A_1 I with the
//             child's medium prolonged (FP64), K_I = I^T A_1 I, b = -P^T y and
//             g = G - C_1 I (Eqs. phi_avar_corrector, phi_grad_corrector)
//   solve     FP64 refinement step, then up to max_refine x (PCG sweep + refinement step)
//   E         |Y| E = K_I + 1/2 (Xi^T (A_n Xi - 2 b) + (A_n Xi - 2 b)^T Xi)   (Eq. Bs_defi)
//   Phi       Phi = I + P Xi on the level-1 grid (Eq. PhiXiI)
// and synchronises the stream once to read the per-unit convergence record.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mch.h"
#include "common.cuh"
#include "k3d.cuh"
#include "kernels.h"
#include "plan.h"

using namespace mch;

namespace {

struct Level {
  LevelPlan plan;
  int n = 0, rho = 1, npts = 0, nv = 0, nvf = 0;
  double *kappa = nullptr;
  uint8_t *labels = nullptr;
  double *G = nullptr, *gI = nullptr, *Sinv64 = nullptr, *Sacc = nullptr, *bacc = nullptr;
  float *Sinv32 = nullptr;
  float *kap32 = nullptr, *minv32 = nullptr;  // 3D mixed precision: FP32 copies
  double *kapff = nullptr;   // 2D mixed, levels > 1: float-float planes of kappa
  double *x = nullptr, *b = nullptr, *minv = nullptr;
  double *ratio = nullptr;
  int *iters = nullptr, *sweeps = nullptr, *ustat = nullptr, *pstat = nullptr, *dropped = nullptr;
  double *E = nullptr, *phi = nullptr;
  const double **par_ptr = nullptr;
  double *par_w = nullptr;
  double *lam = nullptr;          // [pt][R][nc] final multipliers of the forward solve
  double *V = nullptr;            // [pt][R][nvf] backward seeds (levels with children)
  double **par_V = nullptr;       // [pt][slots] parents' seed blocks (levels > 1)
  bool solved = false;
  bool partial = false;           // solved by mch_solve_level_range for a part of its points
  // mch_prepare_level: staged inputs and constraint data computed on the side stream
  bool prepared = false;
  const double *prep_kappa = nullptr;
  const uint8_t *prep_labels = nullptr;
  cudaEvent_t prep_ev = nullptr;
  int prep_launches = 0;
  long long prep_h2d = 0;
  int variant = 0;                // launch shape of the 2D mixed level solve
  mch_level_stats stats{};
};

}  // namespace

struct mch_handle {
  mch_desc d{};
  std::vector<int> strides;
  cudaStream_t st = nullptr;
  cudaStream_t st2 = nullptr;     // side stream of mch_prepare_level
  cudaEvent_t ev_main = nullptr;
  int R = 0, nc = 0, nq = 0, slots = 0;
  std::vector<Level> lv;
  // scratch shared by the levels (solved one after another)
  double *yfine = nullptr, *yc = nullptr;
  size_t yfine_cap = 0;           // doubles in yfine
  double *bnorm = nullptr;  // [unit] b'M^-1 b of the current correction or adjoint problem
  // oversampling (o > 0): A_1 I with kappa masked to R_p (level-1 grid), P^T of it (level
  // grid), and the masked level kappa
  double *yfineR = nullptr, *cR = nullptr, *kapR = nullptr;
  // 2D mixed precision: level-1-grid vectors (cell functions, A_1 I) are float-float planes
  bool ffs = false;
  // 3D level-solve scratch: inner vectors, FP64 residual, rotating accumulators, counters
  void *s3p = nullptr, *s3r = nullptr, *s3d = nullptr, *s3q = nullptr;
  double *s3r64 = nullptr, *s3acc = nullptr;
  int *s3cnt = nullptr;
  size_t s3_units_nv = 0, s3_acc = 0;
  // backward-pass buffers, allocated on the first mch_backward
  bool bw_ready = false;
  bool phi_released = false;  // keep_parents = 0: level-1-grid cell functions freed
  double *psi1 = nullptr, *psi2 = nullptr, *lamadj = nullptr, *gzero = nullptr, *Wd = nullptr,
         *dk = nullptr, *bw_ratio = nullptr;
  int *bw_iters = nullptr, *bw_sweeps = nullptr, *bw_status = nullptr;
  std::vector<void *> allocs;
  std::string err;
  long long h2d = 0, d2h = 0;
  int launches = 0;
  bool timing = false;
  cudaEvent_t ev[32] = {};
  int n_ev = 0;
};

namespace {

mch_status set_err(mch_handle *h, mch_status s, const std::string &msg) {
  if (h) h->err = msg;
  return s;
}

mch_status cuda_fail(mch_handle *h, cudaError_t e, const char *where) {
  return set_err(h, e == cudaErrorMemoryAllocation ? MCH_ERR_OOM : MCH_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

template <typename T>
cudaError_t dalloc(mch_handle *h, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(q, 0, count * sizeof(T) + 16, h->st);
  h->allocs.push_back(q);
  *p = reinterpret_cast<T *>(q);
  return e;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copies `bytes` between caller memory and library device memory in the given direction,
// counting host traffic.
cudaError_t stage(mch_handle *h, void *dst, const void *src, size_t bytes, bool to_device,
                  cudaStream_t on = nullptr) {
  if (to_device) {
    const bool dev = is_device_ptr(src);
    if (!dev) h->h2d += (long long)bytes;
    return cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           on ? on : h->st);
  }
  const bool dev = is_device_ptr(dst);
  if (!dev) h->d2h += (long long)bytes;
  return cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         h->st);
}

int ilog2(int v) {
  int r = 0;
  while ((1 << (r + 1)) <= v) ++r;
  return r;
}

int nvd(int dim, int n) { return dim == 3 ? nv3_of(n) : nv_of(n); }
size_t elems(int dim, int n) { return dim == 3 ? (size_t)n * n * n : (size_t)n * n; }

bool level3d_supported(int n, int P) {
  const int m = P > 0 ? n / P : 0;
  return n >= 4 && P >= 1 && n % P == 0 && m >= 2 && (m & (m - 1)) == 0 && (n & (n - 1)) == 0;
}

bool valid_level(const mch_handle *h, int level) {
  return h && level >= 1 && level <= (int)h->lv.size();
}

void dfree(mch_handle *h, void *p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i] == p) {
      h->allocs.erase(h->allocs.begin() + i);
      break;
    }
  cudaFree(p);
}

double rho_pow(const mch_handle *h, int rho) {
  return h->d.dim == 3 ? (double)rho * rho * rho : (double)rho * rho;
}

// Interpolation and correction data of a child level on the level-1 grid (Phi = I, A_1 I,
// g -= C_1 I); g holds the targets on entry. Returns the number of kernels launched via
// *nl.
cudaError_t launch_child(mch_handle *h, Level &L, double *g, int *nl = nullptr) {
  const mch_desc &d = h->d;
  ChildArgs ca{L.npts, h->R, d.n_fine, ilog2(L.rho), L.nvf, h->slots, ilog2(d.n_fine / d.periods),
               d.periods, d.n_cont, h->nc, L.par_ptr, L.par_w, L.kappa, L.labels, L.phi,
               h->yfine, g, 1.0 / rho_pow(h, L.rho), h->yfineR, d.overs, L.kapff};
  if (d.dim == 2) {
    if (nl) *nl = 1;
    return launch_child_fine2d(ca, h->ffs, h->st);
  }
  if (nl) *nl = 2;
  cudaError_t e = launch_interp3d(ca, h->st, h->ffs);
  if (e != cudaSuccess) return e;
  return launch_fine_apply3d(ca, d.rve_len / d.n_fine, h->st, h->ffs);
}

cudaError_t launch_prolong(mch_handle *h, Level &L) {
  if (h->d.dim == 2)
    return launch_prolong_add2d(L.npts, h->R, h->d.n_fine, L.rho, L.x, L.nv, L.phi, L.nvf, h->st,
                                h->ffs);
  return launch_prolong_add3d(L.npts, h->R, h->d.n_fine, L.rho, L.x, L.nv, L.phi, L.nvf, h->st,
                              h->ffs);
}

// yf is a level-1-grid vector in the handle's storage (ffs) or, for the backward seeds, FP64
cudaError_t launch_restrict(mch_handle *h, Level &L, const double *yf, double scale, double *out,
                            bool ffs) {
  if (h->d.dim == 2)
    return launch_restrict2d(L.npts, h->R, h->d.n_fine, L.rho, yf, L.nvf, scale, out, L.nv, h->st,
                             ffs);
  return launch_restrict3d(L.npts, h->R, h->d.n_fine, L.rho, yf, L.nvf, scale, out, L.nv, h->st,
                           ffs);
}

// grows the 3D level-solve scratch to `units_nv` node entries per vector and `acc` doubles
cudaError_t ensure_s3(mch_handle *h, size_t units_nv, size_t acc) {
  const size_t tsz = h->d.precision == MCH_FP64 ? sizeof(double) : sizeof(float);
  if (units_nv > h->s3_units_nv) {
    for (void **p : {&h->s3p, &h->s3r, &h->s3d, &h->s3q}) {
      dfree(h, *p);
      *p = nullptr;
      unsigned char *q = nullptr;
      cudaError_t e = dalloc(h, &q, units_nv * tsz);
      if (e != cudaSuccess) return e;
      *p = q;
    }
    dfree(h, h->s3r64);
    h->s3r64 = nullptr;
    cudaError_t e = dalloc(h, &h->s3r64, units_nv);
    if (e != cudaSuccess) return e;
    h->s3_units_nv = units_nv;
  }
  if (acc > h->s3_acc) {
    dfree(h, h->s3acc);
    h->s3acc = nullptr;
    cudaError_t e = dalloc(h, &h->s3acc, acc);
    if (e != cudaSuccess) return e;
    h->s3_acc = acc;
  }
  if (!h->s3cnt) return dalloc(h, &h->s3cnt, 4);
  return cudaSuccess;
}

// 3D constrained solves of a level (one cooperative launch); x is overwritten.
cudaError_t solve3d(mch_handle *h, Level &L, const double *g, const double *b, double *x,
                    int *iters, int *sweeps, double *ratio, int *ustat, double *lam,
                    const double *bnorm) {
  const mch_desc &d = h->d;
  const int R = h->R, nc = h->nc;
  const size_t units = (size_t)L.npts * R, un = units * L.nv;
  const size_t acc = 3 * units * (8 + 2 * (size_t)nc);
  const bool fp64 = d.precision == MCH_FP64;
  const size_t tsz = fp64 ? sizeof(double) : sizeof(float);
  cudaError_t e = ensure_s3(h, un, acc);
  if (e != cudaSuccess) return e;
  cudaStream_t st = h->st;
  if ((e = cudaMemsetAsync(x, 0, un * sizeof(double), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(h->s3d, 0, un * tsz, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(h->s3p, 0, un * tsz, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(h->s3acc, 0, acc * sizeof(double), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(h->s3cnt, 0, 4 * sizeof(int), st)) != cudaSuccess) return e;
  const int max_iter = d.max_iter > 0 ? d.max_iter : 4 * L.n + 50;
  const double hn = d.rve_len / L.n;
  if (fp64) {
    Level3Args<double> a{L.npts, R, L.n, d.periods, d.n_cont, nc, L.nv, L.n / d.periods,
                         L.kappa, L.kappa, L.labels, L.Sinv64, L.Sinv64, L.minv, L.minv, g, b, x,
                         h->s3r64, (double *)h->s3p, (double *)h->s3r, (double *)h->s3d,
                         (double *)h->s3q, h->s3acc, h->s3cnt, iters, sweeps, ratio, ustat,
                         (float)d.inner_tol, max_iter, d.rtol, d.max_refine, lam, hn, 0, 0,
                         bnorm};
    return launch_level3d<double>(a, st);
  }
  Level3Args<float> a{L.npts, R, L.n, d.periods, d.n_cont, nc, L.nv, L.n / d.periods,
                      L.kappa, L.kap32, L.labels, L.Sinv32, L.Sinv64, L.minv, L.minv32, g, b, x,
                      h->s3r64, (float *)h->s3p, (float *)h->s3r, (float *)h->s3d,
                      (float *)h->s3q, h->s3acc, h->s3cnt, iters, sweeps, ratio, ustat,
                      (float)d.inner_tol, max_iter, d.rtol, d.max_refine, lam, hn, 0, 0,
                      bnorm};
  return launch_level3d<float>(a, st);
}

// keep_parents = 0: frees every level's cell functions on the level-1 grid.
cudaError_t release_phi(mch_handle *h) {
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return e;
  for (Level &L : h->lv) {
    dfree(h, L.phi);
    L.phi = nullptr;
  }
  h->phi_released = true;
  return cudaSuccess;
}

// Reallocates the cell functions and recomputes those of every solved level from its stored
// level-grid solution, levels in order (Phi = Xi at level 1, Phi = I + P Xi above): the
// same kernels as the forward pass, without a new solve.
cudaError_t restore_phi(mch_handle *h) {
  if (!h->phi_released) return cudaSuccess;
  const int R = h->R;
  for (Level &L : h->lv) {
    cudaError_t e = dalloc(h, &L.phi, (size_t)L.npts * R * L.nvf);
    if (e != cudaSuccess) return e;
  }
  for (size_t l = 1; l < h->lv.size(); ++l) {
    Level &L = h->lv[l];
    std::vector<const double *> hp((size_t)L.npts * h->slots, nullptr);
    for (size_t i = 0; i < hp.size(); ++i) {
      const int pl = L.plan.par_level[i];
      if (pl > 0) hp[i] = h->lv[pl - 1].phi + (size_t)L.plan.par_pos[i] * R * L.nvf;
    }
    cudaError_t e = cudaMemcpyAsync(const_cast<const double **>(L.par_ptr), hp.data(),
                                    hp.size() * sizeof(void *), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return e;
  }
  for (size_t l = 0; l < h->lv.size(); ++l) {
    Level &L = h->lv[l];
    if (!L.solved) continue;
    cudaError_t e;
    if (l == 0) {
      e = h->ffs ? launch_to_ff(L.npts * R, L.x, L.nv, L.phi, L.nvf, L.nv, h->st)
                 : cudaMemcpyAsync(L.phi, L.x, (size_t)L.npts * R * L.nv * sizeof(double),
                                   cudaMemcpyDeviceToDevice, h->st);
    } else {
      e = launch_child(h, L, L.gI);
      if (e == cudaSuccess) e = launch_prolong(h, L);
    }
    if (e != cudaSuccess) return e;
  }
  h->phi_released = false;
  return cudaStreamSynchronize(h->st);
}

// The points [p0, p1) of a level as a level of their own: every per-point array offset by p0
// (the plan's parent tables included), npts = p1 - p0. Flags stay with the real level.
Level range_view(const Level &L, int p0, int p1, int dim, int R, int nc, int slots) {
  Level V = L;
  const size_t o = (size_t)p0, ne = elems(dim, L.n);
  auto off = [&](auto *p, size_t per) { return p ? p + o * per : p; };
  V.npts = p1 - p0;
  V.kappa = off(L.kappa, ne);
  V.labels = off(L.labels, ne);
  V.G = off(L.G, (size_t)nc * R);
  V.gI = off(L.gI, (size_t)nc * R);
  V.Sinv64 = off(L.Sinv64, (size_t)nc * nc);
  V.Sacc = off(L.Sacc, (size_t)nc * nc);
  V.bacc = off(L.bacc, (size_t)nc * (dim + 1));
  V.Sinv32 = off(L.Sinv32, (size_t)nc * nc);
  V.kap32 = off(L.kap32, ne);
  V.minv32 = off(L.minv32, (size_t)L.nv);
  V.kapff = off(L.kapff, ne);
  V.x = off(L.x, (size_t)R * L.nv);
  V.b = off(L.b, (size_t)R * L.nv);
  V.minv = off(L.minv, (size_t)L.nv);
  V.ratio = off(L.ratio, (size_t)R);
  V.iters = off(L.iters, (size_t)R);
  V.sweeps = off(L.sweeps, (size_t)R);
  V.ustat = off(L.ustat, (size_t)R);
  V.pstat = off(L.pstat, 1);
  V.dropped = off(L.dropped, 1);
  V.E = off(L.E, (size_t)R * R);
  V.phi = off(L.phi, (size_t)R * L.nvf);
  V.par_ptr = off(L.par_ptr, (size_t)slots);
  V.par_w = off(L.par_w, (size_t)slots);
  V.lam = off(L.lam, (size_t)R * nc);
  V.V = off(L.V, (size_t)R * L.nvf);
  V.par_V = off(L.par_V, (size_t)slots);
  return V;
}

// Stages the level's kappa and labels and computes its constraint data on stream `on`;
// returns the number of kernels launched through *nl.
cudaError_t setup_level(mch_handle *h, Level &L, const double *kappa, const uint8_t *labels,
                        cudaStream_t on, int *nl) {
  const mch_desc &d = h->d;
  const size_t np = L.npts, ne = elems(d.dim, L.n);
  cudaError_t e = stage(h, L.kappa, kappa, np * ne * sizeof(double), true, on);
  if (e == cudaSuccess) e = stage(h, L.labels, labels, np * ne, true, on);
  if (e != cudaSuccess) return e;
  SetupArgs sa{(int)np, L.n, d.periods, d.n_cont, h->R, h->nc, d.rve_len / L.n, d.rve_len,
               L.kappa, L.labels, L.G, L.Sinv64, L.Sinv32, L.pstat, L.dropped, L.minv, L.nv,
               L.Sacc, L.bacc, L.kap32, L.minv32, d.overs};
  *nl = 2;
  return d.dim == 3 ? launch_setup3d(sa, on) : launch_setup2d(sa, on);
}

}  // namespace

extern "C" {

const char *mch_status_name(mch_status s) {
  switch (s) {
    case MCH_OK: return "MCH_OK";
    case MCH_ERR_ARG: return "MCH_ERR_ARG";
    case MCH_ERR_CUDA: return "MCH_ERR_CUDA";
    case MCH_ERR_OOM: return "MCH_ERR_OOM";
    case MCH_ERR_ORDER: return "MCH_ERR_ORDER";
    case MCH_ERR_NOT_CONVERGED: return "MCH_ERR_NOT_CONVERGED";
    case MCH_ERR_BREAKDOWN: return "MCH_ERR_BREAKDOWN";
    case MCH_ERR_DEGENERATE: return "MCH_ERR_DEGENERATE";
    case MCH_ERR_UNSUPPORTED: return "MCH_ERR_UNSUPPORTED";
  }
  return "MCH_UNKNOWN";
}

const char *mch_last_error(const mch_handle *h) { return h ? h->err.c_str() : "null handle"; }

void mch_destroy(mch_handle *h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  for (void *p : h->allocs) cudaFree(p);
  for (int i = 0; i < h->n_ev; ++i) cudaEventDestroy(h->ev[i]);
  for (Level &L : h->lv)
    if (L.prep_ev) cudaEventDestroy(L.prep_ev);
  if (h->ev_main) cudaEventDestroy(h->ev_main);
  if (h->st2) cudaStreamDestroy(h->st2);
  delete h;
}

mch_status mch_create(const mch_desc *desc, void *cuda_stream, mch_handle **out) {
  if (!out) return MCH_ERR_ARG;
  *out = nullptr;
  if (!desc) return MCH_ERR_ARG;
  const mch_desc &d = *desc;
  if ((d.dim != 2 && d.dim != 3) || d.n_cont < 1 || d.n_cont > MCH_MAX_CONT || d.n_levels < 1 || d.eta < 1 ||
      d.macro_n < 1 || !d.level_stride || d.n_fine < 4 || d.periods < 1 || !(d.rve_len > 0) ||
      (d.precision != MCH_FP64 && d.precision != MCH_MIXED) || d.rtol < 0 || d.inner_tol < 0 ||
      d.max_iter < 0 || d.max_refine < 0 || d.point_batch < 0)
    return MCH_ERR_ARG;
  // oversampling: at least one period in the integration region
  if (d.overs < 0 || d.periods - 2 * d.overs < 1) return MCH_ERR_ARG;
  const int nq = d.dim == 3 ? d.periods * d.periods * d.periods : d.periods * d.periods;
  const int nc = d.n_cont * nq;
  if (nc > (d.dim == 3 ? MCH_MAX_NC3 : MCH_MAX_NC)) return MCH_ERR_UNSUPPORTED;
  // 3D: the Gram and backward kernels take up to 12 cell functions (n_cont <= 3)
  if (d.dim == 3 && d.n_cont > 3) return MCH_ERR_UNSUPPORTED;

  mch_handle *h = new mch_handle();
  h->d = d;
  h->strides.assign(d.level_stride, d.level_stride + d.n_levels);
  h->d.level_stride = h->strides.data();
  if (h->d.rtol == 0) h->d.rtol = 1e-8;
  // default per-sweep reduction: 1e-5 in 2D (the Chebyshev-preconditioned on-chip sweeps
  // reach it and save a refinement step), 1e-4 in 3D (the streaming sweeps pay per iteration)
  if (h->d.inner_tol == 0) h->d.inner_tol = d.dim == 3 ? 1e-4 : 1e-5;
  if (h->d.max_refine == 0) h->d.max_refine = 6;
  h->st = (cudaStream_t)cuda_stream;
  h->R = d.n_cont * (1 + d.dim);
  h->nq = nq;
  h->nc = nc;
  h->ffs = d.precision == MCH_MIXED;
  h->slots = 1 << d.dim;

  std::vector<LevelPlan> plans;
  std::string perr;
  if (!build_plan(d.dim, d.macro_n, h->strides, d.n_fine, d.eta, plans, perr, d.interp)) {
    delete h;
    return MCH_ERR_ARG;
  }
  // every level grid must be a supported power of two divisible by the coarsening
  int scale = 1;
  for (int l = 0; l < d.n_levels; ++l) {
    if (d.n_fine % scale) { delete h; return MCH_ERR_ARG; }
    const int n = d.n_fine / scale;
    const bool ok = d.dim == 2 ? level2d_supported(n, d.periods, d.precision == MCH_FP64)
                               : level3d_supported(n, d.periods);
    if (!ok) {
      delete h;
      return MCH_ERR_UNSUPPORTED;
    }
    scale *= d.eta;
  }

  h->lv.resize(d.n_levels);
  size_t max_unit_nv = 0, max_fine = 0, max_unit_nvc = 0;
  const int nvf = nvd(d.dim, d.n_fine);
  for (int l = 0; l < d.n_levels; ++l) {
    Level &L = h->lv[l];
    L.plan = plans[l];
    L.n = L.plan.n_elem;
    L.rho = d.n_fine / L.n;
    L.npts = (int)L.plan.points.size() / d.dim;
    L.nv = nvd(d.dim, L.n);
    L.nvf = nvf;
    max_unit_nv = std::max(max_unit_nv, (size_t)L.npts * h->R * L.nv);
    max_unit_nvc = std::max(max_unit_nvc, (size_t)L.npts * h->R * L.nv);
    if (l > 0) max_fine = std::max(max_fine, (size_t)L.npts * h->R * nvf);
  }
#define ALLOC(ptr, cnt)                                   \
  do {                                                    \
    cudaError_t e_ = dalloc(h, &(ptr), (size_t)(cnt));    \
    if (e_ != cudaSuccess) {                              \
      mch_destroy(h);                                     \
      return e_ == cudaErrorMemoryAllocation ? MCH_ERR_OOM : MCH_ERR_CUDA; \
    }                                                     \
  } while (0)
  for (int l = 0; l < d.n_levels; ++l) {
    Level &L = h->lv[l];
    const size_t np = L.npts, R = h->R, ne = elems(d.dim, L.n);
    ALLOC(L.kappa, np * ne);
    ALLOC(L.labels, np * ne);
    ALLOC(L.G, np * nc * R);
    ALLOC(L.gI, np * nc * R);
    ALLOC(L.Sinv64, np * nc * nc);
    ALLOC(L.Sacc, np * nc * nc);
    ALLOC(L.bacc, np * nc * (d.dim + 1));
    if (d.precision == MCH_MIXED) ALLOC(L.Sinv32, np * nc * nc);
    if (d.dim == 3 && d.precision == MCH_MIXED) {
      ALLOC(L.kap32, np * ne);
      ALLOC(L.minv32, np * L.nv);
    }
    if (d.precision == MCH_MIXED && l > 0) ALLOC(L.kapff, np * ne);
    ALLOC(L.x, np * R * L.nv);
    ALLOC(L.minv, np * L.nv);
    ALLOC(L.b, np * R * L.nv);
    ALLOC(L.lam, np * R * nc);
    ALLOC(L.ratio, np * R);
    ALLOC(L.sweeps, np * R);
    ALLOC(L.iters, np * R);
    ALLOC(L.ustat, np * R);
    ALLOC(L.pstat, np);
    ALLOC(L.dropped, np);
    ALLOC(L.E, np * R * R);
    ALLOC(L.phi, np * R * nvf);
    if (l > 0) {
      ALLOC(L.par_w, np * h->slots);
      double **pp = nullptr;
      ALLOC(pp, np * h->slots);
      L.par_ptr = const_cast<const double **>(pp);
      std::vector<const double *> hp(np * h->slots, nullptr);
      for (size_t i = 0; i < np * h->slots; ++i) {
        const int pl = L.plan.par_level[i];
        if (pl > 0) hp[i] = h->lv[pl - 1].phi + (size_t)L.plan.par_pos[i] * R * nvf;
      }
      cudaError_t e = cudaMemcpyAsync(pp, hp.data(), hp.size() * sizeof(void *),
                                      cudaMemcpyHostToDevice, h->st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.par_w, L.plan.par_w.data(), L.plan.par_w.size() * sizeof(double),
                            cudaMemcpyHostToDevice, h->st);
      if (e != cudaSuccess) { mch_destroy(h); return MCH_ERR_CUDA; }
    }
  }
  ALLOC(h->yc, max_unit_nvc);
  {
    size_t max_units = 0;
    for (const Level &L : h->lv) max_units = std::max(max_units, (size_t)L.npts * h->R);
    ALLOC(h->bnorm, max_units);
  }
  if (max_fine) ALLOC(h->yfine, max_fine);
  h->yfine_cap = max_fine;
  if (d.overs > 0) {
    size_t max_el = 0;
    for (const Level &L : h->lv) max_el = std::max(max_el, (size_t)L.npts * elems(d.dim, L.n));
    if (max_fine) ALLOC(h->yfineR, max_fine);
    ALLOC(h->cR, max_unit_nvc);
    ALLOC(h->kapR, max_el);
  }
#undef ALLOC
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) { mch_destroy(h); return MCH_ERR_CUDA; }
  *out = h;
  return MCH_OK;
}

mch_status mch_plan_level(const mch_desc *desc, int level, int *n_points, int32_t *idx_out,
                          int32_t *parent_level, int32_t *parent_pos, double *weight) {
  if (!desc || !n_points || !desc->level_stride || level < 1 || level > desc->n_levels)
    return MCH_ERR_ARG;
  std::vector<int> strides(desc->level_stride, desc->level_stride + desc->n_levels);
  std::vector<LevelPlan> plans;
  std::string err;
  if (desc->eta < 1 ||
      !build_plan(desc->dim, desc->macro_n, strides, desc->n_fine, desc->eta, plans, err,
                  desc->interp))
    return MCH_ERR_ARG;
  const LevelPlan &L = plans[level - 1];
  *n_points = (int)L.points.size() / desc->dim;
  if (idx_out)
    for (size_t i = 0; i < L.points.size(); ++i) idx_out[i] = L.points[i];
  for (size_t i = 0; i < L.par_level.size(); ++i) {
    if (parent_level) parent_level[i] = L.par_level[i];
    if (parent_pos) parent_pos[i] = L.par_pos[i];
    if (weight) weight[i] = L.par_w[i];
  }
  return MCH_OK;
}

int mch_level_num_points(const mch_handle *h, int level) {
  return valid_level(h, level) ? h->lv[level - 1].npts : -1;
}

int mch_level_n_elem(const mch_handle *h, int level) {
  return valid_level(h, level) ? h->lv[level - 1].n : -1;
}

mch_status mch_level_points(const mch_handle *h, int level, int32_t *idx_out) {
  if (!valid_level(h, level) || !idx_out) return MCH_ERR_ARG;
  const auto &p = h->lv[level - 1].plan.points;
  for (size_t i = 0; i < p.size(); ++i) idx_out[i] = p[i];
  return MCH_OK;
}

mch_status mch_level_parents(const mch_handle *h, int level, int32_t *parent_level,
                             int32_t *parent_pos, double *weight) {
  if (!valid_level(h, level) || !parent_level || !parent_pos || !weight) return MCH_ERR_ARG;
  const auto &L = h->lv[level - 1].plan;
  for (size_t i = 0; i < L.par_level.size(); ++i) {
    parent_level[i] = L.par_level[i];
    parent_pos[i] = L.par_pos[i];
    weight[i] = L.par_w[i];
  }
  return MCH_OK;
}

}  // extern "C"

namespace {

// Algorithm 1, lines 4-6, for the points [p0, p1) of a level (all of them from
// mch_solve_level); kappa and labels hold those points only.
mch_status solve_range(mch_handle *h, int level, int p0, int p1, const double *kappa,
                       const uint8_t *labels) {
  const int li = level - 1;
  for (int k = 0; k < li; ++k)
    if (!h->lv[k].solved)
      return set_err(h, MCH_ERR_ORDER, "level " + std::to_string(level) +
                                           " needs level " + std::to_string(k + 1) + " first");
  CK(restore_phi(h), "recompute cell functions");
  Level &L0 = h->lv[li];
  const bool whole = p0 == 0 && p1 == L0.npts;
  Level L = range_view(L0, p0, p1, h->d.dim, h->R, h->nc, h->slots);
  const mch_desc &d = h->d;
  const int R = h->R, nc = h->nc, N = d.n_cont, P = d.periods;
  const size_t np = L.npts, ne = elems(d.dim, L.n);
  const bool fp64 = d.precision == MCH_FP64;
  const bool d3 = d.dim == 3;
  cudaStream_t st = h->st;
  h->h2d = h->d2h = 0;
  h->launches = 0;
  L0.solved = false;
  L0.partial = !whole;

  // phase marks for optional event timing: tag 0 setup, 1 interp, 2 pcg, 3 prep, 4 final
  std::vector<int> tags;
  const bool timing = h->timing;
  auto mark = [&](int tag) -> cudaError_t {
    if (!timing) return cudaSuccess;
    tags.push_back(tag);
    return cudaEventRecord(h->ev[tags.size() - 1], st);
  };
  // ---- staged inputs and constraint data (already done if mch_prepare_level was called
  // with the same buffers)
  CK(mark(-1), "event");
  // a pending preparation writes this level's buffers on the side stream: always wait for it
  if (L0.prepared) CK(cudaStreamWaitEvent(st, L0.prep_ev, 0), "wait for prepared level");
  if (whole && L0.prepared && L0.prep_kappa == kappa && L0.prep_labels == labels) {
    h->launches += L0.prep_launches;
    h->h2d += L0.prep_h2d;
  } else {
    int nl = 0;
    CK(setup_level(h, L, kappa, labels, st, &nl), "setup");
    h->launches += nl;
  }
  L0.prepared = false;
  CK(mark(0), "event");

  // |R_p| = the central (P - 2 overs)^d periods (the whole RVE when overs = 0)
  const double rlen = d.rve_len * (double)(P - 2 * d.overs) / P;
  const double inv_vol = 1.0 / (d3 ? rlen * rlen * rlen : rlen * rlen);
  const bool ovs = d.overs > 0;
  const double *g = L.G;
  const double *bvec = nullptr;
  if (li > 0) {
    // ---- interpolation and correction right-hand sides (level-1 grid, FP64)
    CK(cudaMemcpyAsync(L.gI, L.G, np * nc * R * sizeof(double), cudaMemcpyDeviceToDevice, st),
       "targets copy");
    CK(cudaMemsetAsync(L.E, 0, np * R * R * sizeof(double), st), "zero E");
    int nl = 0;
    if (L.kapff) {
      CK(launch_to_ff((int)np, L.kappa, (int)ne, L.kapff, (int)ne, (int)ne, st), "kappa ff");
      ++h->launches;
    }
    CK(launch_child(h, L, L.gI, &nl), "child fine");
    // K_I = I^T A_1 I (or with A_1 restricted to R_p): a symmetric form
    CK(launch_gram((int)np, R, L.nvf, L.phi, ovs ? h->yfineR : h->yfine, inv_vol, L.E, st,
                   h->ffs, true),
       "gram I");
    CK(launch_restrict(h, L, h->yfine, -1.0, L.b, h->ffs), "restrict");
    if (ovs) {
      CK(launch_restrict(h, L, h->yfineR, 1.0, h->cR, h->ffs), "restrict R_p");
      ++h->launches;
    }
    CK(launch_bnorm((int)np, R, L.nv, L.b, L.minv, h->bnorm, st), "b norm");
    h->launches += nl + 3;
    g = L.gI;
    bvec = L.b;
    CK(mark(1), "event");
  }

  // ---- constrained solves: one persistent launch (FP64 refinement around inner sweeps), or
  // point_batch points per launch
  const int max_iter = d.max_iter > 0 ? d.max_iter : 4 * L.n + 50;
  const size_t chunk = d.point_batch > 0 ? std::min(np, (size_t)d.point_batch) : np;
  int solve_launches = 0;
  if (d3) {
    CK(solve3d(h, L, g, bvec, L.x, L.iters, L.sweeps, L.ratio, L.ustat, L.lam,
               bvec ? h->bnorm : nullptr),
       "level 3d");
    ++h->launches;
    ++solve_launches;
  }
  for (size_t p0 = 0; p0 < np && !d3; p0 += chunk) {
    const int cn = (int)std::min(chunk, np - p0);
    const size_t u0 = p0 * R;
    const double *bb = bvec ? bvec + u0 * L.nv : nullptr;
    double *lam = L.lam ? L.lam + u0 * nc : nullptr;
    if (fp64) {
      LevelArgs<double> la{cn, R, L.n, P, N, nc, L.nv, ilog2(L.n / P), ilog2(P),
                           L.kappa + p0 * ne, L.labels + p0 * ne, L.Sinv64 + p0 * nc * nc,
                           L.Sinv64 + p0 * nc * nc, L.minv + p0 * L.nv, g + p0 * nc * R, bb,
                           L.x + u0 * L.nv, L.iters + u0, L.sweeps + u0, L.ratio + u0,
                           L.ustat + u0, (float)d.inner_tol, max_iter, d.rtol, d.max_refine, lam,
                           bvec ? h->bnorm + u0 : nullptr, L0.variant, h->yc + u0 * L.nv};
      CK(launch_level2d<double>(la, st), "level fp64");
    } else {
      LevelArgs<float> la{cn, R, L.n, P, N, nc, L.nv, ilog2(L.n / P), ilog2(P),
                          L.kappa + p0 * ne, L.labels + p0 * ne, L.Sinv32 + p0 * nc * nc,
                          L.Sinv64 + p0 * nc * nc, L.minv + p0 * L.nv, g + p0 * nc * R, bb,
                          L.x + u0 * L.nv, L.iters + u0, L.sweeps + u0, L.ratio + u0,
                          L.ustat + u0, (float)d.inner_tol, max_iter, d.rtol, d.max_refine, lam,
                          bvec ? h->bnorm + u0 : nullptr, L0.variant, h->yc + u0 * L.nv};
      CK(launch_level2d<float>(la, st), "level fp32");
    }
    ++h->launches;
    ++solve_launches;
  }
  CK(mark(2), "event");

  // ---- effective coefficients and the cell functions on the level-1 grid
  // |Y| E = K_I + sym(Xi^T (A_n Xi - 2 b)); with oversampling every operator is restricted to
  // R_p: |R_p| E = K_I,R + sym(Xi^T (A_n,R Xi + 2 P^T A_1,R I))
  ApplyArgs ac{(int)np, R, L.n, 1, L.nv, L.kappa, L.x, bvec, -2.0, h->yc};
  if (ovs) {
    CK(launch_mask_region(d.dim, (int)np, L.n, P, d.overs, L.kappa, h->kapR, st), "mask kappa");
    ++h->launches;
    ac.kappa = h->kapR;
    ac.b = li > 0 ? h->cR : nullptr;
    ac.cb = 2.0;
  }
  CK(d3 ? launch_apply3d(ac, d.rve_len / L.n, st) : launch_apply2d(ac, st), "apply coarse");
  if (li == 0) CK(cudaMemsetAsync(L.E, 0, np * R * R * sizeof(double), st), "zero E");
  CK(launch_gram((int)np, R, L.nv, L.x, h->yc, inv_vol, L.E, st), "gram");
  h->launches += 2;
  if (li == 0) {
    CK(h->ffs ? launch_to_ff((int)(np * R), L.x, L.nv, L.phi, L.nvf, L.nv, st)
              : cudaMemcpyAsync(L.phi, L.x, np * R * L.nv * sizeof(double),
                                cudaMemcpyDeviceToDevice, st),
       "phi copy");
  } else {
    CK(launch_prolong(h, L), "prolong");
    ++h->launches;
  }
  CK(mark(4), "event");

  // ---- convergence record
  std::vector<int> iters(np * R), sweeps(np * R), ustat(np * R), pstat(np), dropped(np);
  std::vector<double> ratio(np * R);
  CK(cudaMemcpyAsync(iters.data(), L.iters, iters.size() * sizeof(int), cudaMemcpyDeviceToHost, st),
     "read iters");
  CK(cudaMemcpyAsync(ustat.data(), L.ustat, ustat.size() * sizeof(int), cudaMemcpyDeviceToHost, st),
     "read status");
  CK(cudaMemcpyAsync(sweeps.data(), L.sweeps, sweeps.size() * sizeof(int), cudaMemcpyDeviceToHost,
                     st),
     "read sweeps");
  CK(cudaMemcpyAsync(pstat.data(), L.pstat, pstat.size() * sizeof(int), cudaMemcpyDeviceToHost, st),
     "read pstat");
  CK(cudaMemcpyAsync(dropped.data(), L.dropped, dropped.size() * sizeof(int),
                     cudaMemcpyDeviceToHost, st),
     "read dropped");
  CK(cudaMemcpyAsync(ratio.data(), L.ratio, ratio.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     st),
     "read ratio");
  CK(cudaStreamSynchronize(st), "level sync");

  mch_level_stats &S = L0.stats;
  S = mch_level_stats{};
  S.n_points = (int)np;
  S.n_elem = L.n;
  bool breakdown = false, degenerate = false, notconv = false;
  int bad_pt = -1, bad_unit = -1;
  for (size_t i = 0; i < np; ++i) {
    S.n_dropped_rows += dropped[i];
    if (pstat[i]) {
      degenerate = true;
      if (bad_pt < 0) bad_pt = (int)i;
    }
  }
  for (size_t u = 0; u < np * R; ++u) {
    S.total_iters += iters[u];
    S.max_iters = std::max(S.max_iters, iters[u]);
    const double rr = ratio[u];
    if (!(rr == rr)) notconv = true;
    else S.max_relres = std::max(S.max_relres, rr);
    if (ustat[u] & 1) {
      breakdown = true;
      if (bad_unit < 0) bad_unit = (int)u;
    }
    if (!(rr < d.rtol)) notconv = true;
  }
  for (size_t u = 0; u < np * R; ++u) S.sweeps = std::max(S.sweeps, sweeps[u]);
  S.pcg_launches = solve_launches;
  const long long nodes = (long long)(L.n - 1) * (L.n - 1) * (d3 ? L.n - 1 : 1);
  const int nch = d3 ? 1 : level2d_cheb_steps(L.n, fp64, L0.variant);
  for (size_t u = 0; u < np * R; ++u) {
    S.pcg_node_iters += (long long)iters[u] * nodes;
    S.pcg_node_applies += ((long long)iters[u] * nch + (long long)sweeps[u] * (nch - 1)) * nodes;
  }
  for (size_t k = 1; k < tags.size(); ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[k - 1], h->ev[k]), "event time");
    switch (tags[k]) {
      case 0: S.setup_ms += ms; break;
      case 1: S.interp_ms += ms; break;
      case 2: S.pcg_ms += ms; break;
      case 3: S.prep_ms += ms; break;
      case 4: S.final_ms += ms; break;
    }
  }
  S.gpu_launches = h->launches;
  S.h2d_bytes = h->h2d;
  S.d2h_bytes = h->d2h;
  if (degenerate)
    return set_err(h, MCH_ERR_DEGENERATE,
                   "point " + std::to_string(bad_pt) + " has flags " +
                       std::to_string(pstat[bad_pt]) +
                       " (1 kappa<=0, 2 label>=n_cont, 4 singular constraints, 8 absent continuum)");
  L0.solved = true;
  if (!d.keep_parents && li == d.n_levels - 1) CK(release_phi(h), "release cell functions");
  if (breakdown)
    return set_err(h, MCH_ERR_BREAKDOWN, "PCG breakdown at unit " + std::to_string(bad_unit));
  if (notconv) {
    char buf[128];
    snprintf(buf, sizeof buf, "largest residual ratio %.3e above rtol %.3e", S.max_relres, d.rtol);
    return set_err(h, MCH_ERR_NOT_CONVERGED, buf);
  }
  h->err.clear();
  return MCH_OK;
}

}  // namespace

extern "C" {

mch_status mch_solve_level(mch_handle *h, int level, const double *kappa, const uint8_t *labels) {
  if (!valid_level(h, level) || !kappa || !labels) return set_err(h, MCH_ERR_ARG, "bad argument");
  return solve_range(h, level, 0, h->lv[level - 1].npts, kappa, labels);
}

mch_status mch_solve_level_range(mch_handle *h, int level, int p0, int p1, const double *kappa,
                                 const uint8_t *labels) {
  if (!valid_level(h, level)) return set_err(h, MCH_ERR_ARG, "bad argument");
  Level &L = h->lv[level - 1];
  if (p0 < 0 || p1 < p0 || p1 > L.npts) return set_err(h, MCH_ERR_ARG, "bad point range");
  if (p0 == p1) {
    // no point of this level here: the level is complete once its cell functions have been
    // imported (mch_set_cell_functions)
    for (int k = 0; k < level - 1; ++k)
      if (!h->lv[k].solved) return set_err(h, MCH_ERR_ORDER, "earlier level not solved");
    L.solved = true;
    L.partial = true;
    return MCH_OK;
  }
  if (!kappa || !labels) return set_err(h, MCH_ERR_ARG, "bad argument");
  return solve_range(h, level, p0, p1, kappa, labels);
}

mch_status mch_set_cell_functions(mch_handle *h, int level, int p0, int p1, const double *phi) {
  if (!valid_level(h, level) || !phi) return set_err(h, MCH_ERR_ARG, "bad argument");
  Level &L = h->lv[level - 1];
  if (p0 < 0 || p1 < p0 || p1 > L.npts) return set_err(h, MCH_ERR_ARG, "bad point range");
  if (p0 == p1) return MCH_OK;
  CK(restore_phi(h), "recompute cell functions");
  const size_t W = (size_t)h->d.n_fine + 1;
  const size_t len = h->d.dim == 3 ? W * W * W : W * W;
  const size_t rows = (size_t)(p1 - p0) * h->R;
  double *dst = L.phi + (size_t)p0 * h->R * L.nvf;
  const bool dev = is_device_ptr(phi);
  if (!dev) h->h2d += (long long)(rows * len * sizeof(double));
  if (h->ffs && dev) {
    CK(launch_to_ff((int)rows, phi, (int)len, dst, L.nvf, (int)len, h->st), "convert phi");
  } else if (h->ffs) {
    // FP64 -> float-float planes, host sources staged through the level-1-grid scratch (or a
    // temporary buffer when the hierarchy has none) in chunks of whole vectors
    double *buf = h->yfine, *tmp = nullptr;
    size_t cap = h->yfine_cap / len;
    if (cap == 0) {
      CK(dalloc(h, &tmp, len), "cell functions buffer");
      buf = tmp;
      cap = 1;
    }
    for (size_t r0 = 0; r0 < rows; r0 += cap) {
      const size_t cnt = std::min(cap, rows - r0);
      CK(cudaMemcpyAsync(buf, phi + r0 * len, cnt * len * sizeof(double),
                         cudaMemcpyHostToDevice, h->st),
         "stage cell functions");
      CK(launch_to_ff((int)cnt, buf, (int)len, dst + r0 * L.nvf, L.nvf, (int)len, h->st),
         "convert phi");
      CK(cudaStreamSynchronize(h->st), "sync");
    }
    if (tmp) dfree(h, tmp);
  } else {
    CK(cudaMemcpy2DAsync(dst, (size_t)L.nvf * sizeof(double), phi, len * sizeof(double),
                         len * sizeof(double), rows,
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st),
       "copy phi");
  }
  CK(cudaStreamSynchronize(h->st), "sync");
  return MCH_OK;
}

mch_status mch_effective_coeffs(mch_handle *h, int level, double *E, int32_t *iters,
                                double *relres) {
  if (!valid_level(h, level) || !E) return set_err(h, MCH_ERR_ARG, "bad argument");
  Level &L = h->lv[level - 1];
  if (!L.solved) return set_err(h, MCH_ERR_ORDER, "level not solved");
  const size_t np = L.npts, R = h->R;
  h->d2h = 0;
  CK(stage(h, E, L.E, np * R * R * sizeof(double), false), "copy E");
  if (iters) CK(stage(h, iters, L.iters, np * R * sizeof(int), false), "copy iters");
  if (relres) CK(stage(h, relres, L.ratio, np * R * sizeof(double), false), "copy relres");
  CK(cudaStreamSynchronize(h->st), "sync");
  L.stats.d2h_bytes += h->d2h;
  return MCH_OK;
}

mch_status mch_cell_functions(mch_handle *h, int level, double *phi) {
  if (!valid_level(h, level) || !phi) return set_err(h, MCH_ERR_ARG, "bad argument");
  Level &L = h->lv[level - 1];
  if (!L.solved) return set_err(h, MCH_ERR_ORDER, "level not solved");
  CK(restore_phi(h), "recompute cell functions");
  // library vectors are padded to nvf entries; the caller's layout is dense (n_fine+1)^2
  const size_t W = (size_t)h->d.n_fine + 1;
  const size_t row = (h->d.dim == 3 ? W * W * W : W * W) * sizeof(double);
  const size_t rows = (size_t)L.npts * h->R;
  const bool dev = is_device_ptr(phi);
  if (!dev) h->d2h += (long long)(row * rows);
  if (h->ffs) {
    // float-float planes -> FP64, through a temporary device buffer for host destinations
    const int len = (int)(row / sizeof(double));
    double *dst = phi, *tmp = nullptr;
    if (!dev) {
      CK(dalloc(h, &tmp, rows * (size_t)len), "cell functions buffer");
      dst = tmp;
    }
    CK(launch_from_ff((int)rows, L.phi, L.nvf, dst, len, len, h->st), "convert phi");
    if (!dev) {
      CK(cudaMemcpyAsync(phi, tmp, rows * row, cudaMemcpyDeviceToHost, h->st), "copy phi");
      CK(cudaStreamSynchronize(h->st), "sync");
      dfree(h, tmp);
    }
  } else {
    CK(cudaMemcpy2DAsync(phi, row, L.phi, (size_t)L.nvf * sizeof(double), row, rows,
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st),
       "copy phi");
  }
  CK(cudaStreamSynchronize(h->st), "sync");
  return MCH_OK;
}

mch_status mch_macro_source(mch_handle *h, int level, const double *weights,
                            const double *center, double alpha, const double *origin,
                            double spacing, double *fbar) {
  if (!valid_level(h, level) || !weights || !center || !origin || !fbar || !(spacing > 0.0) ||
      !(alpha >= 0.0))
    return set_err(h, MCH_ERR_ARG, "bad argument");
  const mch_desc &d = h->d;
  if (d.n_cont > MCH_MACRO_MAXN) return set_err(h, MCH_ERR_UNSUPPORTED, "at most 4 continua");
  Level &L = h->lv[level - 1];
  if (!L.solved) return set_err(h, MCH_ERR_ORDER, "level not solved");
  CK(restore_phi(h), "recompute cell functions");
  const int np = L.npts, N = d.n_cont, D = d.dim;
  std::vector<double> xp((size_t)np * D);
  for (int p = 0; p < np; ++p)
    for (int a = 0; a < D; ++a)
      xp[(size_t)p * D + a] = origin[a] + L.plan.points[(size_t)p * D + a] * spacing;
  double *dxp = nullptr, *dout = nullptr;
  CK(dalloc(h, &dxp, xp.size()), "positions");
  CK(cudaMemcpyAsync(dxp, xp.data(), xp.size() * sizeof(double), cudaMemcpyHostToDevice, h->st),
     "positions");
  h->h2d += (long long)(xp.size() * sizeof(double));
  const bool dev = is_device_ptr(fbar);
  double *out = fbar;
  if (!dev) {
    CK(dalloc(h, &dout, (size_t)np * N), "source buffer");
    out = dout;
  }
  MacroSourceArgs a{};
  a.npts = np;
  a.dim = D;
  a.N = N;
  a.R = h->R;
  a.nf = d.n_fine;
  a.lgr = ilog2(L.rho);
  a.nvf = L.nvf;
  a.P = d.periods;
  a.overs = d.overs;
  a.phi = L.phi;
  a.labels = L.labels;
  a.xp = dxp;
  a.rve_len = d.rve_len;
  a.alpha = alpha;
  for (int j = 0; j < N; ++j) a.w[j] = weights[j];
  for (int m = 0; m < D; ++m) a.c[m] = center[m];
  a.fbar = out;
  CK(launch_macro_source(a, h->ffs, h->st), "macro source");
  ++h->launches;
  if (!dev) {
    CK(cudaMemcpyAsync(fbar, out, (size_t)np * N * sizeof(double), cudaMemcpyDeviceToHost,
                       h->st),
       "copy source");
    h->d2h += (long long)((size_t)np * N * sizeof(double));
  }
  CK(cudaStreamSynchronize(h->st), "sync");
  dfree(h, dxp);
  dfree(h, dout);
  return MCH_OK;
}

mch_status mch_macro_solve(mch_handle *h, const double *const *E, const double *const *fbar,
                           double spacing, double tol, int max_iter, double *U, int *iters,
                           double *relres) {
  if (!h || !E || !fbar || !U || !(spacing > 0.0) || !(tol >= 0.0) || max_iter < 0)
    return set_err(h, MCH_ERR_ARG, "bad argument");
  const mch_desc &d = h->d;
  const int D = d.dim, N = d.n_cont, R = h->R, M = d.macro_n;
  if (N > MCH_MACRO_MAXN) return set_err(h, MCH_ERR_UNSUPPORTED, "at most 4 continua");
  if (M < 2) return set_err(h, MCH_ERR_ARG, "macro grid too small");
  if (tol == 0.0) tol = 1e-12;
  if (max_iter == 0) max_iter = 20000;
  size_t nel = 1, nn = 1;
  for (int a = 0; a < D; ++a) {
    nel *= (size_t)M;
    nn *= (size_t)(M + 1);
  }
  const size_t nu = (size_t)N * nn;
  std::vector<void *> tmp;
  auto take = [&](auto **p, size_t count) {
    cudaError_t e = dalloc(h, p, count);
    if (e == cudaSuccess) tmp.push_back(*p);
    return e;
  };
  auto release = [&]() {
    for (void *q : tmp) dfree(h, q);
    tmp.clear();
  };
  double *Eg = nullptr, *fg = nullptr, *work = nullptr, *Ud = nullptr, *rr = nullptr;
  int *it_d = nullptr;
  cudaError_t e = take(&Eg, nel * R * R);
  if (e == cudaSuccess) e = take(&fg, nel * N);
  if (e == cudaSuccess) e = take(&work, 4 * nu);
  if (e == cudaSuccess) e = take(&rr, 1);
  if (e == cudaSuccess) e = take(&it_d, 1);
  const bool dev = is_device_ptr(U);
  if (e == cudaSuccess && !dev) e = take(&Ud, nu);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(h, e, "macro buffers");
  }
  size_t covered = 0;
  for (size_t l = 0; l < h->lv.size(); ++l) {
    Level &L = h->lv[l];
    const int np = L.npts;
    if (!E[l] || !fbar[l]) {
      release();
      return set_err(h, MCH_ERR_ARG, "missing level coefficients");
    }
    std::vector<int> elem(np);
    for (int p = 0; p < np; ++p) {
      size_t flat = 0, stride = 1;
      for (int a = 0; a < D; ++a) {
        flat += (size_t)L.plan.points[(size_t)p * D + a] * stride;
        stride *= (size_t)M;
      }
      elem[p] = (int)flat;
    }
    int *elem_d = nullptr;
    double *El = nullptr, *fl = nullptr;
    e = take(&elem_d, np);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(elem_d, elem.data(), np * sizeof(int), cudaMemcpyHostToDevice, h->st);
    const double *Esrc = E[l], *fsrc = fbar[l];
    if (e == cudaSuccess && !is_device_ptr(Esrc)) {
      e = take(&El, (size_t)np * R * R);
      if (e == cudaSuccess) e = stage(h, El, Esrc, (size_t)np * R * R * sizeof(double), true);
      Esrc = El;
    }
    if (e == cudaSuccess && !is_device_ptr(fsrc)) {
      e = take(&fl, (size_t)np * N);
      if (e == cudaSuccess) e = stage(h, fl, fsrc, (size_t)np * N * sizeof(double), true);
      fsrc = fl;
    }
    if (e == cudaSuccess) e = launch_macro_gather(np, R, N, elem_d, Esrc, fsrc, Eg, fg, h->st);
    // the host vector must outlive its asynchronous copy
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(h, e, "macro gather");
    }
    ++h->launches;
    covered += (size_t)np;
  }
  if (covered != nel) {
    release();
    return set_err(h, MCH_ERR_ARG, "the levels do not cover the macro grid");
  }
  MacroSolveArgs a{};
  a.dim = D;
  a.M = M;
  a.N = N;
  a.R = R;
  a.max_iter = max_iter;
  a.H = spacing;
  a.tol = tol;
  a.E = Eg;
  a.f = fg;
  a.U = dev ? U : Ud;
  a.r = work;
  a.p = work + nu;
  a.q = work + 2 * nu;
  a.diag = work + 3 * nu;
  a.iters = it_d;
  a.relres = rr;
  e = launch_macro_cg(a, h->st);
  int it_h = 0;
  double rr_h = 0.0;
  if (e == cudaSuccess) {
    ++h->launches;
    if (!dev) {
      e = cudaMemcpyAsync(U, Ud, nu * sizeof(double), cudaMemcpyDeviceToHost, h->st);
      h->d2h += (long long)(nu * sizeof(double));
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&it_h, it_d, sizeof(int), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&rr_h, rr, sizeof(double), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  release();
  if (e != cudaSuccess) return cuda_fail(h, e, "macro solve");
  if (iters) *iters = it_h;
  if (relres) *relres = rr_h;
  if (!(rr_h <= tol)) {
    if (it_h < max_iter) return set_err(h, MCH_ERR_BREAKDOWN, "macro system not positive definite");
    return set_err(h, MCH_ERR_NOT_CONVERGED, "macro solve did not reach the tolerance");
  }
  return MCH_OK;
}

mch_status mch_set_timing(mch_handle *h, int enable) {
  if (!h) return MCH_ERR_ARG;
  if (enable && h->n_ev == 0) {
    for (int i = 0; i < 32; ++i) {
      if (cudaEventCreate(&h->ev[i]) != cudaSuccess) return set_err(h, MCH_ERR_CUDA, "event");
      h->n_ev = i + 1;
    }
  }
  h->timing = enable != 0;
  return MCH_OK;
}

mch_status mch_prepare_level(mch_handle *h, int level, const double *kappa,
                             const uint8_t *labels) {
  if (!valid_level(h, level) || !kappa || !labels) return set_err(h, MCH_ERR_ARG, "bad argument");
  Level &L = h->lv[level - 1];
  if (!h->st2) {
    CK(cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking), "side stream");
    CK(cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming), "event");
  }
  if (!L.prep_ev) CK(cudaEventCreateWithFlags(&L.prep_ev, cudaEventDisableTiming), "event");
  // after everything already enqueued on the handle's stream (the caller's inputs, and the
  // previous use of this level's buffers)
  CK(cudaEventRecord(h->ev_main, h->st), "event");
  CK(cudaStreamWaitEvent(h->st2, h->ev_main, 0), "wait");
  const long long h2d0 = h->h2d;
  int nl = 0;
  CK(setup_level(h, L, kappa, labels, h->st2, &nl), "prepare setup");
  CK(cudaEventRecord(L.prep_ev, h->st2), "event");
  L.prep_h2d = h->h2d - h2d0;
  h->h2d = h2d0;
  L.prep_launches = nl;
  L.prep_kappa = kappa;
  L.prep_labels = labels;
  L.prepared = true;
  return MCH_OK;
}

mch_status mch_set_level_variant(mch_handle *h, int level, int variant) {
  if (!valid_level(h, level)) return set_err(h, MCH_ERR_ARG, "bad level");
  Level &L = h->lv[level - 1];
  const bool fp64 = h->d.precision == MCH_FP64;
  if (variant != 0 && (h->d.dim != 2 || !level2d_variant_ok(L.n, h->d.periods, fp64, variant)))
    return set_err(h, MCH_ERR_UNSUPPORTED, "launch shape not valid for this level");
  L.variant = variant;
  return MCH_OK;
}

mch_status mch_get_level_variant(const mch_handle *h, int level, int *variant, int *count) {
  if (!valid_level(h, level)) return MCH_ERR_ARG;
  const Level &L = h->lv[level - 1];
  if (variant) *variant = L.variant;
  if (count)
    *count = h->d.dim == 2 ? level2d_variant_count(L.n, h->d.precision == MCH_FP64) : 1;
  return MCH_OK;
}

mch_status mch_autotune_level(mch_handle *h, int level, const double *kappa,
                              const uint8_t *labels, int *best, double *best_ms) {
  if (!valid_level(h, level) || !kappa || !labels) return set_err(h, MCH_ERR_ARG, "bad argument");
  Level &L = h->lv[level - 1];
  const mch_desc &d = h->d;
  const bool fp64 = d.precision == MCH_FP64;
  const int count = d.dim == 2 ? level2d_variant_count(L.n, fp64) : 1;
  char key[160];
  snprintf(key, sizeof key, "mch-tune %d %d %d %d %s %d", d.dim, L.n, d.periods, d.n_cont,
           fp64 ? "fp64" : "mixed", L.npts);
  const char *cache = getenv("MCH_TUNE_CACHE");
  int chosen = -1;
  double chosen_ms = 0.0;
  if (cache && *cache) {
    if (FILE *f = fopen(cache, "r")) {
      char line[256];
      const size_t kl = strlen(key);
      while (fgets(line, sizeof line, f)) {
        int v = -1;
        if (strncmp(line, key, kl) == 0 && line[kl] == ' ' && sscanf(line + kl, "%d", &v) == 1 &&
            v >= 0 && v < count && (v == 0 || level2d_variant_ok(L.n, d.periods, fp64, v)))
          chosen = v;
      }
      fclose(f);
    }
  }
  if (chosen < 0 && count > 1) {
    const bool timing = h->timing;
    mch_status st = mch_set_timing(h, 1);
    if (st != MCH_OK) return st;
    double best_t = 1e300;
    for (int v = 0; v < count; ++v) {
      if (v != 0 && !level2d_variant_ok(L.n, d.periods, fp64, v)) continue;
      L.variant = v;
      if (mch_solve_level(h, level, kappa, labels) != MCH_OK) continue;
      const double t = L.stats.pcg_ms;
      if (t < best_t) {
        best_t = t;
        chosen = v;
      }
    }
    h->timing = timing;
    if (chosen < 0) chosen = 0;
    chosen_ms = best_t < 1e300 ? best_t : 0.0;
    if (cache && *cache) {
      if (FILE *f = fopen(cache, "a")) {
        fprintf(f, "%s %d %.4f\n", key, chosen, chosen_ms);
        fclose(f);
      }
    }
  }
  if (chosen < 0) chosen = 0;
  L.variant = chosen;
  if (best) *best = chosen;
  if (best_ms) *best_ms = chosen_ms;
  return mch_solve_level(h, level, kappa, labels);
}

mch_status mch_level_stats_get(const mch_handle *h, int level, mch_level_stats *out) {
  if (!valid_level(h, level) || !out) return MCH_ERR_ARG;
  *out = h->lv[level - 1].stats;
  out->n_points = h->lv[level - 1].npts;
  out->n_elem = h->lv[level - 1].n;
  return MCH_OK;
}

mch_status mch_backward(mch_handle *h, const double *const *dL_dE, double *const *dL_dkappa) {
  if (!h || !dL_dE || !dL_dkappa) return set_err(h, MCH_ERR_ARG, "bad argument");
  const mch_desc &d = h->d;
  const int Lv = d.n_levels, R = h->R, nc = h->nc, N = d.n_cont, P = d.periods;
  for (int l = 0; l < Lv; ++l) {
    if (!h->lv[l].solved) return set_err(h, MCH_ERR_ORDER, "every level must be solved first");
    if (h->lv[l].partial)
      return set_err(h, MCH_ERR_ORDER, "the backward pass needs every point solved on this handle");
    if (!dL_dE[l] || !dL_dkappa[l]) return set_err(h, MCH_ERR_ARG, "null gradient buffer");
  }
  cudaStream_t st = h->st;
  const int nvf = nvd(d.dim, d.n_fine);
  const bool d3 = d.dim == 3;
  CK(restore_phi(h), "recompute cell functions");
  if (!h->bw_ready) {
    size_t mfine = 0, munit = 0, mnc = 0, mrr = 0, mel = 0;
    for (int l = 0; l < Lv; ++l) {
      const Level &L = h->lv[l];
      mfine = std::max(mfine, (size_t)L.npts * R * nvf);
      munit = std::max(munit, (size_t)L.npts * R);
      mnc = std::max(mnc, (size_t)L.npts * R * nc);
      mrr = std::max(mrr, (size_t)L.npts * R * R);
      mel = std::max(mel, (size_t)L.npts * elems(d.dim, L.n));
    }
#define BALLOC(ptr, cnt)                                               \
  do {                                                                 \
    cudaError_t e_ = dalloc(h, &(ptr), (size_t)(cnt));                 \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, "backward buffers"); \
  } while (0)
    BALLOC(h->psi1, mfine);
    BALLOC(h->psi2, mfine);
    BALLOC(h->lamadj, mnc);
    BALLOC(h->gzero, mnc);
    BALLOC(h->Wd, mrr);
    BALLOC(h->dk, mel);
    BALLOC(h->bw_ratio, munit);
    BALLOC(h->bw_iters, munit);
    BALLOC(h->bw_sweeps, munit);
    BALLOC(h->bw_status, munit);
    // seeds on the level-1 grid: levels with children, and with oversampling every level
    // (the level's own term is an adjoint source)
    for (int l = 0; l < Lv; ++l)
      if (l + 1 < Lv || d.overs > 0) BALLOC(h->lv[l].V, (size_t)h->lv[l].npts * R * nvf);
    for (int l = 1; l < Lv; ++l) {
      Level &L = h->lv[l];
      BALLOC(L.par_V, (size_t)L.npts * h->slots);
      std::vector<double *> hp((size_t)L.npts * h->slots, nullptr);
      for (size_t i = 0; i < hp.size(); ++i) {
        const int pl = L.plan.par_level[i];
        if (pl > 0) hp[i] = h->lv[pl - 1].V + (size_t)L.plan.par_pos[i] * R * nvf;
      }
      CK(cudaMemcpyAsync(L.par_V, hp.data(), hp.size() * sizeof(void *), cudaMemcpyHostToDevice,
                         st),
         "seed table");
      CK(cudaStreamSynchronize(st), "seed table");
    }
#undef BALLOC
    h->bw_ready = true;
  }
  h->h2d = h->d2h = 0;
  for (int l = 0; l < Lv; ++l)
    if (h->lv[l].V)
      CK(cudaMemsetAsync(h->lv[l].V, 0, (size_t)h->lv[l].npts * R * nvf * sizeof(double), st),
         "zero seeds");
  const double rlen = d.rve_len * (double)(P - 2 * d.overs) / P;
  const double inv_vol = 1.0 / (d3 ? rlen * rlen * rlen : rlen * rlen);
  const double hf = d.rve_len / d.n_fine;
  const bool fp64 = d.precision == MCH_FP64;
  double worst = 0.0;
  bool breakdown = false;
  for (int li = Lv - 1; li >= 0; --li) {
    Level &L = h->lv[li];
    const size_t np = L.npts;
    CK(stage(h, h->Wd, dL_dE[li], np * R * R * sizeof(double), true), "stage dL/dE");
    const bool seeds = L.V != nullptr;
    AdjArgs aa{(int)np, R, d.n_fine, ilog2(L.rho), nvf, L.nv, nc, ilog2(d.n_fine / P), P,
               h->slots, inv_vol, 1.0 / rho_pow(h, L.rho), h->Wd, L.phi,
               seeds ? h->yc : nullptr, L.lam, seeds ? h->lamadj : nullptr, L.kappa, L.labels,
               L.V, h->psi1, h->psi2, h->dk, L.par_V, L.par_w, h->ffs ? 1 : 0, d.overs};
    if (d.overs > 0)
      CK(d3 ? launch_adj_own3d(aa, hf, st) : launch_adj_own2d(aa, st), "adjoint own term");
    if (seeds) {
      // adjoint constrained solve with right-hand side P^T V and zero targets
      if (L.rho > 1) {
        CK(launch_restrict(h, L, L.V, 1.0, L.b, false), "restrict seeds");
      } else {
        CK(cudaMemcpyAsync(L.b, L.V, np * R * nvf * sizeof(double), cudaMemcpyDeviceToDevice, st),
           "copy seeds");
      }
      CK(cudaMemsetAsync(h->yc, 0, np * R * L.nv * sizeof(double), st), "zero mu");
      CK(launch_bnorm((int)np, R, L.nv, L.b, L.minv, h->bnorm, st), "b norm");
      const int max_iter = d.max_iter > 0 ? d.max_iter : 4 * L.n + 50;
      if (d3) {
        CK(solve3d(h, L, h->gzero, L.b, h->yc, h->bw_iters, h->bw_sweeps, h->bw_ratio,
                   h->bw_status, h->lamadj, h->bnorm),
           "adjoint 3d");
      } else if (fp64) {
        LevelArgs<double> la{(int)np, R, L.n, P, N, nc, L.nv, ilog2(L.n / P), ilog2(P), L.kappa,
                             L.labels, L.Sinv64, L.Sinv64, L.minv, h->gzero, L.b, h->yc,
                             h->bw_iters, h->bw_sweeps, h->bw_ratio, h->bw_status,
                             (float)d.inner_tol, max_iter, d.rtol, d.max_refine, h->lamadj,
                             h->bnorm, L.variant};
        CK(launch_level2d<double>(la, st), "adjoint fp64");
      } else {
        LevelArgs<float> la{(int)np, R, L.n, P, N, nc, L.nv, ilog2(L.n / P), ilog2(P), L.kappa,
                            L.labels, L.Sinv32, L.Sinv64, L.minv, h->gzero, L.b, h->yc,
                            h->bw_iters, h->bw_sweeps, h->bw_ratio, h->bw_status,
                            (float)d.inner_tol, max_iter, d.rtol, d.max_refine, h->lamadj,
                            h->bnorm, L.variant};
        CK(launch_level2d<float>(la, st), "adjoint fp32");
      }
    }
    if (d3) {
      CK(launch_adj_combine3d(aa, st), "adjoint combine");
      CK(launch_adj_grad3d(aa, hf, st), "adjoint gradient");
      if (li > 0) CK(launch_adj_seed3d(aa, hf, st), "adjoint seeds");
    } else {
      CK(launch_adj_combine2d(aa, st), "adjoint combine");
      CK(launch_adj_grad2d(aa, st), "adjoint gradient");
      if (li > 0) CK(launch_adj_seed2d(aa, st), "adjoint seeds");
    }
    CK(stage(h, dL_dkappa[li], h->dk, np * elems(d.dim, L.n) * sizeof(double), false),
       "copy dL/dkappa");
    if (seeds) {
      std::vector<double> ratio(np * R);
      std::vector<int> stat(np * R);
      CK(cudaMemcpyAsync(ratio.data(), h->bw_ratio, ratio.size() * sizeof(double),
                         cudaMemcpyDeviceToHost, st),
         "read adjoint ratio");
      CK(cudaMemcpyAsync(stat.data(), h->bw_status, stat.size() * sizeof(int),
                         cudaMemcpyDeviceToHost, st),
         "read adjoint status");
      CK(cudaStreamSynchronize(st), "adjoint sync");
      for (size_t u = 0; u < np * R; ++u) {
        worst = std::max(worst, ratio[u] == ratio[u] ? ratio[u] : 1e300);
        breakdown |= stat[u] != 0;
      }
    }
  }
  CK(cudaStreamSynchronize(st), "backward sync");
  if (!d.keep_parents) CK(release_phi(h), "release cell functions");
  if (breakdown) return set_err(h, MCH_ERR_BREAKDOWN, "adjoint PCG breakdown");
  if (!(worst < d.rtol)) {
    char buf[128];
    snprintf(buf, sizeof buf, "adjoint residual ratio %.3e above rtol %.3e", worst, d.rtol);
    return set_err(h, MCH_ERR_NOT_CONVERGED, buf);
  }
  h->err.clear();
  return MCH_OK;
}

}  // extern "C"
