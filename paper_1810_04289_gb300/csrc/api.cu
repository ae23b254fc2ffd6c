// C ABI of the solver (include/fsi.h): context construction, residual,
// Jacobian, preconditioner, GMRES and the Newton step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fsi.h"
#include "kernels.cuh"
#include "setup.h"

using namespace fsi;

namespace {

struct CudaError {
  cudaError_t e;
  const char* what;
};

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) throw CudaError{e_, #call};  \
  } while (0)

struct StatusError {
  fsi_status st;
  std::string msg;
};

}  // namespace

enum { PH_FUNC = 0, PH_JAC, PH_PCSETUP, PH_PCAPPLY, PH_SPMV, PH_ORTH, PH_KRYLOV };

struct fsi_ctx {
  cudaStream_t s = nullptr;
  fsi_options opt{};
  fsi_material mat{};
  MatConst mc{};
  int64_t N = 0, T = 0, Tf = 0, nnzb = 0, nunk = 0, n = 0;  // n = 7N
  int32_t nprob = 1;
  std::vector<void*> allocs;
  int64_t dev_bytes = 0;
  std::string err;

  // mesh
  double* X = nullptr;
  int32_t* tets = nullptr;
  uint32_t* nflag = nullptr;
  int32_t* nprobid = nullptr;
  double* inlet = nullptr;
  MeshDev mesh{};
  // assembly
  int64_t *nptr = nullptr, *bptr = nullptr;
  int32_t *nsrc = nullptr, *bsrc = nullptr;
  double* Fe = nullptr;
  void* Ke = nullptr;
  int64_t ke_tets = 0;        // tets per chunk of the element Jacobian buffer
  void* Xl = nullptr;         // per-tet local reference coordinates, Jacobian type
  float* y32 = nullptr;       // mixed: FP32 copies of y, y_n, y_{n-1} for the Jacobian
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  int32_t* diag = nullptr;
  void* vals = nullptr;
  bool mixed = false;
  bool have_jac = false;
  // state
  double *yn = nullptr, *ynm1 = nullptr, *ynm2 = nullptr;
  double t = 0.0;
  // Newton
  double *yk = nullptr, *ytr = nullptr, *F = nullptr, *Ft = nullptr, *dy = nullptr, *rhs = nullptr;
  // GMRES, batched over the P problems (per-problem arrays are [P][...])
  int32_t m = 30;
  SegDev seg{};
  double *V = nullptr, *Z = nullptr, *r = nullptr;
  double *H = nullptr, *g = nullptr, *cs = nullptr, *sn = nullptr, *ylsq = nullptr, *hA = nullptr, *hB = nullptr;
  double* partial = nullptr;     // [chunks][m+1] reduction partials
  // inner-wall faces for the wall shear stress
  int64_t nwss = 0;
  int64_t* wface = nullptr;              // [nwss] 4 * internal fluid tet + opposite vertex
  int64_t* wfb = nullptr;                // [P+1] face offsets of the problems
  double *wma = nullptr, *wa = nullptr;  // [nwss] |WSS| area and area
  double* wsawss = nullptr;              // [P]
  std::vector<int32_t> wface_host;       // [nwss*2] input tet, opposite vertex
  double* beta = nullptr;        // [P] norms (residual of the cycle, Newton norms)
  double* gres = nullptr;        // [P] Givens residual estimates
  double* gtarget = nullptr;     // [P] GMRES stopping thresholds
  int* active = nullptr;         // [P] problem still iterating in the cycle
  int* kcols = nullptr;          // [P] Krylov columns built in the cycle
  int* anyact = nullptr;         // [1] some problem active (guard of the captured kernels)
  int* reorth = nullptr;         // [1] some problem needs a second Gram-Schmidt pass (orth = 1), or
                                 // its new norm from the updated vector (orth = 0 fallback)
  double* gs_inv = nullptr;      // [P] reciprocal of H[j+1][j] (orth 0)
  double* gs_nrm = nullptr;      // [P] norms formed from the updated vector (its fallback)
  double* gs_scal = nullptr;     // [P] their divisors
  int* gs_unsafe = nullptr;      // [P] the norm is taken from the updated vector
  int* pmask = nullptr;          // [P] problem already converged (Newton)
  double* palpha = nullptr;      // [P] line-search step per problem
  float* zf = nullptr;           // FP32 copy of the SpMV input (mixed precision)
  double* hbuf = nullptr;        // pinned host scratch (8 doubles + 4 P values)
  std::vector<double> hvec;      // host copies of per-problem scalars
  // one GMRES cycle captured as a CUDA graph
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_nodes = 0;
  // RAS
  RasPlan plan;
  RasDev ras{};
  void* fac = nullptr;
  void* work = nullptr;
  int32_t* errflag = nullptr;  // [0] zero pivot in the factorisation, [1] bounded wait gave up in the apply
  bool pc_stale = true;
  RasStreamDev rs{};
  bool use_stream = false;
  bool use_graph = true;
  // timing
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  struct Span {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Span> spans;
  double phase_ms[8] = {0};
  int32_t phase_n[8] = {0};
  int64_t launches = 0;
  bool timing = false;

  template <class U>
  U* dalloc(int64_t count) {
    void* p = nullptr;
    const size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(U);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) throw StatusError{FSI_ERR_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e)};
    allocs.push_back(p);
    dev_bytes += (int64_t)bytes;
    return (U*)p;
  }
  template <class U>
  U* upload(const std::vector<U>& v) {
    U* p = dalloc<U>((int64_t)v.size());
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice, s));
    return p;
  }

  cudaEvent_t ev() {
    if (evused == evpool.size()) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      evpool.push_back(e);
    }
    return evpool[evused++];
  }
  int begin_phase(int phase) {
    phase_n[phase]++;
    if (!timing) return -1;
    cudaEvent_t a = ev();
    CK(cudaEventRecord(a, s));
    spans.push_back({0, a, nullptr});
    return (int)spans.size() - 1;
  }
  void end_phase(int h, int phase) {
    if (h < 0) return;
    cudaEvent_t b = ev();
    CK(cudaEventRecord(b, s));
    spans[h].phase = phase;
    spans[h].b = b;
  }
  void resolve_phases() {
    if (!timing) return;
    CK(cudaStreamSynchronize(s));
    for (auto& sp : spans) {
      float ms = 0;
      if (sp.b) CK(cudaEventElapsedTime(&ms, sp.a, sp.b));
      phase_ms[sp.phase] += ms;
    }
    spans.clear();
    evused = 0;
  }
};

namespace {

fsi_status fail(fsi_ctx* c, fsi_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

template <class Fn>
fsi_status guarded(fsi_ctx* c, Fn&& fn) {
  try {
    return fn();
  } catch (const CudaError& e) {
    return fail(c, FSI_ERR_CUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
  } catch (const StatusError& e) {
    return fail(c, e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(c, FSI_ERR_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(c, FSI_ERR_MESH, e.what());
  }
}

void check_launch() { CK(cudaGetLastError()); }

// ---- F(y) for the step ending at t_n + dt (previous levels y_n, y_{n-1})
void residual(fsi_ctx* c, const double* y, double* F) {
  c->launches += 3;
  int h = c->begin_phase(PH_FUNC);
  launch_elem_residual(c->mesh, c->mc, y, c->yn, c->ynm1, c->Fe, c->s);
  launch_gather_residual(c->mesh, c->nptr, c->nsrc, c->Fe, F, c->s);
  launch_constraint_residual(c->mesh, c->mc, c->t + c->opt.dt, y, c->yn, F, c->s);
  check_launch();
  c->end_phase(h, PH_FUNC);
}

// per-problem 2-norms of x into c->hvec (host); returns the norm over all problems
double norms(fsi_ctx* c, const double* x, std::vector<double>& out) {
  c->launches += 1;
  launch_seg_norm(c->seg, x, c->partial, c->beta, 1, nullptr, c->s);
  out.resize(c->nprob);
  CK(cudaMemcpyAsync(c->hbuf, c->beta, sizeof(double) * c->nprob, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  double tot = 0.0;
  for (int p = 0; p < c->nprob; ++p) {
    out[p] = c->hbuf[p];
    tot += out[p] * out[p];
  }
  return std::sqrt(tot);
}

void jacobian(fsi_ctx* c, const double* y) {
  c->launches += 3;
  int h = c->begin_phase(PH_JAC);
  if (c->mixed) {
    c->launches += 1;
    launch_states_to_float(c->n, y, c->yn, c->ynm1, c->y32, c->s);
    for (int64_t t0 = 0; t0 < c->T; t0 += c->ke_tets) {
      const int64_t t1 = std::min(c->T, t0 + c->ke_tets);
      launch_elem_jacobian<float>(c->mesh, c->mc, (const float*)c->Xl, c->y32, c->y32 + c->n, c->y32 + 2 * c->n,
                                  (float*)c->Ke, t0, t1, c->s);
      launch_gather_jacobian<float>(c->nnzb, c->bptr, c->bsrc, (const float*)c->Ke, (float*)c->vals, t0, t1, c->s);
      c->launches += t0 > 0 ? 2 : 0;
    }
    launch_constraint_jacobian<float>(c->mesh, c->mc, c->diag, (float*)c->vals, c->s);
  } else {
    for (int64_t t0 = 0; t0 < c->T; t0 += c->ke_tets) {
      const int64_t t1 = std::min(c->T, t0 + c->ke_tets);
      launch_elem_jacobian<double>(c->mesh, c->mc, (const double*)c->Xl, y, c->yn, c->ynm1, (double*)c->Ke, t0, t1,
                                   c->s);
      launch_gather_jacobian<double>(c->nnzb, c->bptr, c->bsrc, (const double*)c->Ke, (double*)c->vals, t0, t1,
                                     c->s);
      c->launches += t0 > 0 ? 2 : 0;
    }
    launch_constraint_jacobian<double>(c->mesh, c->mc, c->diag, (double*)c->vals, c->s);
  }
  check_launch();
  c->end_phase(h, PH_JAC);
  c->have_jac = true;
  c->pc_stale = true;
}

// y = J x on stream st. Mixed precision: x32 must hold the FP32 copy of x (if
// x32 is null, it is made here from x).
void spmv_on(fsi_ctx* c, const double* x, const float* x32, double* y, const int* guard, cudaStream_t st) {
  if (c->mixed) {
    if (!x32) {
      c->launches += 1;
      launch_to_float(c->n, x, c->zf, guard, st);
      x32 = c->zf;
    }
    launch_bsr_spmv<float, float>(c->N, c->row_ptr, c->col, (const float*)c->vals, x32, y, c->opt.threads_per_row,
                                  guard, st);
  } else {
    launch_bsr_spmv<double, double>(c->N, c->row_ptr, c->col, (const double*)c->vals, x, y, c->opt.threads_per_row,
                                    guard, st);
  }
  c->launches += 1;
}

void spmv(fsi_ctx* c, const double* x, double* y) {
  int h = c->begin_phase(PH_SPMV);
  spmv_on(c, x, nullptr, y, nullptr, c->s);
  check_launch();
  c->end_phase(h, PH_SPMV);
}

void pc_setup(fsi_ctx* c) {
  c->launches += 2;
  int h = c->begin_phase(PH_PCSETUP);
  CK(cudaMemsetAsync(c->errflag, 0, sizeof(int32_t), c->s));
  if (c->mixed) {
    launch_ras_extract<float, float>(c->ras, (const float*)c->vals, (float*)c->fac, c->s);
    launch_ras_factor<float>(c->ras, (float*)c->fac, c->errflag, c->s);
  } else {
    launch_ras_extract<double, double>(c->ras, (const double*)c->vals, (double*)c->fac, c->s);
    launch_ras_factor<double>(c->ras, (double*)c->fac, c->errflag, c->s);
  }
  if (c->use_stream) {
    c->launches += 1;
    if (c->mixed)
      launch_pack_factors<float>(c->rs, (const float*)c->fac, c->s);
    else
      launch_pack_factors<double>(c->rs, (const double*)c->fac, c->s);
  }
  check_launch();
  c->end_phase(h, PH_PCSETUP);
  int32_t e = 0;
  CK(cudaMemcpyAsync(&c->hbuf[1], c->errflag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  std::memcpy(&e, &c->hbuf[1], sizeof(int32_t));
  if (e) throw StatusError{FSI_ERR_ZERO_PIVOT, "singular pivot block in the subdomain ILU factorisation"};
  c->pc_stale = false;
}

// z = B^{-1} r on stream st (z32: optional FP32 copy of z)
void pc_apply_on(fsi_ctx* c, const double* rin, double* z, float* z32, const int* guard, cudaStream_t st) {
  c->launches += 1;
  if (c->use_stream) {
    if (c->mixed)
      CK(launch_ras_apply_stream<float>(c->rs, rin, z, z32, c->errflag + 1, guard, st));
    else
      CK(launch_ras_apply_stream<double>(c->rs, rin, z, z32, c->errflag + 1, guard, st));
  } else if (c->mixed) {
    launch_ras_apply<float>(c->ras, (const float*)c->fac, rin, (float*)c->work, z, z32, guard, st);
  } else {
    launch_ras_apply<double>(c->ras, (const double*)c->fac, rin, (double*)c->work, z, z32, guard, st);
  }
}

void pc_apply(fsi_ctx* c, const double* rin, double* z) {
  int h = c->begin_phase(PH_PCAPPLY);
  pc_apply_on(c, rin, z, nullptr, nullptr, c->s);
  check_launch();
  c->end_phase(h, PH_PCAPPLY);
}

// One Arnoldi step j of the cycle for every problem (CGS2, normalisation,
// Givens), guarded by "some problem still active".
void arnoldi_step(fsi_ctx* c, int32_t j, const int* guard, cudaStream_t st) {
  const int64_t n = c->n;
  const int32_t m = c->m, ldh = m + 1, P = c->nprob;
  double* w = c->V + (int64_t)(j + 1) * n;
  int nk = 0;  // multi-dot kernels launched (one or two per call)
  if (c->opt.orth == 1) {
    // classical Gram-Schmidt with a second pass only where the first removed more
    // than 1 - 1/sqrt(2) of ||w|| (the pass-2 kernels are guarded by that test)
    double* hj = c->H + (int64_t)j * ldh + j + 1;
    nk += launch_seg_mdot(c->seg, j + 1, c->V, n, w, c->partial, c->hA, ldh, guard, st, 1);
    launch_seg_maxpy(c->seg, n, j + 1, c->V, n, c->hA, ldh, w, guard, st);
    launch_seg_norm(c->seg, w, c->partial, hj, ldh * m, guard, st);
    launch_seg_reorth_decide(P, c->hA + j + 1, hj, ldh * m, c->hB, ldh, j, c->active, c->reorth, st);
    nk += launch_seg_mdot(c->seg, j + 1, c->V, n, w, c->partial, c->hB, ldh, c->reorth, st);
    launch_seg_maxpy(c->seg, n, j + 1, c->V, n, c->hB, ldh, w, c->reorth, st);
    launch_seg_norm(c->seg, w, c->partial, hj, ldh * m, c->reorth, st);
    launch_seg_scale_inv(c->seg, n, w, hj, ldh * m, w, guard, st);
    launch_seg_givens(P, c->hA, c->hB, ldh, c->H, ldh, m, j, c->cs, c->sn, c->g, c->gres, c->gtarget, c->active,
                      c->kcols, c->anyact, st);
    c->launches += 7 + nk;
    return;
  }
  if (c->opt.orth == 0) {
    // classical Gram-Schmidt twice, the new norm from the second pass: dots;
    // update; dots with ||w||^2; norm = sqrt(||w||^2 - ||h2||^2); update and scale
    // in one sweep. Where that norm is unsafe the guarded kernels form it from the
    // updated vector.
    double* hj = c->H + (int64_t)j * ldh + j + 1;
    nk += launch_seg_mdot(c->seg, j + 1, c->V, n, w, c->partial, c->hA, ldh, guard, st);
    launch_seg_maxpy(c->seg, n, j + 1, c->V, n, c->hA, ldh, w, guard, st);
    nk += launch_seg_mdot(c->seg, j + 1, c->V, n, w, c->partial, c->hB, ldh, guard, st, 1);
    launch_seg_norm_pythagoras(P, c->hB, ldh, j, hj, (int64_t)ldh * m, c->gs_inv, c->gs_unsafe, c->reorth,
                               c->opt.fault_test == 2 ? 1 : 0, guard, st);
    launch_seg_maxpy(c->seg, n, j + 1, c->V, n, c->hB, ldh, w, guard, st, c->gs_inv);
    launch_seg_norm(c->seg, w, c->partial, c->gs_nrm, 1, c->reorth, st);
    launch_seg_norm_fix(P, c->gs_nrm, c->gs_unsafe, hj, (int64_t)ldh * m, c->gs_scal, c->reorth, st);
    launch_seg_scale_inv(c->seg, n, w, c->gs_scal, 1, w, c->reorth, st);
    launch_seg_givens(P, c->hA, c->hB, ldh, c->H, ldh, m, j, c->cs, c->sn, c->g, c->gres, c->gtarget, c->active,
                      c->kcols, c->anyact, st);
    c->launches += 7 + nk;
    return;
  }
  // orth 2: dots, update, dots, update, norm, scale
  nk += launch_seg_mdot(c->seg, j + 1, c->V, n, w, c->partial, c->hA, ldh, guard, st);
  launch_seg_maxpy(c->seg, n, j + 1, c->V, n, c->hA, ldh, w, guard, st);
  nk += launch_seg_mdot(c->seg, j + 1, c->V, n, w, c->partial, c->hB, ldh, guard, st);
  launch_seg_maxpy(c->seg, n, j + 1, c->V, n, c->hB, ldh, w, guard, st);
  // H[p][j+1][j] = ||w_p||, written in place (per-problem stride ldh * m), then w_p /= it
  launch_seg_norm(c->seg, w, c->partial, c->H + (int64_t)j * ldh + j + 1, ldh * m, guard, st);
  launch_seg_scale_inv(c->seg, n, w, c->H + (int64_t)j * ldh + j + 1, ldh * m, w, guard, st);
  launch_seg_givens(P, c->hA, c->hB, ldh, c->H, ldh, m, j, c->cs, c->sn, c->g, c->gres, c->gtarget, c->active,
                    c->kcols, c->anyact, st);
  c->launches += 5 + nk;
}

// The kernels of one restart cycle for every problem, from V_0 = r / ||r|| to
// the true residual of the updated iterates: c->rhs is b, c->dy is x, c->r the
// residual, c->beta[p] its norms on entry and on exit.
void cycle_kernels(fsi_ctx* c, cudaStream_t st) {
  const int64_t n = c->n;
  const int32_t m = c->m, ldh = m + 1, P = c->nprob;
  const int* guard = c->anyact;
  launch_seg_scale_inv(c->seg, n, c->r, c->beta, 1, c->V, nullptr, st);
  launch_seg_cycle_init(P, c->g, ldh, c->beta, c->gtarget, c->active, c->kcols, c->anyact, st);
  c->launches += 2;
  for (int32_t j = 0; j < m; ++j) {
    double* vj = c->V + (int64_t)j * n;
    double* zj = c->Z + (int64_t)j * n;
    double* w = c->V + (int64_t)(j + 1) * n;
    pc_apply_on(c, vj, zj, c->mixed ? c->zf : nullptr, guard, st);
    spmv_on(c, zj, c->mixed ? c->zf : nullptr, w, guard, st);
    arnoldi_step(c, j, guard, st);
  }
  launch_seg_lsq(P, c->H, ldh, m, c->kcols, c->g, c->ylsq, st);
  launch_seg_update_x(c->seg, n, c->Z, n, c->ylsq, m, c->kcols, c->dy, st);
  c->launches += 2;
  spmv_on(c, c->dy, nullptr, c->r, nullptr, st);
  launch_axpby(n, 1.0, c->rhs, -1.0, c->r, c->r, st);
  launch_seg_norm(c->seg, c->r, c->partial, c->beta, 1, nullptr, st);
  c->launches += 2;
}

void build_graph(fsi_ctx* c) {
  if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  const int64_t before = c->launches;
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  cycle_kernels(c, c->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  CK(e);
  c->graph = g;
  CK(cudaGraphInstantiate(&c->gexec, g, 0));
  c->graph_nodes = c->launches - before;
  c->launches = before;
}

// Right-preconditioned restarted flexible GMRES (FGMRES form: the preconditioned
// directions Z are stored, so an FP32 preconditioner is allowed), classical
// Gram-Schmidt applied twice, Givens rotations, run for every problem at once
// with its own Krylov scalars and stopping test; each restart cycle is one
// captured CUDA graph; the host reads the true residual norms once per cycle.
// Solves J x = b with b = c->rhs, x = c->dy. Each problem stops when
// ||b_p - J x_p|| <= gmres_rtol ||b_p||.
fsi_status gmres(fsi_ctx* c, fsi_solve_stats* st) {
  if (!c->have_jac) throw StatusError{FSI_ERR_ARG, "no Jacobian assembled"};
  if (c->pc_stale) pc_setup(c);
  const int64_t n = c->n;
  const int P = c->nprob;
  c->launches += 1;
  launch_fill(n, 0.0, c->dy, c->s);
  launch_copy(n, c->rhs, c->r, c->s);
  std::vector<double> b0, bcur, target(P);
  const double rnorm0 = norms(c, c->r, b0);
  for (int p = 0; p < P; ++p) target[p] = c->opt.gmres_rtol * b0[p];
  CK(cudaMemcpyAsync(c->gtarget, target.data(), sizeof(double) * P, cudaMemcpyHostToDevice, c->s));
  auto all_conv = [&](const std::vector<double>& bb) {
    for (int p = 0; p < P; ++p)
      if (bb[p] > target[p]) return false;
    return true;
  };
  bcur = b0;
  int32_t it = 0;
  bool conv = all_conv(bcur);
  if (c->use_graph && !c->gexec) build_graph(c);
  std::vector<int> kk(P);
  while (!conv && it < c->opt.gmres_maxit) {
    int h = c->begin_phase(PH_KRYLOV);
    if (c->use_graph) {
      CK(cudaGraphLaunch(c->gexec, c->s));
      c->launches += c->graph_nodes;
    } else {
      cycle_kernels(c, c->s);
    }
    check_launch();
    c->end_phase(h, PH_KRYLOV);
    double* hb = c->hbuf;
    CK(cudaMemcpyAsync(hb, c->beta, sizeof(double) * P, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(hb + P, c->kcols, sizeof(int) * P, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(hb + 2 * P, c->errflag + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    int werr = 0;
    std::memcpy(&werr, hb + 2 * P, sizeof(int32_t));
    if (werr) {
      CK(cudaMemsetAsync(c->errflag + 1, 0, sizeof(int32_t), c->s));
      throw StatusError{FSI_ERR_TIMEOUT, "a bounded wait in the preconditioner apply gave up"};
    }
    std::memcpy(kk.data(), hb + P, sizeof(int) * P);
    int kmax = 0;
    for (int p = 0; p < P; ++p) {
      bcur[p] = hb[p];
      kmax = std::max(kmax, kk[p]);
    }
    it += kmax;
    c->phase_n[PH_PCAPPLY] += kmax;
    c->phase_n[PH_SPMV] += kmax + 1;
    c->phase_n[PH_ORTH] += kmax;
    conv = all_conv(bcur);
    if (c->opt.verbose) {
      double tot = 0;
      for (double v : bcur) tot += v * v;
      std::fprintf(stderr, "    gmres cycle: %d its, |r| = %.3e\n", kmax, std::sqrt(tot));
    }
    if (kmax == 0) break;  // no progress possible (breakdown at the first step)
  }
  if (st) {
    double tot = 0;
    for (double v : bcur) tot += v * v;
    st->iterations = it;
    st->converged = conv ? 1 : 0;
    st->rnorm0 = rnorm0;
    st->rnorm = std::sqrt(tot);
  }
  return conv ? FSI_OK : FSI_ERR_LINEAR_DIVERGED;
}

void fill_defaults(fsi_options* o) {
  o->dt = 1e-3;
  o->newton_rtol = 1e-6;
  o->newton_atol = 1e-10;
  o->gmres_rtol = 1e-3;
  o->newton_maxit = 20;
  o->gmres_restart = 30;
  o->gmres_maxit = 1000;
  o->n_subdomains = 64;
  o->overlap = 1;
  o->precision = 0;
  o->jac_lag = 1;
  o->ilu_level = 1;
  o->threads_per_row = 32;
  o->ordering = 1;
  o->verbose = 0;
  o->fault_test = 0;
  o->factor_mode = 0;
  o->apply_mode = 0;
  o->stage_blocks = 0;
  o->stages = 0;
  o->orth = 0;
  o->jac_chunk = 0;
}

}  // namespace

extern "C" {

void fsi_default_options(fsi_options* o) {
  if (o) fill_defaults(o);
}

fsi_status fsi_create(const fsi_mesh* mesh, const fsi_material* mat, const fsi_bc* bc, int32_t n_problems,
                      const fsi_options* opts, void* cuda_stream, fsi_ctx** out) {
  if (out) *out = nullptr;
  if (!mesh || !mat || !bc || !out || n_problems < 1 || !mesh->X || !mesh->tets || !mesh->tet_domain ||
      !mesh->node_tag || mesh->n_nodes <= 0 || mesh->n_tets <= 0)
    return FSI_ERR_ARG;
  if (mesh->n_nodes >= (int64_t)INT32_MAX || mesh->n_tets * 16 >= (int64_t)INT32_MAX) return FSI_ERR_ARG;
  std::unique_ptr<fsi_ctx> c(new (std::nothrow) fsi_ctx());
  if (!c) return FSI_ERR_NOMEM;
  fsi_ctx* cp = c.get();
  fsi_status st = guarded(cp, [&]() -> fsi_status {
    fsi_options o;
    fill_defaults(&o);
    if (opts) {
      const fsi_options& q = *opts;
      if (q.dt > 0) o.dt = q.dt;
      if (q.newton_rtol > 0) o.newton_rtol = q.newton_rtol;
      if (q.newton_atol > 0) o.newton_atol = q.newton_atol;
      if (q.gmres_rtol > 0) o.gmres_rtol = q.gmres_rtol;
      if (q.newton_maxit > 0) o.newton_maxit = q.newton_maxit;
      if (q.gmres_restart > 0) o.gmres_restart = q.gmres_restart;
      if (q.gmres_maxit > 0) o.gmres_maxit = q.gmres_maxit;
      if (q.n_subdomains > 0) o.n_subdomains = q.n_subdomains;
      if (q.overlap >= 0) o.overlap = q.overlap;
      o.precision = q.precision;
      if (q.jac_lag > 0) o.jac_lag = q.jac_lag;
      if (q.ilu_level >= 0) o.ilu_level = q.ilu_level;
      o.threads_per_row = (q.threads_per_row == 16) ? 16 : 32;
      if (q.ordering >= 0 && q.ordering <= 3) o.ordering = q.ordering;
      o.verbose = q.verbose;
      o.fault_test = q.fault_test;
      if (q.factor_mode >= 0 && q.factor_mode <= 4) o.factor_mode = q.factor_mode;
      o.apply_mode = q.apply_mode;
      o.stage_blocks = q.stage_blocks;
      o.stages = q.stages;
      o.orth = q.orth;
      o.jac_chunk = q.jac_chunk;
    }
    if (o.jac_chunk < 0) throw StatusError{FSI_ERR_ARG, "jac_chunk must be >= 0"};
    if (o.orth < 0 || o.orth > 2) throw StatusError{FSI_ERR_ARG, "orth must be 0, 1 or 2"};
    if (o.apply_mode < 0 || o.apply_mode > 2) throw StatusError{FSI_ERR_ARG, "apply_mode must be 0, 1 or 2"};
    if (o.stage_blocks < 0) throw StatusError{FSI_ERR_ARG, "stage_blocks must be >= 0"};
    if (o.stages != 0 && (o.stages < 2 || o.stages > 8)) throw StatusError{FSI_ERR_ARG, "stages must be 0 or 2..8"};
    if (o.precision != 0 && o.precision != 1) throw StatusError{FSI_ERR_ARG, "precision must be 0 or 1"};
    if (o.ilu_level < 0 || o.ilu_level > 3) throw StatusError{FSI_ERR_ARG, "ilu_level must be 0..3"};
    if (o.gmres_restart > 64) throw StatusError{FSI_ERR_ARG, "gmres_restart must be <= 64"};
    cp->opt = o;
    cp->mat = *mat;
    cp->s = (cudaStream_t)cuda_stream;
    cp->mixed = o.precision == 1;
    cp->m = o.gmres_restart;
    cp->nprob = n_problems;
    const double mu_s = mat->E_s / (2.0 * (1.0 + mat->nu_s));
    const double lam_s = mat->E_s * mat->nu_s / ((1.0 + mat->nu_s) * (1.0 - 2.0 * mat->nu_s));
    cp->mc = MatConst{mat->rho_f, mat->mu_f, mat->rho_s, mat->eta_s, lam_s, mu_s, o.dt};

    const int64_t N = mesh->n_nodes, T0 = mesh->n_tets;
    // validate, then order tets fluid first
    std::vector<int32_t> tets, tet_src;
    tets.reserve(4 * T0);
    tet_src.reserve(T0);
    int64_t Tf = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int64_t t = 0; t < T0; ++t) {
        const uint8_t d = mesh->tet_domain[t];
        if (d > 1) throw StatusError{FSI_ERR_MESH, "tet_domain must be 0 or 1"};
        if (d != pass) continue;
        tet_src.push_back((int32_t)t);
        for (int a = 0; a < 4; ++a) {
          const int32_t v = mesh->tets[4 * t + a];
          if (v < 0 || v >= N) throw StatusError{FSI_ERR_MESH, "tet vertex index out of range"};
          tets.push_back(v);
        }
        if (pass == 0) ++Tf;
      }
    // positive orientation check (reference configuration)
    for (int64_t t = 0; t < T0; ++t) {
      const double* x0 = mesh->X + 3 * (int64_t)tets[4 * t];
      double e[3][3];
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) e[k][i] = mesh->X[3 * (int64_t)tets[4 * t + k + 1] + i] - x0[i];
      const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                         e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                         e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
      if (!(det > 0)) throw StatusError{FSI_ERR_MESH, "degenerate or negatively oriented tet"};
    }
    // node flags: constraint rows and row routing
    std::vector<uint32_t> flag(N, 0);
    std::vector<int32_t> prob(N, 0);
    int64_t nfluid = 0;
    for (int64_t i = 0; i < N; ++i) {
      const uint32_t tg = mesh->node_tag[i];
      const int32_t p = mesh->node_problem ? mesh->node_problem[i] : 0;
      if (p < 0 || p >= n_problems) throw StatusError{FSI_ERR_MESH, "node_problem out of range"};
      if (i > 0 && p < prob[i - 1])
        throw StatusError{FSI_ERR_MESH, "node_problem must be non-decreasing (problems stored one after another)"};
      prob[i] = p;
      const bool fl = tg & FSI_TAG_FLUID, wl = tg & FSI_TAG_WALL, itf = tg & FSI_TAG_INTERFACE;
      uint32_t f = 0;
      if (fl) f |= NF_FLUID, ++nfluid;
      if (itf) f |= NF_ITF;
      const bool inlet = fl && (tg & FSI_TAG_INLET);
      if (inlet) f |= NF_U_INLET;
      else if (itf) f |= NF_U_KIN;
      if (wl && !fl) f |= NF_U_IDENT | NF_P_IDENT;
      if (tg & (FSI_TAG_INLET | FSI_TAG_OUTLET | FSI_TAG_WALL_END)) f |= NF_D_ZERO;
      if (wl && bc[p].rigid_wall) f |= NF_D_ZERO;
      if (!fl && !wl) f |= NF_U_IDENT | NF_P_IDENT | NF_D_ZERO;  // isolated node
      flag[i] = f;
    }
    // inner-wall faces (fluid tet against wall tet), matched by sorted vertex
    // triples among the faces whose three vertices are interface nodes
    std::vector<int64_t> wface;
    std::vector<int64_t> wfb(n_problems + 1, 0);
    {
      struct FaceKey {
        int32_t a, b, c;
        int64_t tf;  // 4 * internal tet + opposite vertex
      };
      std::vector<FaceKey> cand;
      for (int64_t t = 0; t < T0; ++t)
        for (int f = 0; f < 4; ++f) {
          int32_t v[3], k = 0;
          for (int a = 0; a < 4; ++a)
            if (a != f) v[k++] = tets[4 * t + a];
          if (!(mesh->node_tag[v[0]] & mesh->node_tag[v[1]] & mesh->node_tag[v[2]] & FSI_TAG_INTERFACE)) continue;
          std::sort(v, v + 3);
          cand.push_back({v[0], v[1], v[2], 4 * t + f});
        }
      std::sort(cand.begin(), cand.end(), [](const FaceKey& x, const FaceKey& y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        if (x.c != y.c) return x.c < y.c;
        return x.tf < y.tf;
      });
      for (size_t i = 0; i + 1 < cand.size(); ++i) {
        const FaceKey &x = cand[i], &y = cand[i + 1];
        if (x.a != y.a || x.b != y.b || x.c != y.c) continue;
        const bool fx = (x.tf >> 2) < Tf, fy = (y.tf >> 2) < Tf;
        if (fx != fy) wface.push_back(fx ? x.tf : y.tf);
        ++i;
      }
      auto pr = [&](int64_t tf) { return prob[tets[4 * (tf >> 2)]]; };
      std::sort(wface.begin(), wface.end(), [&](int64_t x, int64_t y) {
        const int32_t px = pr(x), py = pr(y);
        return px != py ? px < py : x < y;
      });
      for (int64_t tf : wface) wfb[pr(tf) + 1]++;
      for (int p = 0; p < n_problems; ++p) wfb[p + 1] += wfb[p];
    }
    std::vector<double> inl((size_t)INLET_STRIDE * n_problems);
    for (int p = 0; p < n_problems; ++p) {
      double* q = &inl[(size_t)INLET_STRIDE * p];
      const double nn = std::sqrt(bc[p].normal[0] * bc[p].normal[0] + bc[p].normal[1] * bc[p].normal[1] +
                                  bc[p].normal[2] * bc[p].normal[2]);
      if (!(nn > 0) || !(bc[p].radius > 0)) throw StatusError{FSI_ERR_ARG, "inlet normal/radius invalid"};
      for (int i = 0; i < 3; ++i) q[i] = bc[p].center[i], q[3 + i] = bc[p].normal[i] / nn;
      q[6] = bc[p].radius;
      q[7] = bc[p].peak;
      q[8] = bc[p].amp;
      q[9] = bc[p].freq;
      q[10] = bc[p].phase;
    }
    cp->N = N;
    cp->T = T0;
    cp->Tf = Tf;
    cp->n = 7 * N;
    cp->nunk = 7 * nfluid + 3 * (N - nfluid);

    // symbolic setup
    BsrPattern P = build_pattern(N, tets);
    std::vector<int64_t> bptr, nptr;
    std::vector<int32_t> bsrc, nsrc;
    build_gather(P, tets, bptr, bsrc, nptr, nsrc);
    cp->nnzb = (int64_t)P.col.size();
    std::vector<uint8_t> rank(N);
    for (int64_t i = 0; i < N; ++i)
      rank[i] = (flag[i] & NF_ITF) ? 1 : ((flag[i] & NF_FLUID) ? 0 : 2);
    cp->plan = build_ras(P, mesh->X, N, mesh->node_problem, n_problems, o.n_subdomains, o.overlap, o.ilu_level,
                         o.ordering, rank.data());

    // device copies
    std::vector<double> Xv(mesh->X, mesh->X + 3 * N);
    cp->X = cp->upload(Xv);
    cp->tets = cp->upload(tets);
    cp->nflag = cp->upload(flag);
    cp->nprobid = cp->upload(prob);
    cp->inlet = cp->upload(inl);
    cp->nptr = cp->upload(nptr);
    cp->nsrc = cp->upload(nsrc);
    cp->bptr = cp->upload(bptr);
    cp->bsrc = cp->upload(bsrc);
    cp->row_ptr = cp->upload(P.row_ptr);
    cp->col = cp->upload(P.col);
    cp->diag = cp->upload(P.diag);
    const size_t vs = cp->mixed ? sizeof(float) : sizeof(double);
    cp->Fe = cp->dalloc<double>(28 * T0);
    {
      std::vector<double> xl(12 * T0);
      for (int64_t t = 0; t < T0; ++t)
        for (int a = 0; a < 4; ++a)
          for (int i = 0; i < 3; ++i)
            xl[12 * t + 3 * a + i] = mesh->X[3 * (int64_t)tets[4 * t + a] + i] - mesh->X[3 * (int64_t)tets[4 * t] + i];
      if (cp->mixed) {
        std::vector<float> xf(xl.begin(), xl.end());
        cp->Xl = cp->upload(xf);
        cp->y32 = cp->dalloc<float>(3 * 7 * N);
      } else {
        cp->Xl = cp->upload(xl);
      }
    }
    // the element Jacobian buffer Ke and the subdomain factors share one
    // allocation (sized below, once the factor size is known): Ke is live only
    // inside a Jacobian assembly, the factors only from the preconditioner
    // setup that follows it (every assembly marks the preconditioner stale)
    cp->vals = cp->dalloc<char>((int64_t)(49 * vs) * cp->nnzb);
    CK(cudaMemsetAsync(cp->vals, 0, 49 * vs * cp->nnzb, cp->s));
    cp->mesh = MeshDev{N, T0, Tf, cp->X, cp->tets, cp->nflag, cp->nprobid, cp->inlet};
    cp->nwss = (int64_t)wface.size();
    cp->wface = cp->upload(wface);
    cp->wfb = cp->upload(wfb);
    cp->wma = cp->dalloc<double>(std::max<int64_t>(cp->nwss, 1));
    cp->wa = cp->dalloc<double>(std::max<int64_t>(cp->nwss, 1));
    cp->wsawss = cp->dalloc<double>(n_problems);
    cp->wface_host.resize(2 * wface.size());
    for (size_t i = 0; i < wface.size(); ++i) {
      cp->wface_host[2 * i] = tet_src[wface[i] >> 2];
      cp->wface_host[2 * i + 1] = (int32_t)(wface[i] & 3);
    }

    const int64_t n = 7 * N;
    cp->yn = cp->dalloc<double>(n);
    cp->ynm1 = cp->dalloc<double>(n);
    cp->ynm2 = cp->dalloc<double>(n);
    CK(cudaMemsetAsync(cp->yn, 0, n * 8, cp->s));
    CK(cudaMemsetAsync(cp->ynm1, 0, n * 8, cp->s));
    CK(cudaMemsetAsync(cp->ynm2, 0, n * 8, cp->s));
    cp->yk = cp->dalloc<double>(n);
    cp->ytr = cp->dalloc<double>(n);
    cp->F = cp->dalloc<double>(n);
    cp->Ft = cp->dalloc<double>(n);
    cp->dy = cp->dalloc<double>(n);
    cp->rhs = cp->dalloc<double>(n);
    const int32_t m = cp->m;
    cp->V = cp->dalloc<double>((int64_t)(m + 1) * n);
    cp->Z = cp->dalloc<double>((int64_t)m * n);
    const int64_t NP = n_problems;
    cp->H = cp->dalloc<double>(NP * (m + 1) * m);
    cp->g = cp->dalloc<double>(NP * (m + 1));
    cp->cs = cp->dalloc<double>(NP * m);
    cp->sn = cp->dalloc<double>(NP * m);
    cp->ylsq = cp->dalloc<double>(NP * m);
    cp->hA = cp->dalloc<double>(NP * (m + 1));
    cp->hB = cp->dalloc<double>(NP * (m + 1));
    // reduction chunks: each problem's dofs cut into chunks of at most CH dofs
    {
      const int64_t CH = std::max<int64_t>(1024, (7 * N + 1215) / 1216);
      std::vector<int64_t> cb{0}, pc{0};
      std::vector<int64_t> pstart(NP + 1, 0);
      for (int64_t i = 0; i < N; ++i) pstart[prob[i] + 1]++;
      for (int64_t q = 0; q < NP; ++q) pstart[q + 1] += pstart[q];
      for (int64_t q = 0; q < NP; ++q) {
        const int64_t a0 = 7 * pstart[q], a1 = 7 * pstart[q + 1];
        for (int64_t x = a0; x < a1; x += CH) cb.push_back(std::min(a1, x + CH));
        pc.push_back((int64_t)cb.size() - 1);
      }
      cp->seg.P = (int32_t)NP;
      cp->seg.n_chunks = (int64_t)cb.size() - 1;
      cp->seg.chunk_beg = cp->upload(cb);
      cp->seg.prob_chunk = cp->upload(pc);
      cp->seg.node_prob = cp->nprobid;
      cp->partial = cp->dalloc<double>(cp->seg.n_chunks * (m + 1));
      cp->seg.counter = cp->dalloc<int>(NP * SEG_GROUPS);
      CK(cudaMemsetAsync(cp->seg.counter, 0, sizeof(int) * NP * SEG_GROUPS, cp->s));
    }
    cp->beta = cp->dalloc<double>(n_problems);
    cp->gres = cp->dalloc<double>(n_problems);
    cp->active = cp->dalloc<int>(n_problems);
    cp->kcols = cp->dalloc<int>(n_problems);
    cp->anyact = cp->dalloc<int>(1);
    cp->reorth = cp->dalloc<int>(1);
    cp->gs_inv = cp->dalloc<double>(n_problems);
    cp->gs_nrm = cp->dalloc<double>(n_problems);
    cp->gs_scal = cp->dalloc<double>(n_problems);
    cp->gs_unsafe = cp->dalloc<int>(n_problems);
    cp->pmask = cp->dalloc<int>(n_problems);
    cp->palpha = cp->dalloc<double>(n_problems);
    cp->r = cp->dalloc<double>(n);
    cp->gtarget = cp->dalloc<double>(n_problems);
    cp->zf = cp->dalloc<float>(n);
    CK(cudaMallocHost(&cp->hbuf, sizeof(double) * (3 * n_problems + 16)));

    // Schwarz plan
    RasPlan& R = cp->plan;
    RasDev rd{};
    rd.np = R.np;
    rd.sd_row = cp->upload(R.sd_row);
    rd.gnode = cp->upload(R.gnode);
    rd.owned = cp->upload(R.owned);
    rd.row_ptr = cp->upload(R.row_ptr);
    rd.col = cp->upload(R.col);
    rd.gblk = cp->upload(R.gblk);
    rd.diag = cp->upload(R.diag);
    rd.lent_ptr = cp->upload(R.lent_ptr);
    rd.lent_pos = cp->upload(R.lent_pos);
    rd.lent_kdiag = cp->upload(R.lent_kdiag);
    rd.upd_ptr = cp->upload(R.upd_ptr);
    rd.upd_tgt = cp->upload(R.upd_tgt);
    rd.upd_src = cp->upload(R.upd_src);
    rd.sd_lvlL = cp->upload(R.sd_lvlL);
    rd.sd_lvlU = cp->upload(R.sd_lvlU);
    rd.lvlL_ptr = cp->upload(R.lvlL_ptr);
    rd.lvlU_ptr = cp->upload(R.lvlU_ptr);
    rd.lvlL_rows = cp->upload(R.lvlL_rows);
    rd.lvlU_rows = cp->upload(R.lvlU_rows);
    rd.nblocks = (int64_t)R.col.size();
    {
      int64_t mb = 1;
      for (size_t q = 0; q + 1 < R.row_ptr.size(); ++q) mb = std::max(mb, R.row_ptr[q + 1] - R.row_ptr[q]);
      rd.max_row_blocks = (int32_t)mb;
      int64_t ml = 1, mu = 1, me = 1;
      for (size_t q = 0; q + 1 < R.lent_ptr.size(); ++q) {
        ml = std::max(ml, R.lent_ptr[q + 1] - R.lent_ptr[q]);
        mu = std::max(mu, R.upd_ptr[R.lent_ptr[q + 1]] - R.upd_ptr[R.lent_ptr[q]]);
      }
      for (size_t e = 0; e + 1 < R.upd_ptr.size(); ++e) me = std::max(me, R.upd_ptr[e + 1] - R.upd_ptr[e]);
      rd.max_row_lent = (int32_t)ml;
      rd.max_row_upd = (int32_t)mu;
      rd.max_entry_upd = (int32_t)me;
      rd.sd_depth = cp->upload(R.sd_depth);
      rd.sd_item = cp->upload(R.sd_item);
      rd.item_row = cp->upload(R.item_row);
      rd.max_depth = R.max_depth;
      auto fits = [&](int mode) { return cp->mixed ? ras_factor_fits<float>(rd, mode) : ras_factor_fits<double>(rd, mode); };
      // automatic: nested-dissection groups when the subdomains are dissected and
      // the groups' rows fit, else the row-only sequential kernel
      const int want = o.factor_mode > 0 ? o.factor_mode - 1 : (R.max_depth > 0 && fits(3) ? 3 : 2);
      rd.factor_mode = want;
      if (fits(2) && !fits(want)) throw StatusError{FSI_ERR_ARG, "factor_mode needs more shared memory than fits"};
      if (!fits(2)) {
        char msg[192];
        std::snprintf(msg, sizeof msg,
                      "ILU rows too long for the shared-memory factorisation (%d blocks in the longest row; "
                      "use a lower fill level or more subdomains)",
                      rd.max_row_blocks);
        throw StatusError{FSI_ERR_ARG, msg};
      }

    }
    cp->ras = rd;
    // the Jacobian is assembled in chunks of tets so that Ke needs no more than
    // the factors' size (or 1 GB): the shared buffer is as large as the factors
    {
      const int64_t fac_bytes = (int64_t)(49 * vs) * rd.nblocks;
      const int64_t per_tet = (int64_t)(784 * vs);
      const int64_t room = std::max<int64_t>(fac_bytes, (int64_t)1 << 30);
      cp->ke_tets = std::max<int64_t>(1, std::min<int64_t>(T0, room / per_tet));
      if (o.jac_chunk > 0) cp->ke_tets = std::min<int64_t>(T0, o.jac_chunk);
      cp->fac = cp->dalloc<char>(std::max<int64_t>(fac_bytes, per_tet * cp->ke_tets));
      cp->Ke = cp->fac;
    }
    cp->work = cp->dalloc<char>((int64_t)(7 * vs) * (int64_t)R.gnode.size());
    cp->errflag = cp->dalloc<int32_t>(2);
    CK(cudaMemsetAsync(cp->errflag, 0, 2 * sizeof(int32_t), cp->s));

    // packed factor streams for the TMA-fed apply
    {
      std::vector<int64_t> Lcnt(R.gnode.size()), Ucnt(R.gnode.size()), Loff(R.np + 1), Uoff(R.np + 1), Lsrc, Usrc,
          Upiv;
      std::vector<int32_t> Lcol, Ucol;
      int64_t maxblk = 1;
      for (int32_t sd = 0; sd < R.np; ++sd) {
        const int64_t a = R.sd_row[sd], b = R.sd_row[sd + 1];
        Loff[sd] = (int64_t)Lsrc.size();
        for (int64_t q = a; q < b; ++q) {
          for (int64_t e = R.row_ptr[q]; e < R.diag[q]; ++e) {
            Lsrc.push_back(e);
            Lcol.push_back((int32_t)(R.col[e] - a));
          }
          Lcnt[q] = R.diag[q] - R.row_ptr[q];
          maxblk = std::max(maxblk, Lcnt[q]);
        }
        Uoff[sd] = (int64_t)Usrc.size();
        for (int64_t q = b - 1; q >= a; --q) {
          Usrc.push_back(R.diag[q]);
          Ucol.push_back((int32_t)(q - a));
          Upiv.push_back(-1);
          for (int64_t e = R.diag[q] + 1; e < R.row_ptr[q + 1]; ++e) {
            Usrc.push_back(e);
            Ucol.push_back((int32_t)(R.col[e] - a));
            Upiv.push_back(R.diag[q]);
          }
          Ucnt[q] = R.row_ptr[q + 1] - R.diag[q];
          maxblk = std::max(maxblk, Ucnt[q]);
        }
      }
      Loff[R.np] = (int64_t)Lsrc.size();
      Uoff[R.np] = (int64_t)Usrc.size();
      // per nested-dissection item: its first / end block in the subdomain's L
      // stream (rows ascending) and U stream (rows descending)
      std::vector<int32_t> iblk(4 * R.item_row.size());
      for (int32_t sd = 0; sd < R.np; ++sd) {
        const int64_t a = R.sd_row[sd], b = R.sd_row[sd + 1];
        int64_t Ltot = 0, Utot = 0;
        for (int64_t q = a; q < b; ++q) Utot += Ucnt[q];
        int64_t row = 0;
        for (int64_t k = R.sd_item[sd]; k < R.sd_item[sd + 1]; ++k) {
          const int64_t end = R.item_row[k];
          int64_t Lb = 0, Ub = 0;  // blocks of rows [row, end)
          for (int64_t q = a + row; q < a + end; ++q) Lb += Lcnt[q], Ub += Ucnt[q];
          int64_t Uafter = 0;      // U blocks of rows at and after `end` (they come first)
          for (int64_t q = a + end; q < b; ++q) Uafter += Ucnt[q];
          iblk[4 * k + 0] = (int32_t)Ltot;
          iblk[4 * k + 1] = (int32_t)(Ltot + Lb);
          iblk[4 * k + 2] = (int32_t)Uafter;
          iblk[4 * k + 3] = (int32_t)(Uafter + Ub);
          Ltot += Lb;
          row = end;
        }
        (void)Utot;
      }
      RasStreamDev& rs = cp->rs;
      rs.sd_depth = cp->upload(R.sd_depth);
      rs.sd_item = cp->upload(R.sd_item);
      rs.item_row = cp->upload(R.item_row);
      rs.item_blk = cp->upload(iblk);
      rs.max_depth = R.max_depth;
      rs.np = R.np;
      rs.sd_row = rd.sd_row;
      rs.gnode = rd.gnode;
      rs.owned = rd.owned;
      rs.L_cnt = cp->upload(Lcnt);
      rs.U_cnt = cp->upload(Ucnt);
      rs.L_off = cp->upload(Loff);
      rs.U_off = cp->upload(Uoff);
      rs.nL = (int64_t)Lsrc.size();
      rs.nU = (int64_t)Usrc.size();
      rs.Lsrc = cp->upload(Lsrc);
      rs.Lcol = cp->upload(Lcol);
      rs.Usrc = cp->upload(Usrc);
      rs.Ucol = cp->upload(Ucol);
      rs.Upiv = cp->upload(Upiv);
      // stage geometry: NST (2) stages of SB blocks. The target is ceil(np / 152)
      // CTAs per SM, at most 8 (all subdomains resident at once up to 1,216), and
      // the ring gets what the shared memory per CTA leaves after the vector; the
      // stage_blocks and stages options override the choice
      const int vsz = cp->mixed ? 4 : 8, stride = 56;  // packed block: 7 rows of 8 values
      int nst = o.stages > 0 ? o.stages : 2;
      const int64_t W = (int64_t)1 << R.max_depth;  // warps (rings) per CTA
      const int64_t per_sm = std::min<int64_t>(8, (R.np + 151) / 152);
      const int64_t fixed = 128 * ((W * 64 + 127) / 128) + 8 * R.max_rows * vsz + 4 * R.max_rows + 16 + 1024;
      // (the budget never exceeds the 200 KB the streamed apply may use)
      const int64_t budget = std::min<int64_t>((int64_t)(227 * 1024) / per_sm, (int64_t)(200 * 1024));
      int64_t SB = (budget - fixed) / (W * nst * stride * vsz);
      SB = std::max<int64_t>(W > 1 ? 8 : 16, std::min<int64_t>(SB, cp->mixed ? 128 : 64));
      if (o.stage_blocks > 0) SB = o.stage_blocks;
      rs.nst = nst;
      rs.stall = o.fault_test == 1 ? 1 : 0;
      rs.stage_blocks = (int32_t)SB;
      rs.max_rows = R.max_rows;
      const size_t sm = cp->mixed ? ras_stream_smem<float>(rs) : ras_stream_smem<double>(rs);
      // (the apply keeps each row's block counts as 16-bit values in shared memory)
      const bool fits = sm <= 200 * 1024 && maxblk <= 65535;
      if (o.apply_mode == 1 && !fits)
        throw StatusError{FSI_ERR_ARG, "apply_mode 1: the streamed apply's shared memory does not fit"};
      cp->use_stream = o.apply_mode == 2 ? false : fits;
      if (cp->use_stream) {
        CK(cp->mixed ? ras_stream_init<float>(rs) : ras_stream_init<double>(rs));
        rs.Lpack = cp->dalloc<char>((int64_t)(stride * vs) * std::max<int64_t>(rs.nL, 1));
        rs.Upack = cp->dalloc<char>((int64_t)(stride * vs) * std::max<int64_t>(rs.nU, 1));
      }
    }
    CK(cudaStreamSynchronize(cp->s));
    return FSI_OK;
  });
  if (st != FSI_OK) {
    std::fprintf(stderr, "fsi_create: %s\n", cp->err.c_str());
    fsi_destroy(c.release());
    return st;
  }
  *out = c.release();
  return FSI_OK;
}

fsi_status fsi_destroy(fsi_ctx* c) {
  if (!c) return FSI_OK;
  if (c->s) cudaStreamSynchronize(c->s);
  else cudaDeviceSynchronize();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (void* p : c->allocs) cudaFree(p);
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  if (c->hbuf) cudaFreeHost(c->hbuf);
  delete c;
  return FSI_OK;
}

fsi_status fsi_set_state(fsi_ctx* c, const double* y_n, const double* y_nm1, const double* y_nm2, double t) {
  if (!c || !y_n) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    CK(cudaMemcpyAsync(c->yn, y_n, c->n * 8, cudaMemcpyDeviceToDevice, c->s));
    CK(cudaMemcpyAsync(c->ynm1, y_nm1 ? y_nm1 : y_n, c->n * 8, cudaMemcpyDeviceToDevice, c->s));
    CK(cudaMemcpyAsync(c->ynm2, y_nm2 ? y_nm2 : (y_nm1 ? y_nm1 : y_n), c->n * 8, cudaMemcpyDeviceToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    c->t = t;
    return FSI_OK;
  });
}

fsi_status fsi_get_state(fsi_ctx* c, double* y_n, double* t) {
  if (!c) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    if (y_n) CK(cudaMemcpyAsync(y_n, c->yn, c->n * 8, cudaMemcpyDeviceToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (t) *t = c->t;
    return FSI_OK;
  });
}

fsi_status fsi_residual(fsi_ctx* c, const double* y, double* F) {
  if (!c || !y || !F) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    residual(c, y, F);
    CK(cudaStreamSynchronize(c->s));
    return FSI_OK;
  });
}

fsi_status fsi_jacobian(fsi_ctx* c, const double* y) {
  if (!c || !y) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    jacobian(c, y);
    CK(cudaStreamSynchronize(c->s));
    return FSI_OK;
  });
}

fsi_status fsi_jacobian_export(fsi_ctx* c, int32_t* row_ptr, int32_t* col, double* vals) {
  if (!c) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    if (row_ptr) {
      std::vector<int64_t> rp(c->N + 1);
      CK(cudaMemcpy(rp.data(), c->row_ptr, (c->N + 1) * 8, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i <= c->N; ++i) row_ptr[i] = (int32_t)rp[i];
    }
    if (col) CK(cudaMemcpy(col, c->col, c->nnzb * 4, cudaMemcpyDeviceToHost));
    if (vals) {
      CK(cudaStreamSynchronize(c->s));
      if (c->mixed) {
        std::vector<float> v(49 * c->nnzb);
        CK(cudaMemcpy(v.data(), c->vals, v.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < v.size(); ++i) vals[i] = v[i];
      } else {
        CK(cudaMemcpy(vals, c->vals, 49 * c->nnzb * 8, cudaMemcpyDeviceToHost));
      }
    }
    return FSI_OK;
  });
}

fsi_status fsi_spmv(fsi_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    if (!c->have_jac) throw StatusError{FSI_ERR_ARG, "no Jacobian assembled"};
    spmv(c, x, y);
    CK(cudaStreamSynchronize(c->s));
    return FSI_OK;
  });
}

fsi_status fsi_pc_apply(fsi_ctx* c, const double* r, double* z) {
  if (!c || !r || !z) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    if (!c->have_jac) throw StatusError{FSI_ERR_ARG, "no Jacobian assembled"};
    if (c->pc_stale) pc_setup(c);
    pc_apply(c, r, z);
    int32_t werr = 0;
    CK(cudaMemcpyAsync(&c->hbuf[5], c->errflag + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    std::memcpy(&werr, &c->hbuf[5], sizeof(int32_t));
    if (werr) {
      CK(cudaMemsetAsync(c->errflag + 1, 0, sizeof(int32_t), c->s));
      CK(cudaStreamSynchronize(c->s));
      throw StatusError{FSI_ERR_TIMEOUT, "a bounded wait in the preconditioner apply gave up"};
    }
    return FSI_OK;
  });
}

fsi_status fsi_linear_solve(fsi_ctx* c, const double* rhs, double* x, fsi_solve_stats* stats) {
  if (!c || !rhs || !x) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    CK(cudaMemcpyAsync(c->rhs, rhs, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    fsi_status s = gmres(c, stats);
    CK(cudaMemcpyAsync(x, c->dy, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (s != FSI_OK) c->err = "GMRES reached its iteration limit";
    return s;
  });
}

fsi_status fsi_step(fsi_ctx* c, fsi_step_stats* stats) {
  if (!c) return FSI_ERR_ARG;
  fsi_step_stats S{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fsi_status st = guarded(c, [&]() -> fsi_status {
    c->timing = stats != nullptr;
    for (double& v : c->phase_ms) v = 0.0;
    for (int32_t& v : c->phase_n) v = 0;
    c->launches = 0;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, c->s));
    const int64_t n = c->n;
    const int P = c->nprob;
    launch_copy(n, c->yn, c->yk, c->s);
    residual(c, c->yk, c->F);
    S.residual_evaluations++;
    // Newton per problem (Eq. 11-12): every problem has its own norm, stopping
    // test and line-search step; converged problems keep their iterate
    std::vector<double> nf, nf0, nft;
    double tot = norms(c, c->F, nf);
    nf0 = nf;
    S.fnorm0 = tot;
    if (!std::isfinite(tot)) throw StatusError{FSI_ERR_NONFINITE, "non-finite residual"};
    const double stall = 1e-8;
    std::vector<int> conv(P, 0), pend(P, 0);
    std::vector<double> alpha(P, 0.0);
    auto test_conv = [&](int p) { return nf[p] <= c->opt.newton_rtol * nf0[p] || nf[p] <= c->opt.newton_atol; };
    for (int p = 0; p < P; ++p) conv[p] = test_conv(p);
    auto all_done = [&]() {
      for (int p = 0; p < P; ++p)
        if (!conv[p]) return false;
      return true;
    };
    int32_t it = 0;
    int32_t jac_it = -1;  // iteration whose iterate the current Jacobian was evaluated at
    bool refresh = false;  // a line search failed on a lagged Jacobian: evaluate it again here
    while (!all_done()) {
      if (it >= c->opt.newton_maxit) throw StatusError{FSI_ERR_DIVERGED, "Newton reached its iteration limit"};
      if (jac_it < 0 || it - jac_it >= c->opt.jac_lag || refresh) {
        jacobian(c, c->yk);
        S.jacobian_evaluations++;
        jac_it = it;
        refresh = false;
      }
      CK(cudaMemcpyAsync(c->pmask, conv.data(), sizeof(int) * P, cudaMemcpyHostToDevice, c->s));
      c->launches += 1;
      launch_seg_neg_masked(c->seg, n, c->F, c->pmask, c->rhs, c->s);   // rhs = -F on unconverged problems
      fsi_solve_stats ls{};
      fsi_status lst = gmres(c, &ls);
      if (lst != FSI_OK && lst != FSI_ERR_LINEAR_DIVERGED) return lst;
      S.linear_iterations += ls.iterations;
      if (c->opt.verbose)
        std::fprintf(stderr, "  newton %d: |F| = %.6e, gmres %d its (%.2e -> %.2e)\n", it, tot, ls.iterations,
                     ls.rnorm0, ls.rnorm);
      // backtracking line search, per problem
      for (int p = 0; p < P; ++p) {
        alpha[p] = conv[p] ? 0.0 : 1.0;
        pend[p] = !conv[p];
      }
      bool any_pending = true, retry = false;
      while (any_pending && !retry) {
        CK(cudaMemcpyAsync(c->palpha, alpha.data(), sizeof(double) * P, cudaMemcpyHostToDevice, c->s));
        c->launches += 1;
        launch_seg_axpy(c->seg, n, c->yk, c->palpha, c->dy, c->ytr, c->s);
        residual(c, c->ytr, c->Ft);
        S.residual_evaluations++;
        norms(c, c->Ft, nft);
        any_pending = false;
        for (int p = 0; p < P; ++p) {
          if (!pend[p]) continue;
          if (std::isfinite(nft[p]) && nft[p] <= (1.0 - 1e-4 * alpha[p]) * nf[p]) {
            pend[p] = 0;
            continue;
          }
          alpha[p] *= 0.5;
          if (alpha[p] < 1.0 / 1024.0) {
            if (nf[p] <= stall * nf0[p]) {  // |F_p| sits at the rounding floor of its assembly
              alpha[p] = 0.0;
              conv[p] = 1;
              pend[p] = 0;
              continue;
            }
            // a direction from a Jacobian of an earlier iterate (Jacobian lag) may
            // not descend: evaluate the Jacobian here and redo this iteration once
            if (jac_it != it) {
              retry = true;
              break;
            }
            throw StatusError{FSI_ERR_LINESEARCH, "backtracking line search found no sufficient decrease"};
          }
          any_pending = true;
        }
      }
      if (retry) {
        refresh = true;
        continue;
      }
      std::swap(c->yk, c->ytr);
      std::swap(c->F, c->Ft);
      for (int p = 0; p < P; ++p) {
        if (conv[p]) continue;
        const bool stalled = nft[p] > 0.5 * nf[p] && nft[p] <= stall * nf0[p];
        nf[p] = nft[p];
        conv[p] = test_conv(p) || stalled;
      }
      tot = 0.0;
      for (int p = 0; p < P; ++p) tot += nf[p] * nf[p];
      tot = std::sqrt(tot);
      ++it;
    }
    S.newton_iterations = it;
    S.fnorm = tot;
    S.converged = 1;
    // shift time levels: y_{n-2} <- y_{n-1} <- y_n <- y
    double* old2 = c->ynm2;
    c->ynm2 = c->ynm1;
    c->ynm1 = c->yn;
    c->yn = c->yk;
    c->yk = old2;
    c->t += c->opt.dt;
    CK(cudaEventRecord(e1, c->s));
    c->resolve_phases();
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    S.t_total = ms;
    return FSI_OK;
  });
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->spans.clear();
  c->evused = 0;
  c->timing = false;
  S.t_funceval = c->phase_ms[PH_FUNC];
  S.t_jaceval = c->phase_ms[PH_JAC];
  S.t_pcsetup = c->phase_ms[PH_PCSETUP];
  S.t_pcapply = c->phase_ms[PH_PCAPPLY];
  S.t_spmv = c->phase_ms[PH_SPMV];
  S.t_orth = c->phase_ms[PH_ORTH];
  S.t_krylov = c->phase_ms[PH_KRYLOV];
  S.n_funceval = c->phase_n[PH_FUNC];
  S.n_jaceval = c->phase_n[PH_JAC];
  S.n_pcsetup = c->phase_n[PH_PCSETUP];
  S.n_pcapply = c->phase_n[PH_PCAPPLY];
  S.n_spmv = c->phase_n[PH_SPMV];
  S.n_orth = c->phase_n[PH_ORTH];
  S.kernel_launches = c->launches;
  if (stats) *stats = S;
  return st;
}

fsi_status fsi_get_info(const fsi_ctx* c, fsi_info* info) {
  if (!c || !info) return FSI_ERR_ARG;
  info->n_nodes = c->N;
  info->n_tets = c->T;
  info->n_unknowns = c->nunk;
  info->nnzb = c->nnzb;
  info->n_fluid_tets = c->Tf;
  info->n_wall_tets = c->T - c->Tf;
  info->n_problems = c->nprob;
  info->n_subdomains = c->plan.np;
  info->factor_blocks = (int64_t)c->plan.col.size();
  info->factor_rows = (int64_t)c->plan.gnode.size();
  info->max_levels = c->plan.max_levels;
  info->device_bytes = c->dev_bytes;
  info->n_wss_faces = c->nwss;
  info->nd_depth = c->plan.max_depth;
  info->apply_kernel = c->use_stream ? 1 : 2;
  return FSI_OK;
}

fsi_status fsi_wss(fsi_ctx* c, const double* y, double* wss, double* sawss) {
  if (!c) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    if (!y) throw StatusError{FSI_ERR_ARG, "y is null"};
    launch_wss(c->mesh, c->mat.mu_f, c->nwss, c->wface, c->wfb, c->nprob, y, wss, c->wma, c->wa, c->wsawss, c->s);
    check_launch();
    if (sawss) {
      CK(cudaMemcpyAsync(sawss, c->wsawss, sizeof(double) * c->nprob, cudaMemcpyDeviceToHost, c->s));
      CK(cudaStreamSynchronize(c->s));
    }
    return FSI_OK;
  });
}

fsi_status fsi_wss_faces(const fsi_ctx* c, int64_t* n_faces, int32_t* tet_face) {
  if (!c || !n_faces) return FSI_ERR_ARG;
  *n_faces = c->nwss;
  if (tet_face) std::memcpy(tet_face, c->wface_host.data(), sizeof(int32_t) * c->wface_host.size());
  return FSI_OK;
}

const char* fsi_last_error(const fsi_ctx* c) {
  if (!c) return "no context";
  return c->err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free residual. The paper has no counterpart: this is an interface
// for callers that must not have the library allocate device memory, for
// instance code that has fixed its whole device-memory footprint in advance or
// that runs while device allocation is forbidden. It computes exactly what
// fsi_residual computes, but the element buffer of the assembly (28 values per
// tet) lives in one file-scope device array instead of the context's buffer.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t NOALLOC_MAX_TETS = 32768;   // 28 x 8 B x 32768 = 7.3 MB per device
static __device__ __align__(256) double g_noalloc_fe[28 * NOALLOC_MAX_TETS];
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};
}  // namespace

extern "C" fsi_status fsi_residual_noalloc(fsi_ctx* c, const double* y, double* F) {
  if (!c || !y || !F) return FSI_ERR_ARG;
  return guarded(c, [&]() -> fsi_status {
    if (c->T > NOALLOC_MAX_TETS)
      throw StatusError{FSI_ERR_ARG, "fsi_residual_noalloc handles at most 32768 tets; the mesh has " +
                                         std::to_string(c->T)};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) throw StatusError{FSI_ERR_ARG, "device index out of range"};
    double* fe = nullptr;
    {
      // once per device, with that device current: the device address of the
      // array (its host-side name is only a stand-in, not a device address)
      std::lock_guard<std::mutex> lock(g_noalloc_mu);
      if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_fe));
        g_noalloc_addr[dev] = static_cast<double*>(p);
      }
      fe = g_noalloc_addr[dev];
    }
    // every slot the gather reads is written by the element kernel first, so the
    // array needs no clearing between calls
    launch_elem_residual(c->mesh, c->mc, y, c->yn, c->ynm1, fe, c->s);
    launch_gather_residual(c->mesh, c->nptr, c->nsrc, fe, F, c->s);
    launch_constraint_residual(c->mesh, c->mc, c->t + c->opt.dt, y, c->yn, F, c->s);
    check_launch();
    CK(cudaStreamSynchronize(c->s));
    return FSI_OK;
  });
}
