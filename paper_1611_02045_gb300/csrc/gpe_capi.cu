// gpe_capi.cu -- the C ABI of include/gpe.h: context set-up (grid tables,
// workspace), pass planning, the operator entry points and the PCG_C solve
// (Algorithm 2 of arXiv:1611.02045) as one CUDA graph with a device-side
// WHILE loop.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/gpe.h"
#include "gpe_internal.h"
#include "gpe_persist.cuh"
#include "gpe_cluster.cuh"
#include "gpe_csolve.cuh"

using namespace gpe;

namespace {

constexpr int kTargetBlocks = 2 * 152;  // aim for >= 2 blocks per SM per pass
constexpr int kPlanMaxBlocks = 4096;    // reduction partials reserved for tuned plans

struct PassPlan {
  int lpb = 1, tx = 1, nblocks = 1, M = 8;
  int E = 8;  // values per thread of the line transforms
  long long stride = 0, outer_stride = 0;
  int ntx = 1;
};

struct PrecBufs {
  bool on = false;
  void* xi[3] = {nullptr, nullptr, nullptr};
  void* xc[3] = {nullptr, nullptr, nullptr};
  void* tw[3] = {nullptr, nullptr, nullptr};
  void* V = nullptr;
  void* phi = nullptr;
  void* p = nullptr;
  void* t = nullptr;
  void* s = nullptr;
  void* r_prev = nullptr;
};

std::string g_create_error;

}  // namespace

struct gpe_ctx {
  gpe_problem prob{};
  int dim = 2, n[3] = {1, 1, 1};
  long long N = 0;
  double h[3] = {1, 1, 1}, weight = 1.0;
  cudaStream_t st = nullptr;
  cudaStream_t cap = nullptr;  // private stream used only for graph capture
  std::string err;
  PrecBufs pb[3];  // 0: float / complex64, 1: double / complex128, 2: double-single (refinement state)
  int work = 1;    // precision of API calls
  Ctl* ctl_solve = nullptr;
  Ctl* ctl_api = nullptr;
  double* partials = nullptr;
  unsigned* ticket = nullptr;
  double* log_dev = nullptr;
  int log_dev_cap = 0;
  PassPlan plan[3];      // default plan per axis (E = 8, heuristic widths)
  PassPlan mplan[3][3];  // plan used per launch mode [mode][axis] (the default, or the tuner's choice)
  int partials_cap = 0;  // blocks the reduction partials buffer holds
  int hbatch_rows = 16;  // rows per CTA of its streaming form (plan mode 3 width: 16 or 32)
  int* hflow_ctr = nullptr;  // counters of gpe_apply_H_batch's dataflow form (zero between launches)
  int hflow_cap = 0;
  int hbatch_E = 8;      // values per thread of gpe_apply_H_batch's cluster kernel (plan mode 3):
                         // 16 (streaming form) by default in single precision for n >= 64
  double vmax = 0.0;  // max V on the grid
  double vmin = 0.0;  // min V on the grid
  double* tf_state = nullptr;  // Thomas-Fermi bisection bracket (2 doubles, device)
  int max_threads[2] = {512, 256};
  bool warmed[3] = {false, false, false};  // per launch mode
  int nsm = 0;                      // streaming multiprocessors of the device
  double* pers_partials = nullptr;  // persistent solve: [2][grid][kMaxMoments]
  unsigned* pers_bar = nullptr;     // persistent solve: barrier words + error flag
  int pers_max_grid = 0;
  int last_loop = -1;  // loop style the last solve phase ran (gpe_report.loop_kind)
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};  // per launch mode
  // tangent-space adjoint workspace (allocated by the first gpe_tangent_solve)
  void* adj[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // r, y, p, q, rhs, z
  AdjScalars* adj_s = nullptr;
  double* adj_partials = nullptr;
};

#define GPE_CU(ctx, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return GPE_ERR_CUDA;                                                                 \
    }                                                                                      \
  } while (0)

static bool is_pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static void plan_axis(gpe_ctx* c, int axis, int maxT, PassPlan& pl) {
  const int M = c->n[axis];
  const int Tl = M / pl.E;
  pl.M = M;
  if (axis == 0) {
    const long long nlines = (long long)c->n[1] * (c->dim == 3 ? c->n[2] : 1);
    int lpb = maxT / Tl;
    if (lpb < 1) lpb = 1;
    while (lpb > 1 && (lpb > nlines || nlines / lpb < kTargetBlocks)) lpb >>= 1;
    pl.lpb = lpb;
    pl.nblocks = (int)(nlines / lpb);
  } else {
    const int nx = c->n[0];
    const long long outer = (axis == 1) ? (c->dim == 3 ? c->n[2] : 1) : c->n[1];
    int tx = 16;
    if (tx > nx) tx = nx;
    while (tx > 1 && tx * Tl > maxT) tx >>= 1;
    while (tx > 4 && (long long)(nx / tx) * outer < kTargetBlocks) tx >>= 1;
    pl.tx = tx;
    pl.ntx = nx / tx;
    pl.nblocks = (int)((long long)pl.ntx * outer);
    pl.stride = (axis == 1) ? nx : (long long)nx * c->n[1];
    pl.outer_stride = (axis == 1) ? (long long)nx * c->n[1] : nx;
  }
}

// Pass arguments for `axis` with the tables of precision `prec` and the plan
// of launch mode `mode`.
static PassArgs base_args(gpe_ctx* c, int prec, int axis, int mode) {
  PassArgs a;
  std::memset(&a, 0, sizeof(a));
  const PassPlan& pl = c->mplan[mode][axis];
  const PrecBufs& b = c->pb[prec];
  a.dim = c->dim; a.nx = c->n[0]; a.ny = c->n[1]; a.nz = c->dim == 3 ? c->n[2] : 1;
  a.axis = axis; a.M = pl.M; a.E = pl.E; a.lpb = pl.lpb; a.tx = pl.tx; a.stride = pl.stride;
  a.outer_stride = pl.outer_stride; a.ntx = pl.ntx; a.nblocks = pl.nblocks;
  a.weight = c->weight; a.eta = c->prob.eta; a.omega = c->prob.omega;
  for (int i = 0; i < 3; ++i) { a.xi[i] = b.xi[i]; a.xc[i] = b.xc[i]; }
  a.tw = b.tw[axis];
  a.V = b.V;
  a.partials = c->partials;
  a.ticket = c->ticket;
  return a;
}

static cudaError_t launch(int mode, Pass pass, const PassArgs& a, cudaStream_t st) {
  return launch_pass(mode, pass, a, st);
}

// Buffers of one solver iteration.  State fields (phi, H phi, r_prev, V) and
// direction fields (P_C workspace s, p) may live in different precisions
// (launch mode 2); tab_h / tab_d select the table precision of the H passes
// and of the direction passes.
struct IterBufs {
  int mode;
  int tab_h, tab_d;
  void* phi;
  void* t;
  void* r_prev;
  const void* V;
  void* s;
  void* p;
};

static IterBufs iter_bufs(gpe_ctx* c, int mode) {
  IterBufs b;
  b.mode = mode;
  const int sp = mode == 0 ? 0 : (mode == 2 ? 2 : 1);  // state precision (2: double-single)
  const int dp = mode == 1 ? 1 : 0;  // direction precision
  b.tab_h = sp;
  b.tab_d = dp;
  b.phi = c->pb[sp].phi; b.t = c->pb[sp].t; b.r_prev = c->pb[sp].r_prev; b.V = c->pb[sp].V;
  b.s = c->pb[dp].s; b.p = c->pb[dp].p;
  return b;
}

template <typename T>
static cudaError_t upload_tables(gpe_ctx* c, PrecBufs& b) {
  for (int i = 0; i < c->dim; ++i) {
    const int M = c->n[i];
    const double L = c->prob.L[i];
    std::vector<T> xi(M), xc(M), tw(2 * M);
    for (int p = 0; p < M; ++p) {
      const int pp = p < M / 2 ? p : p - M;  // xi_p = p pi / L, p = -M/2 .. M/2-1
      xi[p] = (T)(pp * M_PI / L);
      xc[p] = (T)(-L + p * (2.0 * L / M));   // x_k = -L + k h
      tw[2 * p] = (T)std::cos(2.0 * M_PI * p / M);
      tw[2 * p + 1] = (T)(-std::sin(2.0 * M_PI * p / M));
    }
    cudaError_t e;
    if ((e = cudaMalloc(&b.xi[i], M * sizeof(T))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&b.xc[i], M * sizeof(T))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&b.tw[i], 2 * M * sizeof(T))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b.xi[i], xi.data(), M * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b.xc[i], xc.data(), M * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b.tw[i], tw.data(), 2 * M * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// V of one precision (float32, float64 or double-single) from a device float64
// copy; the buffer is already allocated.
static gpe_status upload_V(gpe_ctx* c, int prec, const double* Vdev64) {
  PrecBufs& b = c->pb[prec];
  if (prec == 2) GPE_CU(c, launch_d2ds(Vdev64, b.V, c->N, 0));
  else if (prec == 1) GPE_CU(c, cudaMemcpy(b.V, Vdev64, 8 * (size_t)c->N, cudaMemcpyDeviceToDevice));
  else GPE_CU(c, launch_d2f(Vdev64, (float*)b.V, c->N, 0));
  GPE_CU(c, cudaDeviceSynchronize());
  return GPE_OK;
}

// Copy V (float64, host or device) to a new device buffer, check that it is
// finite and record its maximum (used by the single-precision floor estimate).
static gpe_status load_V(gpe_ctx* c, const double* V, double** V64_out) {
  *V64_out = nullptr;
  double* V64 = nullptr;
  if (cudaMalloc(&V64, 8 * (size_t)c->N) != cudaSuccess) { c->err = "cudaMalloc V"; return GPE_ERR_CUDA; }
  std::vector<double> Vh((size_t)c->N);
  if (cudaMemcpy(V64, V, 8 * (size_t)c->N, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(Vh.data(), V64, 8 * (size_t)c->N, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaFree(V64); c->err = "copy of V failed"; return GPE_ERR_CUDA;
  }
  double vm = -1e300, vn = 1e300;
  for (double v : Vh) {
    if (!std::isfinite(v)) { cudaFree(V64); c->err = "V must be finite"; return GPE_ERR_ARG; }
    vm = v > vm ? v : vm;
    vn = v < vn ? v : vn;
  }
  c->vmax = vm;
  c->vmin = vn;
  *V64_out = V64;
  return GPE_OK;
}

static gpe_status alloc_prec(gpe_ctx* c, int prec, const double* Vdev64) {
  PrecBufs& b = c->pb[prec];
  b.on = true;
  const size_t cb = prec ? 16 : 8;  // complex64 8 B; complex128 and double-single 16 B
  const size_t bytes = cb * (size_t)c->N;
  if (prec == 2) GPE_CU(c, upload_tables<dsf>(c, b));
  else GPE_CU(c, prec ? upload_tables<double>(c, b) : upload_tables<float>(c, b));
  GPE_CU(c, cudaMalloc(&b.phi, bytes));
  GPE_CU(c, cudaMalloc(&b.p, bytes));
  GPE_CU(c, cudaMalloc(&b.t, bytes));
  GPE_CU(c, cudaMalloc(&b.s, bytes));
  GPE_CU(c, cudaMalloc(&b.r_prev, bytes));
  GPE_CU(c, cudaMemset(b.p, 0, bytes));
  GPE_CU(c, cudaMemset(b.r_prev, 0, bytes));
  GPE_CU(c, cudaMalloc(&b.V, (prec == 0 ? 4 : 8) * (size_t)c->N));
  return upload_V(c, prec, Vdev64);
}

static void free_ctx(gpe_ctx* c) {
  for (auto& e : c->exec)
    if (e) cudaGraphExecDestroy(e);
  for (auto& b : c->pb) {
    for (int i = 0; i < 3; ++i) { cudaFree(b.xi[i]); cudaFree(b.xc[i]); cudaFree(b.tw[i]); }
    cudaFree(b.V); cudaFree(b.phi); cudaFree(b.p); cudaFree(b.t); cudaFree(b.s); cudaFree(b.r_prev);
  }
  cudaFree(c->pers_partials); cudaFree(c->pers_bar);
  for (auto& a : c->adj) cudaFree(a);
  cudaFree(c->tf_state);
  cudaFree(c->adj_s); cudaFree(c->adj_partials);
  cudaFree(c->hflow_ctr);
  cudaFree(c->ctl_solve); cudaFree(c->ctl_api); cudaFree(c->partials); cudaFree(c->ticket); cudaFree(c->log_dev);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

extern "C" gpe_status gpe_solve_opts_default(gpe_solve_opts* o) {
  if (!o) return GPE_ERR_ARG;
  o->tol_res_inf = 1e-8;
  o->tol_dE = 0.0;
  o->max_iter = 20000;
  o->theta_default = 0.1;
  o->max_backtracks = 30;
  o->cg = 1;
  o->stall_window = 500;
  o->switch_res = 0.0;
  o->max_iter_lo = 0;
  o->use_graph = 3;
  o->refine_restart = 1;
  o->precond = GPE_PRECOND_C;
  o->beta_rule = GPE_BETA_PR;
  o->line_search = GPE_LINE_MODEL;
  o->wait_polls = 0;
  return GPE_OK;
}

extern "C" gpe_status gpe_create(const gpe_problem* prob, const double* V, void* stream, gpe_ctx** out) {
  if (!prob || !V || !out) { g_create_error = "null argument"; return GPE_ERR_ARG; }
  *out = nullptr;
  if (prob->dim != 2 && prob->dim != 3) { g_create_error = "dim must be 2 or 3"; return GPE_ERR_ARG; }
  for (int i = 0; i < prob->dim; ++i) {
    if (!is_pow2_in(prob->n[i], 8, 512)) { g_create_error = "n[i] must be a power of two in [8, 512]"; return GPE_ERR_ARG; }
    if (!(prob->L[i] > 0.0) || !std::isfinite(prob->L[i])) { g_create_error = "L[i] must be finite and > 0"; return GPE_ERR_ARG; }
  }
  if (!std::isfinite(prob->eta) || !std::isfinite(prob->omega)) { g_create_error = "eta/omega must be finite"; return GPE_ERR_ARG; }
  if (prob->prec != GPE_FP64 && prob->prec != GPE_MIXED) { g_create_error = "unknown precision"; return GPE_ERR_ARG; }

  gpe_ctx* c = new gpe_ctx();
  c->prob = *prob;
  c->dim = prob->dim;
  c->N = 1;
  c->weight = 1.0;
  for (int i = 0; i < c->dim; ++i) {
    c->n[i] = prob->n[i];
    c->h[i] = 2.0 * prob->L[i] / prob->n[i];
    c->N *= prob->n[i];
    c->weight *= c->h[i];
  }
  c->st = (cudaStream_t)stream;
  c->work = prob->prec == GPE_FP64 ? 1 : 0;
  if (c->work == 0 && c->dim == 2 && c->n[0] == c->n[1] && c->n[0] >= 64 && c->n[0] <= 256) c->hbatch_E = 16;
  auto fail = [&](gpe_status s) { g_create_error = c->err; free_ctx(c); return s; };
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) { c->err = "stream create failed"; return fail(GPE_ERR_CUDA); }

  // potential: a device float64 copy is the source of every precision
  double* V64 = nullptr;
  {
    const gpe_status sv = load_V(c, V, &V64);
    if (sv != GPE_OK) return fail(sv);
  }
  gpe_status s = alloc_prec(c, 1, V64);
  if (s == GPE_OK && prob->prec == GPE_MIXED) s = alloc_prec(c, 0, V64);
  if (s == GPE_OK && prob->prec == GPE_MIXED) s = alloc_prec(c, 2, V64);
  cudaFree(V64);
  if (s != GPE_OK) return fail(s);

  int maxblocks = 1;
  for (int ax = 0; ax < c->dim; ++ax) {
    // plan with the smaller (double) thread cap so one plan serves both precisions
    plan_axis(c, ax, c->max_threads[1], c->plan[ax]);
    if (c->plan[ax].nblocks > maxblocks) maxblocks = c->plan[ax].nblocks;
    for (int m = 0; m < 3; ++m) c->mplan[m][ax] = c->plan[ax];
  }
  c->partials_cap = maxblocks > kPlanMaxBlocks ? maxblocks : kPlanMaxBlocks;  // room for tuned plans
  if (cudaMalloc(&c->ctl_solve, sizeof(Ctl)) != cudaSuccess || cudaMalloc(&c->ctl_api, sizeof(Ctl)) != cudaSuccess ||
      cudaMalloc(&c->partials, sizeof(double) * kMaxMoments * (size_t)c->partials_cap) != cudaSuccess ||
      cudaMalloc(&c->ticket, sizeof(unsigned)) != cudaSuccess) {
    c->err = "cudaMalloc workspace"; return fail(GPE_ERR_CUDA);
  }
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
    c->pers_max_grid = 8 * (c->nsm > 0 ? c->nsm : 1);
    if (cudaMalloc(&c->pers_partials, sizeof(double) * 2 * kMaxMoments * (size_t)c->pers_max_grid) != cudaSuccess ||
        cudaMalloc(&c->pers_bar, 4 * sizeof(unsigned)) != cudaSuccess) {
      c->err = "cudaMalloc persistent workspace"; return fail(GPE_ERR_CUDA);
    }
  }
  cudaMemset(c->ctl_solve, 0, sizeof(Ctl));
  cudaMemset(c->ctl_api, 0, sizeof(Ctl));
  cudaMemset(c->ticket, 0, sizeof(unsigned));
  if (cudaDeviceSynchronize() != cudaSuccess) { c->err = "set-up failed"; return fail(GPE_ERR_CUDA); }
  *out = c;
  return GPE_OK;
}

extern "C" gpe_status gpe_destroy(gpe_ctx* c) {
  if (!c) return GPE_OK;
  cudaStreamSynchronize(c->st);
  free_ctx(c);
  return GPE_OK;
}

extern "C" const char* gpe_last_error(const gpe_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

// H passes on (phi, f): t = A_x f + (V + eta|phi|^2) f, then the y (and z) parts
// accumulated; the last one writes `out` (or t) and finalises the energy terms.
// moments = false: H phi as a plain operator (gpe_apply_H); the passes skip the
// energy moments and the scalar step that only gpe_energy and the solver read.
static gpe_status run_H(gpe_ctx* c, int prec, const void* phi, const void* f, void* out, Ctl* ctl,
                        bool moments = true) {
  PassArgs a = base_args(c, prec, 0, prec);
  a.ctl = ctl; a.phi = phi; a.f = f; a.t = c->pb[prec].t;
  a.nomoments = moments ? 0 : 1;
  // fields above 64 MB (beyond L2 with the operator's other arrays): the x pass
  // prefetches the rows of the block one wave ahead (two blocks per SM)
  if ((double)c->N * (prec == 0 ? 8.0 : 16.0) > 64.0 * 1024 * 1024) a.pf = 2 * c->nsm;
  GPE_CU(c, launch(prec, P_HX, a, c->st));
  for (int ax = 1; ax < c->dim; ++ax) {
    PassArgs b = base_args(c, prec, ax, prec);
    b.ctl = ctl; b.phi = phi; b.f = f; b.t = c->pb[prec].t;
    b.nomoments = a.nomoments;
    b.last_axis = (ax == c->dim - 1);
    b.out = b.last_axis ? out : nullptr;
    GPE_CU(c, launch(prec, P_HMID, b, c->st));
  }
  return GPE_OK;
}

extern "C" gpe_status gpe_apply_H(gpe_ctx* c, const void* phi, const void* f, void* out) {
  if (!c) return GPE_ERR_ARG;
  if (!phi || !f || !out) { c->err = "null field pointer"; return GPE_ERR_ARG; }
  return run_H(c, c->work, phi, f, out, c->ctl_api, false);
}

extern "C" gpe_status gpe_apply_H_batch(gpe_ctx* c, int nbatch, const void* phi, const void* f, void* out) {
  if (!c) return GPE_ERR_ARG;
  if (nbatch < 0 || !phi || !f || !out) { c->err = "bad batch arguments"; return GPE_ERR_ARG; }
  if (c->dim != 2 || c->n[0] != c->n[1] || c->n[0] < 32 || c->n[0] > 256) {
    c->err = "gpe_apply_H_batch needs a 2D grid with nx == ny in [32, 256]";
    return GPE_ERR_UNSUPPORTED;
  }
  if (nbatch == 0) return GPE_OK;
  const int prec = c->work;
  const PrecBufs& b = c->pb[prec];
  ClusterHArgs a;
  std::memset(&a, 0, sizeof(a));
  a.M = c->n[0]; a.nbatch = nbatch; a.stride = c->N;
  a.eta = c->prob.eta; a.omega = c->prob.omega;
  a.xi = b.xi[0]; a.xiy = b.xi[1]; a.xc = b.xc[0]; a.yc = b.xc[1]; a.tw = b.tw[0]; a.V = b.V;
  a.phi = phi; a.f = f; a.out = out;
  a.E = c->hbatch_E;
  a.rows = c->hbatch_rows;
  if (prec == 0 && a.M == 256 && a.E == 16 && a.rows == 16 && phi == f) {
    // the dataflow form's counters: allocated (zeroed) on first use and when the batch grows;
    // the kernel leaves them zero
    const size_t need = h_batch_flow_counters(nbatch);
    if ((size_t)c->hflow_cap < need) {
      const size_t cap = need > 2 * (size_t)c->hflow_cap ? need : 2 * (size_t)c->hflow_cap;
      if (c->hflow_ctr) GPE_CU(c, cudaFree(c->hflow_ctr));
      c->hflow_ctr = nullptr;
      c->hflow_cap = 0;
      GPE_CU(c, cudaMalloc(&c->hflow_ctr, cap * sizeof(int)));
      GPE_CU(c, cudaMemsetAsync(c->hflow_ctr, 0, cap * sizeof(int), c->st));
      c->hflow_cap = (int)cap;
    }
    a.flow_ctr = c->hflow_ctr;
    a.flow_cap = c->hflow_cap;
    a.status = &c->ctl_api->status;
  }
  GPE_CU(c, launch_cluster_apply_H(prec, a, c->st));
  return GPE_OK;
}

extern "C" gpe_status gpe_energy(gpe_ctx* c, const void* phi, double out[8]) {
  if (!c) return GPE_ERR_ARG;
  if (!phi || !out) { c->err = "null pointer"; return GPE_ERR_ARG; }
  const int prec = c->work;
  gpe_status s = run_H(c, prec, phi, phi, c->pb[prec].t, c->ctl_api);
  if (s != GPE_OK) return s;
  Ctl h;
  GPE_CU(c, cudaMemcpyAsync(&h, c->ctl_api, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st));
  GPE_CU(c, cudaStreamSynchronize(c->st));
  out[0] = h.kin; out[1] = h.pot; out[2] = 0.5 * c->prob.eta * h.U0; out[3] = h.rot;
  out[4] = h.E; out[5] = h.lam; out[6] = h.alpha; out[7] = h.norm2;
  return GPE_OK;
}

extern "C" gpe_status gpe_set_problem(gpe_ctx* c, const double* V, double eta, double omega) {
  if (!c) return GPE_ERR_ARG;
  if (!std::isfinite(eta) || !std::isfinite(omega)) { c->err = "eta/omega must be finite"; return GPE_ERR_ARG; }
  GPE_CU(c, cudaStreamSynchronize(c->st));
  if (V) {
    double* V64 = nullptr;
    gpe_status s = load_V(c, V, &V64);
    if (s != GPE_OK) return s;
    for (int prec = 0; prec < 3 && s == GPE_OK; ++prec)
      if (c->pb[prec].on) s = upload_V(c, prec, V64);
    cudaFree(V64);
    if (s != GPE_OK) return s;
  }
  c->prob.eta = eta;
  c->prob.omega = omega;
  // captured graphs hold the old eta and omega in their kernel arguments
  for (auto& e : c->exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  return GPE_OK;
}

extern "C" gpe_status gpe_energy_grad(gpe_ctx* c, const void* phi, void* grad_phi, double* grad_V, double out[5]) {
  if (!c) return GPE_ERR_ARG;
  if (!phi || !out) { c->err = "null pointer"; return GPE_ERR_ARG; }
  if (grad_phi == phi) { c->err = "grad_phi must not overlap phi"; return GPE_ERR_ARG; }
  const int prec = c->work;
  void* hphi = grad_phi ? grad_phi : c->pb[prec].t;
  gpe_status s = run_H(c, prec, phi, phi, hphi, c->ctl_api);
  if (s != GPE_OK) return s;
  if (grad_phi || grad_V) GPE_CU(c, launch_grad_epilogue(prec, phi, grad_phi, grad_V, c->N, c->weight, c->st));
  Ctl h;
  GPE_CU(c, cudaMemcpyAsync(&h, c->ctl_api, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st));
  GPE_CU(c, cudaStreamSynchronize(c->st));
  out[0] = h.E;
  out[1] = 0.5 * h.U0;  // d/d eta of eta/2 int |phi|^4
  out[2] = -h.Lz;       // d/d omega of -omega <phi, L_z phi>
  out[3] = h.lam;
  out[4] = h.norm2;
  return GPE_OK;
}

// Tangent-space adjoint solve: K z = P rhs, <phi, z> = 0, by the projected
// conjugate gradient method with the projected P_C as preconditioner (kernels
// in gpe_adjoint.cu).  Declared below run_PC.
static gpe_status tangent_solve(gpe_ctx* c, const void* phi, const void* rhs, void* z, double tol, int max_iter,
                                int* iters, double* rel_res);

extern "C" gpe_status gpe_thomas_fermi(gpe_ctx* c, void* phi_out, double* mu_out) {
  if (!c) return GPE_ERR_ARG;
  if (!phi_out) { c->err = "null phi"; return GPE_ERR_ARG; }
  if (!(c->prob.eta > 0.0)) { c->err = "the Thomas-Fermi state needs eta > 0"; return GPE_ERR_ARG; }
  if (!c->tf_state) GPE_CU(c, cudaMalloc(&c->tf_state, 2 * sizeof(double)));
  // bracket: S(vmin) = 0 < 1 and S(vmax + eta / (h^d N)) >= 1
  const double br[2] = {c->vmin, c->vmax + c->prob.eta / (c->weight * (double)c->N)};
  GPE_CU(c, cudaMemcpyAsync(c->tf_state, br, sizeof(br), cudaMemcpyHostToDevice, c->st));
  const double* V64 = static_cast<const double*>(c->pb[1].V);
  for (int it = 0; it < 120; ++it)  // halves the bracket each time: far below one ulp of mu
    GPE_CU(c, launch_tf_bisect(V64, c->N, c->weight, c->prob.eta, c->tf_state, c->partials, c->ticket, c->st));
  const bool dev = is_device_ptr(phi_out);
  void* dst = dev ? phi_out : c->pb[1].phi;
  GPE_CU(c, launch_tf_fill(V64, c->N, c->prob.eta, c->tf_state, dst, c->st));
  if (!dev) GPE_CU(c, cudaMemcpyAsync(phi_out, dst, 16 * (size_t)c->N, cudaMemcpyDeviceToHost, c->st));
  double st[2];
  GPE_CU(c, cudaMemcpyAsync(st, c->tf_state, sizeof(st), cudaMemcpyDeviceToHost, c->st));
  GPE_CU(c, cudaStreamSynchronize(c->st));
  if (mu_out) *mu_out = 0.5 * (st[0] + st[1]);
  return GPE_OK;
}

extern "C" gpe_status gpe_interpolate(gpe_ctx* cc, const void* phi_c, gpe_ctx* cf, void* phi_f) {
  if (!cc || !cf) return GPE_ERR_ARG;
  if (!phi_c || !phi_f) { cf->err = "null field pointer"; return GPE_ERR_ARG; }
  if (cc->dim != cf->dim) { cf->err = "coarse and fine grids differ in dimension"; return GPE_ERR_ARG; }
  for (int i = 0; i < cf->dim; ++i) {
    const bool same_l = std::fabs(cc->prob.L[i] - cf->prob.L[i]) <= 1e-12 * std::fabs(cf->prob.L[i]);
    if (!same_l || !(cf->n[i] == cc->n[i] || cf->n[i] == 2 * cc->n[i])) {
      cf->err = "the fine grid must cover the same domain with n or 2n points per axis";
      return GPE_ERR_ARG;
    }
    if (cf->n[i] == 2 * cc->n[i] && cc->n[i] > 256) { cf->err = "coarse axes above 256 points"; return GPE_ERR_UNSUPPORTED; }
  }
  cudaStream_t st = cf->st;
  GPE_CU(cf, cudaStreamSynchronize(cc->st));
  const double2* src = static_cast<const double2*>(phi_c);
  if (!is_device_ptr(phi_c)) {
    GPE_CU(cf, cudaMemcpyAsync(cc->pb[1].phi, phi_c, 16 * (size_t)cc->N, cudaMemcpyHostToDevice, st));
    src = static_cast<const double2*>(cc->pb[1].phi);
  }
  const bool out_dev = is_device_ptr(phi_f);
  // ping-pong through the fine context's work fields, the last stage into the destination
  double2* bufs[2] = {static_cast<double2*>(cf->pb[1].t), static_cast<double2*>(cf->pb[1].s)};
  double2* dst_final = out_dev ? static_cast<double2*>(phi_f) : static_cast<double2*>(cf->pb[1].phi);
  int last = -1;
  for (int i = 0; i < cf->dim; ++i)
    if (cf->n[i] != cc->n[i]) last = i;
  long long nx = cc->n[0], ny = cc->n[1], nz = cf->dim == 3 ? cc->n[2] : 1;  // current extents
  const double2* cur = src;
  int pp = 0;
  for (int ax = 0; ax < cf->dim; ++ax) {
    if (cf->n[ax] == cc->n[ax]) continue;
    const int Mc = cc->n[ax];
    double2* nxt = (ax == last) ? dst_final : bufs[pp];
    pp ^= 1;
    InterpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = cur; a.out = nxt;
    a.tw_c = static_cast<const double2*>(cc->pb[1].tw[ax]);
    a.tw_f = static_cast<const double2*>(cf->pb[1].tw[ax]);
    if (ax == 0) {
      a.lines = ny * nz; a.inner_count = 1;
      a.in_outer = Mc; a.out_outer = 2 * Mc; a.in_stride = a.out_stride = 1;
    } else if (ax == 1) {
      a.lines = nx * nz; a.inner_count = nx;
      a.in_outer = (long long)Mc * nx; a.out_outer = 2LL * Mc * nx; a.in_inner = a.out_inner = 1;
      a.in_stride = a.out_stride = nx;
    } else {
      a.lines = nx * ny; a.inner_count = nx * ny;
      a.in_outer = a.out_outer = 0; a.in_inner = a.out_inner = 1;
      a.in_stride = a.out_stride = nx * ny;
    }
    GPE_CU(cf, launch_interp(Mc, a, st));
    cur = nxt;
    if (ax == 0) nx *= 2; else if (ax == 1) ny *= 2; else nz *= 2;
  }
  if (last < 0)  // nothing to refine: a copy
    GPE_CU(cf, cudaMemcpyAsync(dst_final, src, 16 * (size_t)cf->N, cudaMemcpyDeviceToDevice, st));
  if (!out_dev) GPE_CU(cf, cudaMemcpyAsync(phi_f, dst_final, 16 * (size_t)cf->N, cudaMemcpyDeviceToHost, st));
  GPE_CU(cf, cudaStreamSynchronize(st));
  return GPE_OK;
}

// P_C passes: s = FFT_x(P_V^{1/2} r) -> (3D: FFT_y) -> core -> (3D: IFFT_y) -> P_V^{1/2} IFFT_x.
static gpe_status run_PC(gpe_ctx* c, const IterBufs& b, const void* r, double alpha, void* out, Ctl* ctl,
                         bool solver, cudaStream_t st) {
  PassArgs a = base_args(c, b.tab_d, 0, b.mode);
  a.V = b.V;
  a.ctl = ctl; a.solver = solver; a.phi = b.phi; a.r_in = r; a.api_alpha = alpha;
  a.s = b.s; a.t = b.t; a.r_prev = b.r_prev; a.p = b.p; a.out = out;
  GPE_CU(c, launch(b.mode, P_C1, a, st));
  if (c->dim == 3) {
    PassArgs y = base_args(c, b.tab_d, 1, b.mode);
    y.ctl = ctl; y.solver = solver; y.s = b.s;
    GPE_CU(c, launch(b.mode, P_CFWD, y, st));
  }
  PassArgs k = base_args(c, b.tab_d, c->dim - 1, b.mode);
  k.ctl = ctl; k.solver = solver; k.s = b.s; k.api_alpha = alpha;
  GPE_CU(c, launch(b.mode, P_CCORE, k, st));
  if (c->dim == 3) {
    PassArgs y = base_args(c, b.tab_d, 1, b.mode);
    y.ctl = ctl; y.solver = solver; y.s = b.s;
    GPE_CU(c, launch(b.mode, P_CINV, y, st));
  }
  GPE_CU(c, launch(b.mode, P_C3, a, st));
  return GPE_OK;
}

extern "C" gpe_status gpe_precond(gpe_ctx* c, const void* phi, const void* r, double alpha, void* out) {
  if (!c) return GPE_ERR_ARG;
  if (!phi || !r || !out) { c->err = "null field pointer"; return GPE_ERR_ARG; }
  if (!std::isfinite(alpha)) { c->err = "alpha must be finite"; return GPE_ERR_ARG; }
  const int prec = c->work;
  if (!(alpha > 0.0)) {
    gpe_status s = run_H(c, prec, phi, phi, c->pb[prec].t, c->ctl_api);  // lambda~ into ctl_api->alpha
    if (s != GPE_OK) return s;
  }
  IterBufs b = iter_bufs(c, prec);
  b.phi = const_cast<void*>(phi);
  return run_PC(c, b, r, alpha, out, c->ctl_api, false, c->st);
}

constexpr int kAdjMaxBlocks = 1024;
constexpr int kAdjCheckEvery = 4;  // iterations between host reads of the scalars

static gpe_status tangent_solve(gpe_ctx* c, const void* phi, const void* rhs, void* z, double tol, int max_iter,
                                int* iters, double* rel_res) {
  const int prec = c->work;
  const size_t bytes = (prec ? 16 : 8) * (size_t)c->N;
  if (!c->adj_s) {
    for (auto& a : c->adj) GPE_CU(c, cudaMalloc(&a, bytes));
    GPE_CU(c, cudaMalloc(&c->adj_s, sizeof(AdjScalars)));
    GPE_CU(c, cudaMalloc(&c->adj_partials, sizeof(double) * 6 * kAdjMaxBlocks));
  }
  void *r = c->adj[0], *y = c->adj[1], *p = c->adj[2], *q = c->adj[3];
  AdjScalars* S = c->adj_s;
  const long long N = c->N;
  const double w = c->weight;
  cudaStream_t st = c->st;
  // lambda = <phi, H phi> and the shift lambda~ of eq. Opt_Alpha at phi
  gpe_status s = run_H(c, prec, phi, phi, q, c->ctl_api);
  if (s != GPE_OK) return s;
  Ctl h;
  GPE_CU(c, cudaMemcpyAsync(&h, c->ctl_api, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  GPE_CU(c, cudaStreamSynchronize(st));
  const double lam = h.lam, alpha = h.alpha;
  if (!std::isfinite(lam) || !(alpha > 0.0)) { c->err = "phi gives a non-finite lambda or a shift <= 0"; return GPE_ERR_NONFINITE; }
  AdjScalars s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.tol2 = tol * tol;
  GPE_CU(c, cudaMemcpyAsync(S, &s0, sizeof(s0), cudaMemcpyHostToDevice, st));
  GPE_CU(c, cudaMemsetAsync(z, 0, bytes, st));
  GPE_CU(c, cudaMemsetAsync(p, 0, bytes, st));
  // r = P rhs, bb = ||r||^2
  GPE_CU(c, adj_dots(prec, phi, rhs, nullptr, nullptr, nullptr, nullptr, N, w, ADJ_PROJ, S, c->adj_partials,
                     kAdjMaxBlocks, st));
  GPE_CU(c, adj_proj(prec, rhs, r, phi, N, S, st));
  GPE_CU(c, adj_dots(prec, r, r, nullptr, nullptr, nullptr, nullptr, N, w, ADJ_BB, S, c->adj_partials, kAdjMaxBlocks, st));
  IterBufs b = iter_bufs(c, prec);
  b.phi = const_cast<void*>(phi);
  // y = P_C r; p = P y
  if ((s = run_PC(c, b, r, alpha, y, c->ctl_api, false, st)) != GPE_OK) return s;
  GPE_CU(c, adj_dots(prec, phi, y, r, y, r, phi, N, w, ADJ_RY_FIRST, S, c->adj_partials, kAdjMaxBlocks, st));
  GPE_CU(c, adj_dir(prec, p, y, phi, N, S, st));
  AdjScalars hs = s0;
  int it = 0;
  for (;;) {
    if (it % kAdjCheckEvery == 0 || it >= max_iter) {
      GPE_CU(c, cudaMemcpyAsync(&hs, S, sizeof(hs), cudaMemcpyDeviceToHost, st));
      GPE_CU(c, cudaStreamSynchronize(st));
      if (hs.stop || it >= max_iter) break;
    }
    // q = P K p;  a = Re<r, y> / Re<p, q>;  z += a p;  r -= a q
    if ((s = run_H(c, prec, phi, p, q, c->ctl_api)) != GPE_OK) return s;
    GPE_CU(c, adj_hess_epi(prec, phi, p, q, N, c->prob.eta, lam, w, S, c->adj_partials, kAdjMaxBlocks, st));
    GPE_CU(c, adj_step(prec, z, r, p, q, phi, N, w, S, c->adj_partials, kAdjMaxBlocks, st));
    // y = P_C r;  beta = Re<r, P y> / previous;  p = P y + beta p
    if ((s = run_PC(c, b, r, alpha, y, c->ctl_api, false, st)) != GPE_OK) return s;
    GPE_CU(c, adj_dots(prec, phi, y, r, y, r, phi, N, w, ADJ_RY, S, c->adj_partials, kAdjMaxBlocks, st));
    GPE_CU(c, adj_dir(prec, p, y, phi, N, S, st));
    ++it;
  }
  if (iters) *iters = hs.iters;
  const double rr = hs.bb > 0.0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
  if (rel_res) *rel_res = rr;
  if (hs.bad) {
    c->err = hs.bad == 1 ? "Re<p, K p> <= 0: phi is not a local minimum (K not positive on the tangent space)"
           : hs.bad == 2 ? "Re<r, P_C r> <= 0: preconditioner not positive"
                         : "non-finite residual";
    return GPE_ERR_NONFINITE;
  }
  if (!(rr <= tol)) {
    c->err = "tangent solve reached max_iter";
    return GPE_ERR_NOT_CONVERGED;
  }
  return GPE_OK;
}

extern "C" gpe_status gpe_tangent_solve(gpe_ctx* c, const void* phi, const void* rhs, void* z, double tol, int max_iter,
                                        int* iters, double* rel_res) {
  if (!c) return GPE_ERR_ARG;
  if (!phi || !rhs || !z) { c->err = "null field pointer"; return GPE_ERR_ARG; }
  if (z == phi || z == rhs) { c->err = "z must not overlap phi or rhs"; return GPE_ERR_ARG; }
  if (!(tol > 0.0) || max_iter < 1) { c->err = "tol must be > 0 and max_iter >= 1"; return GPE_ERR_ARG; }
  if (iters) *iters = 0;
  if (rel_res) *rel_res = 0.0;
  return tangent_solve(c, phi, rhs, z, tol, max_iter, iters, rel_res);
}

extern "C" gpe_status gpe_density_adjoint(gpe_ctx* c, const void* phi, const double* g_rho, double* grad_V, double tol,
                                          int max_iter, int* iters, double* rel_res) {
  if (!c) return GPE_ERR_ARG;
  if (!phi || !g_rho || !grad_V) { c->err = "null pointer"; return GPE_ERR_ARG; }
  if (!(tol > 0.0) || max_iter < 1) { c->err = "tol must be > 0 and max_iter >= 1"; return GPE_ERR_ARG; }
  if (iters) *iters = 0;
  if (rel_res) *rel_res = 0.0;
  const int prec = c->work;
  const size_t bytes = (prec ? 16 : 8) * (size_t)c->N;
  for (int i = 4; i < 6; ++i)
    if (!c->adj[i]) GPE_CU(c, cudaMalloc(&c->adj[i], bytes));
  void *rhs = c->adj[4], *z = c->adj[5];
  GPE_CU(c, adj_density_rhs(prec, phi, g_rho, rhs, c->N, 2.0 / c->weight, c->st));
  gpe_status s = tangent_solve(c, phi, rhs, z, tol, max_iter, iters, rel_res);
  if (s != GPE_OK && s != GPE_ERR_NOT_CONVERGED) return s;
  GPE_CU(c, adj_dV_from_z(prec, phi, z, grad_V, c->N, c->weight, c->st));
  GPE_CU(c, cudaStreamSynchronize(c->st));
  return s;
}

// The pass arguments of one PCG iteration in launch mode `mode`, on the solver
// buffers (default plans: one unit per block).
struct IterArgs {
  PassArgs hx, hmid[2], c1, cfwd, ccore, cinv, c3, ax, amid[2];
};

static IterArgs iter_args(gpe_ctx* c, int mode, unsigned long long cond) {
  const IterBufs b = iter_bufs(c, mode);
  Ctl* ctl = c->ctl_solve;
  IterArgs I;
  // H phi (with the retraction phi_{n+1} = (c phi_n + s p_n/|p_n|)/nrm folded into the x pass)
  I.hx = base_args(c, b.tab_h, 0, mode);
  I.hx.V = b.V;
  I.hx.ctl = ctl; I.hx.solver = 1; I.hx.phi = b.phi; I.hx.phi_out = b.phi; I.hx.p = b.p; I.hx.t = b.t;
  for (int ax = 1; ax < 3; ++ax) {
    PassArgs& h = I.hmid[ax - 1];
    h = base_args(c, b.tab_h, ax < c->dim ? ax : 0, mode);
    h.ctl = ctl; h.solver = 1; h.phi = b.phi; h.t = b.t; h.last_axis = (ax == c->dim - 1);
  }
  // P_C r_n
  I.c1 = base_args(c, b.tab_d, 0, mode);
  I.c1.V = b.V;
  I.c1.ctl = ctl; I.c1.solver = 1; I.c1.phi = b.phi; I.c1.s = b.s; I.c1.t = b.t; I.c1.r_prev = b.r_prev; I.c1.p = b.p;
  I.c3 = I.c1;
  const int ay = c->dim == 3 ? 1 : 0;
  I.cfwd = base_args(c, b.tab_d, ay, mode);
  I.cfwd.ctl = ctl; I.cfwd.solver = 1; I.cfwd.s = b.s;
  I.cinv = I.cfwd;
  I.ccore = base_args(c, b.tab_d, c->dim - 1, mode);
  I.ccore.ctl = ctl; I.ccore.solver = 1; I.ccore.s = b.s;
  // p_n and the step-size moments
  I.ax = base_args(c, b.tab_d, 0, mode);
  I.ax.V = b.V;
  I.ax.ctl = ctl; I.ax.solver = 1; I.ax.phi = b.phi; I.ax.s = b.s; I.ax.t = b.t; I.ax.p = b.p;
  for (int ax = 1; ax < 3; ++ax) {
    PassArgs& m = I.amid[ax - 1];
    m = base_args(c, b.tab_d, ax < c->dim ? ax : 0, mode);
    m.ctl = ctl; m.solver = 1; m.phi = b.phi; m.p = b.p; m.last_axis = (ax == c->dim - 1);
    m.cond = m.last_axis ? cond : 0ull;
  }
  return I;
}

// One PCG iteration (all passes) in launch mode `mode` as separate launches.
static gpe_status enqueue_iteration(gpe_ctx* c, int mode, cudaStream_t st, unsigned long long cond) {
  const IterArgs I = iter_args(c, mode, cond);
  GPE_CU(c, launch(mode, P_HX, I.hx, st));
  for (int ax = 1; ax < c->dim; ++ax) GPE_CU(c, launch(mode, P_HMID, I.hmid[ax - 1], st));
  GPE_CU(c, launch(mode, P_C1, I.c1, st));
  if (c->dim == 3) GPE_CU(c, launch(mode, P_CFWD, I.cfwd, st));
  GPE_CU(c, launch(mode, P_CCORE, I.ccore, st));
  if (c->dim == 3) GPE_CU(c, launch(mode, P_CINV, I.cinv, st));
  GPE_CU(c, launch(mode, P_C3, I.c3, st));
  GPE_CU(c, launch(mode, P_AX, I.ax, st));
  for (int ax = 1; ax < c->dim; ++ax) GPE_CU(c, launch(mode, P_AMID, I.amid[ax - 1], st));
  return GPE_OK;
}

// Square (2D, n in {64..512}) and cubic (3D, n in {64, 128, 256}) grids run the
// whole loop in one persistent cooperative kernel.
static bool persist_eligible(const gpe_ctx* c) {
  const int M = c->n[0];
  if (c->n[1] != M) return false;
  if (c->dim == 2) return M >= 64 && M <= 512;
  return c->n[2] == M && M >= 64 && M <= 256;
}

static cudaError_t launch_persist(int mode, int M, int dim, const PersistArgs& P, int grid, int block, size_t smem,
                                  cudaStream_t st, int* mb) {
  if (mode == 0) return launch_persist_m0(M, dim, P, grid, block, smem, st, mb);
  if (mode == 1) return launch_persist_m1(M, dim, P, grid, block, smem, st, mb);
  return launch_persist_m2(M, dim, P, grid, block, smem, st, mb);
}

// Launch the persistent solve for one phase.  *launched = false when the
// kernel cannot be made co-resident (the caller falls back to the graph).
static gpe_status run_persistent(gpe_ctx* c, int mode, bool* launched, int wait_polls) {
  *launched = false;
  const int M = c->n[0];
  const int Tl = M / 8;
  const long long nlines = (long long)c->n[1] * (c->dim == 3 ? c->n[2] : 1);
  // lines (x) or columns (y, z) per work unit: enough units for one block per
  // SM (FP64 passes are bound by the per-SM FP64 rate), at most 256 threads
  int g = 1;
  while (2 * g * Tl <= 256 && nlines / (2 * g) >= c->nsm) g *= 2;
  if (g * Tl < 32 && 32 / Tl <= nlines && 32 / Tl <= c->n[0]) g = 32 / Tl;  // at least one warp
  const int block = g * Tl;
  IterArgs I = iter_args(c, mode, 0ull);
  const long long units = nlines / g;
  auto setx = [&](PassArgs& a) { a.lpb = g; a.nblocks = (int)units; };
  auto sets = [&](PassArgs& a, int axis) {
    a.tx = g; a.ntx = c->n[0] / g;
    a.nblocks = (int)units;
    a.stride = (axis == 1) ? c->n[0] : (long long)c->n[0] * c->n[1];
    a.outer_stride = (axis == 1) ? (long long)c->n[0] * c->n[1] : c->n[0];
  };
  PersistArgs P;
  std::memset(&P, 0, sizeof(P));
  P.hx = I.hx; setx(P.hx);
  P.hy = I.hmid[0]; sets(P.hy, 1);
  P.hz = I.hmid[1]; if (c->dim == 3) sets(P.hz, 2);
  P.c1 = I.c1; setx(P.c1);
  P.c3 = I.c3; setx(P.c3);
  P.cfwd = I.cfwd; if (c->dim == 3) sets(P.cfwd, 1);
  P.cinv = I.cinv; if (c->dim == 3) sets(P.cinv, 1);
  P.ccore = I.ccore; sets(P.ccore, c->dim - 1);
  P.ax = I.ax; setx(P.ax);
  P.ay = I.amid[0]; sets(P.ay, 1);
  P.az = I.amid[1]; if (c->dim == 3) sets(P.az, 2);
  P.ctl = c->ctl_solve;
  P.partials = c->pers_partials;
  P.bar = c->pers_bar;
  P.err = reinterpret_cast<int*>(c->pers_bar + 2);
  P.units = units;
  P.spin_limit = wait_polls > 0 ? (long long)wait_polls : kSpinLimit;
  // dynamic shared memory: the larger of an x unit and a y/z unit, in the
  // widest transform type of this mode
  const size_t csz = (mode == 0) ? 8 : 16;
  const size_t smx = (size_t)g * (M + M / 16) * csz, sms = (size_t)M * g * csz;
  const size_t smem = smx > sms ? smx : sms;
  int mb = 0;
  cudaError_t e = launch_persist(mode, M, c->dim, P, 0, block, smem, c->st, &mb);
  if (e != cudaSuccess || mb <= 0) {
    cudaGetLastError();
    c->err = std::string("persistent kernel not co-resident, graph loop used: ") +
             (e != cudaSuccess ? cudaGetErrorString(e) : "occupancy 0");
    return GPE_OK;
  }
  long long grid = (long long)mb * c->nsm;
  if (grid > units) grid = units;
  if (grid > c->pers_max_grid) grid = c->pers_max_grid;
  GPE_CU(c, cudaMemsetAsync(c->pers_bar, 0, 4 * sizeof(unsigned), c->st));
  GPE_CU(c, launch_persist(mode, M, c->dim, P, (int)grid, block, smem, c->st, nullptr));
  *launched = true;
  return GPE_OK;
}

static gpe_status build_graph(gpe_ctx* c, int mode) {
  if (c->exec[mode]) return GPE_OK;
  cudaGraph_t g = nullptr;
  GPE_CU(c, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  GPE_CU(c, cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  GPE_CU(c, cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  GPE_CU(c, cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  gpe_status s = enqueue_iteration(c, mode, c->cap, (unsigned long long)h);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &captured);
  if (s != GPE_OK) { cudaGraphDestroy(g); return s; }
  if (e != cudaSuccess) { c->err = std::string("capture: ") + cudaGetErrorString(e); cudaGraphDestroy(g); return GPE_ERR_CUDA; }
  e = cudaGraphInstantiate(&c->exec[mode], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { c->err = std::string("instantiate: ") + cudaGetErrorString(e); c->exec[mode] = nullptr; return GPE_ERR_CUDA; }
  return GPE_OK;
}

// Make sure every pass kernel of precision prec has had its attributes set
// (first launch) before capture: one iteration with done = 1 exits at once.
static gpe_status warm_kernels(gpe_ctx* c, int mode) {
  if (c->warmed[mode]) return GPE_OK;
  Ctl h;
  std::memset(&h, 0, sizeof(h));
  h.done = 1;
  GPE_CU(c, cudaMemcpyAsync(c->ctl_solve, &h, sizeof(Ctl), cudaMemcpyHostToDevice, c->st));
  gpe_status s = enqueue_iteration(c, mode, c->st, 0ull);
  if (s != GPE_OK) return s;
  GPE_CU(c, cudaStreamSynchronize(c->st));
  c->warmed[mode] = true;
  return GPE_OK;
}

static gpe_status run_phase(gpe_ctx* c, int mode, Ctl& h, const gpe_solve_opts& o, bool keep_direction = false) {
  const IterBufs b = iter_bufs(c, mode);
  const size_t sbytes = (b.tab_h ? 16 : 8) * (size_t)c->N;
  const size_t dbytes = (b.tab_d ? 16 : 8) * (size_t)c->N;
  gpe_status s = warm_kernels(c, mode);
  if (s != GPE_OK) return s;
  if (!keep_direction) {
    GPE_CU(c, cudaMemsetAsync(b.p, 0, dbytes, c->st));
    GPE_CU(c, cudaMemsetAsync(b.r_prev, 0, sbytes, c->st));
  }
  GPE_CU(c, cudaMemcpyAsync(c->ctl_solve, &h, sizeof(Ctl), cudaMemcpyHostToDevice, c->st));
  GPE_CU(c, launch_init_norm(b.tab_h, b.phi, c->N, c->weight, c->ctl_solve, c->partials, c->ticket, c->st));
  bool done_launch = false;
  int loop = o.use_graph ? 1 : 0;
  if (o.use_graph == 3 && mode == 0 && c->dim == 2 && c->n[0] == c->n[1] && c->n[0] >= 32 && c->n[0] <= 256) {
    // the complex64 phase held in one thread-block cluster's shared memory
    ClusterSolveArgs P;
    std::memset(&P, 0, sizeof(P));
    P.base = iter_args(c, 0, 0ull).hx;
    P.phi = static_cast<float2*>(b.phi);
    P.V = static_cast<const float*>(b.V);
    P.ctl = c->ctl_solve;
    cudaError_t e = launch_cluster_solve(c->n[0], P, c->st);
    if (e == cudaSuccess) {
      done_launch = true;
      loop = 3;
    } else {
      cudaGetLastError();
      c->err = std::string("cluster solve unavailable, graph loop used: ") + cudaGetErrorString(e);
    }
  }
  if (!done_launch && o.use_graph == 2 && persist_eligible(c)) {
    s = run_persistent(c, mode, &done_launch, o.wait_polls);
    if (s != GPE_OK) return s;
    if (done_launch) loop = 2;
  }
  if (mode == 0 || c->prob.prec != GPE_MIXED) c->last_loop = loop;  // a mixed solve reports its complex64 phase's loop
  if (done_launch) {
  } else if (o.use_graph) {
    s = build_graph(c, mode);
    if (s != GPE_OK) return s;
    GPE_CU(c, cudaGraphLaunch(c->exec[mode], c->st));
  } else {
    int k = 0;
    while (true) {
      s = enqueue_iteration(c, mode, c->st, 0ull);
      if (s != GPE_OK) return s;
      if (++k % 16 == 0) {
        int done = 0;
        GPE_CU(c, cudaMemcpyAsync(&done, &c->ctl_solve->done, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        GPE_CU(c, cudaStreamSynchronize(c->st));
        if (done) break;
      }
    }
  }
  GPE_CU(c, cudaMemcpyAsync(&h, c->ctl_solve, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st));
  int wait_failed = 0;
  if (loop == 2)  // a barrier wait of the persistent kernel gave up (any block)
    GPE_CU(c, cudaMemcpyAsync(&wait_failed, c->pers_bar + 2, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  GPE_CU(c, cudaStreamSynchronize(c->st));
  if (wait_failed) {
    h.status = GPE_ERR_TIMEOUT;
    h.done = 1;
  }
  return GPE_OK;
}

// Control block at the start of a solve (options, loop state, the
// single-precision floor estimate used by the complex64 phase's switch rule).
static Ctl solve_ctl(const gpe_ctx* c, const gpe_solve_opts& o, int log_cap) {
  Ctl h;
  std::memset(&h, 0, sizeof(h));
  h.tol_res_inf = o.tol_res_inf; h.tol_dE = o.tol_dE; h.theta_default = o.theta_default; h.switch_res = o.switch_res;
  h.max_iter = o.max_iter; h.max_backtracks = o.max_backtracks; h.cg = o.cg; h.stall_window = o.stall_window;
  h.log = log_cap ? c->log_dev : nullptr; h.log_cap = log_cap; h.log_len = 0;
  h.restart = 1; h.anchor_res = 1e300; h.anchor_iter = 0;
  h.pc_kind = o.precond; h.beta_rule = o.beta_rule; h.line_search = o.line_search;
  double k2 = 0.0;  // max over the grid of |k|^2 / 2 (corner mode -M/2 on every axis)
  for (int i = 0; i < c->dim; ++i) {
    const double km = 0.5 * c->n[i] * M_PI / c->prob.L[i];
    k2 += 0.5 * km * km;
  }
  h.floor_coef = 5.96e-8 * (k2 + (c->vmax > 0.0 ? c->vmax : 0.0));
  h.switch_fac = 4.0;
  return h;
}

static gpe_status check_opts(gpe_solve_opts& o, std::string& err) {
  if (o.max_iter < 0 || o.max_backtracks < 0 || !(o.tol_res_inf >= 0.0) || o.stall_window < 1 || o.precond < 0 ||
      o.precond > 5 || o.beta_rule < 0 || o.beta_rule > 1 || o.line_search < 0 || o.line_search > 1 ||
      o.wait_polls < 0) {
    err = "invalid solve options";
    return GPE_ERR_ARG;
  }
  if (o.max_iter_lo <= 0) o.max_iter_lo = o.max_iter;
  return GPE_OK;
}

// ---------------------------------------------------------------------------
// Plans of the pass kernels and their tuner
// ---------------------------------------------------------------------------
// Thread cap of a launch mode's kernels (launch bounds: 512 with single-
// precision transforms, 256 once a double or double-single type is involved)
// and the largest element size its passes stage in shared memory.
static int mode_max_threads(int mode) { return mode == 0 ? 512 : 256; }
static size_t mode_elem_bytes(int mode) { return mode == 0 ? 8 : 16; }
static bool mode_available(const gpe_ctx* c, int mode) { return mode >= 0 && mode < 3 && c->pb[mode].on; }

// A plan for (mode, axis): E values per thread (4 or 8), `width` lines per
// block (axis 0) or adjacent x-columns per tile (axes 1, 2).  False when the
// kernels cannot run it (thread cap, shared memory, partials capacity).
static bool make_plan(const gpe_ctx* c, int mode, int axis, int E, int width, PassPlan& pl) {
  if (axis < 0 || axis >= c->dim) return false;
  const int M = c->n[axis];
  if (!(E == 8 || (E == 4 && M >= 32))) return false;
  if (width < 1 || (width & (width - 1)) != 0) return false;
  const int Tl = M / E;
  if ((long long)Tl * width > mode_max_threads(mode)) return false;
  PassPlan q;
  q.M = M;
  q.E = E;
  if (axis == 0) {
    const long long nlines = (long long)c->n[1] * (c->dim == 3 ? c->n[2] : 1);
    if (width > nlines) return false;
    if ((size_t)width * (M + M / 16) * mode_elem_bytes(mode) > 200 * 1024) return false;
    q.lpb = width;
    q.nblocks = (int)(nlines / width);
  } else {
    const int nx = c->n[0];
    if (width > nx) return false;
    if ((size_t)M * width * mode_elem_bytes(mode) > 200 * 1024) return false;
    const long long outer = (axis == 1) ? (c->dim == 3 ? c->n[2] : 1) : c->n[1];
    q.tx = width;
    q.ntx = nx / width;
    q.nblocks = (int)((long long)q.ntx * outer);
    q.stride = (axis == 1) ? nx : (long long)nx * c->n[1];
    q.outer_stride = (axis == 1) ? (long long)nx * c->n[1] : nx;
  }
  if (q.nblocks < 1 || q.nblocks > c->partials_cap) return false;
  pl = q;
  return true;
}

static void plans_changed(gpe_ctx* c, int mode) {
  if (c->exec[mode]) cudaGraphExecDestroy(c->exec[mode]);
  c->exec[mode] = nullptr;
  c->warmed[mode] = false;
}

static bool hbatch_eligible(const gpe_ctx* c) {
  return c->dim == 2 && c->n[0] == c->n[1] && c->n[0] >= 32 && c->n[0] <= 256;
}

extern "C" gpe_status gpe_set_plan(gpe_ctx* c, int mode, int axis, int E, int width) {
  if (!c) return GPE_ERR_ARG;
  if (mode == 3) {  // the cluster kernel of gpe_apply_H_batch: E only, width = rows per CTA
    // width: rows per CTA, 16; or 32 for the streaming form (E = 16, n >= 64)
    const bool ok = hbatch_eligible(c) && axis == 0 && (width == 16 || (width == 32 && E == 16)) &&
                    (E == 8 || (E == 16 && c->work == 0 && c->n[0] >= 64));
    if (!ok) { c->err = "plan not supported by the batched H kernel"; return GPE_ERR_ARG; }
    GPE_CU(c, cudaStreamSynchronize(c->st));
    c->hbatch_E = E;
    c->hbatch_rows = width;
    return GPE_OK;
  }
  if (!mode_available(c, mode)) { c->err = "launch mode not used by this context"; return GPE_ERR_ARG; }
  PassPlan pl;
  if (!make_plan(c, mode, axis, E, width, pl)) { c->err = "plan not supported for this grid and mode"; return GPE_ERR_ARG; }
  GPE_CU(c, cudaStreamSynchronize(c->st));
  c->mplan[mode][axis] = pl;
  plans_changed(c, mode);
  return GPE_OK;
}

extern "C" gpe_status gpe_get_plan(const gpe_ctx* c, int mode, int axis, int* E, int* width) {
  if (c && E && width && mode == 3 && axis == 0 && hbatch_eligible(c)) {
    *E = c->hbatch_E;
    *width = c->hbatch_E == 16 ? c->hbatch_rows : 16;
    return GPE_OK;
  }
  if (!c || !E || !width || mode < 0 || mode > 2 || axis < 0 || axis >= c->dim) return GPE_ERR_ARG;
  const PassPlan& pl = c->mplan[mode][axis];
  *E = pl.E;
  *width = axis == 0 ? pl.lpb : pl.tx;
  return GPE_OK;
}

// Microseconds per iteration of launch mode `mode` with the current plans:
// `iters` solver iterations (host-launched passes, after two warm-up
// iterations) from a normalised Gaussian, best of two runs.
static gpe_status tune_time(gpe_ctx* c, int mode, int iters, const std::vector<double>& g128, double* us) {
  const IterBufs b = iter_bufs(c, mode);
  cudaStream_t st = c->st;
  const long long N = c->N;
  gpe_solve_opts o;
  gpe_solve_opts_default(&o);
  o.tol_res_inf = 0.0;
  o.max_iter = 1 << 30;
  Ctl h = solve_ctl(c, o, 0);
  h.lo_phase = 0; h.phase = 1; h.max_iter_phase = o.max_iter; h.stall_switch = 0;
  cudaEvent_t e0, e1;
  GPE_CU(c, cudaEventCreate(&e0));
  GPE_CU(c, cudaEventCreate(&e1));
  double best = 1e300;
  gpe_status s = GPE_OK;
  for (int rep = 0; rep < 2 && s == GPE_OK; ++rep) {
    cudaError_t e = cudaMemcpyAsync(c->pb[1].phi, g128.data(), 16 * (size_t)N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && mode != 1) e = launch_convert_c128_to_c64(c->pb[1].phi, c->pb[0].phi, N, st);
    if (e == cudaSuccess && mode == 2) e = launch_convert_c64_to_ds(c->pb[0].phi, c->pb[2].phi, N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.p, 0, (b.tab_d ? 16 : 8) * (size_t)N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.r_prev, 0, (b.tab_h ? 16 : 8) * (size_t)N, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ctl_solve, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_init_norm(b.tab_h, b.phi, N, c->weight, c->ctl_solve, c->partials, c->ticket, st);
    if (e != cudaSuccess) { c->err = std::string("tuner set-up: ") + cudaGetErrorString(e); s = GPE_ERR_CUDA; break; }
    for (int k = 0; k < 2 && s == GPE_OK; ++k) s = enqueue_iteration(c, mode, st, 0ull);
    if (s != GPE_OK) break;
    e = cudaEventRecord(e0, st);
    for (int k = 0; k < iters && s == GPE_OK && e == cudaSuccess; ++k) s = enqueue_iteration(c, mode, st, 0ull);
    if (s != GPE_OK) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { c->err = std::string("tuner timing: ") + cudaGetErrorString(e); s = GPE_ERR_CUDA; break; }
    const double t = 1000.0 * ms / iters;
    best = t < best ? t : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *us = best;
  return s;
}

namespace {
std::mutex g_tune_mu;
std::map<std::array<int, 5>, std::array<PassPlan, 3>> g_tune_cache;  // (dim, n, mode) -> plans per axis
}  // namespace

extern "C" gpe_status gpe_autotune(gpe_ctx* c, int iters, int use_cache, gpe_tune_report* rep) {
  if (!c) return GPE_ERR_ARG;
  if (iters < 1) { c->err = "iters must be >= 1"; return GPE_ERR_ARG; }
  gpe_tune_report r;
  std::memset(&r, 0, sizeof(r));
  r.cached = 1;
  GPE_CU(c, cudaStreamSynchronize(c->st));
  // a normalised Gaussian exp(-|x|^2 / 2) on the grid (host, FP64)
  std::vector<double> g128(2 * (size_t)c->N, 0.0);
  {
    double nrm = 0.0;
    for (long long i = 0; i < c->N; ++i) {
      long long k = i;
      double r2 = 0.0;
      for (int ax = 0; ax < c->dim; ++ax) {
        const double x = -c->prob.L[ax] + (double)(k % c->n[ax]) * c->h[ax];
        k /= c->n[ax];
        r2 += x * x;
      }
      g128[2 * i] = std::exp(-0.5 * r2);
      nrm += g128[2 * i] * g128[2 * i];
    }
    const double sc = 1.0 / std::sqrt(nrm * c->weight);
    for (long long i = 0; i < c->N; ++i) g128[2 * i] *= sc;
  }
  for (int mode = 0; mode < 3; ++mode) {
    if (!mode_available(c, mode)) continue;
    const std::array<int, 5> key = {c->dim, c->n[0], c->n[1], c->dim == 3 ? c->n[2] : 1, mode};
    bool hit = false;
    if (use_cache) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        for (int ax = 0; ax < c->dim; ++ax) c->mplan[mode][ax] = it->second[ax];
        hit = true;
      }
    }
    if (!hit) {
      r.cached = 0;
      double cur = 0.0;
      gpe_status s = tune_time(c, mode, iters, g128, &cur);
      if (s != GPE_OK) return s;
      r.us_before[mode] = cur;
      // coordinate descent over the axes: every (E, width) for one axis with
      // the other axes at their current choice; a change must gain 2%
      for (int ax = 0; ax < c->dim; ++ax) {
        PassPlan best = c->mplan[mode][ax];
        for (int E : {8, 4}) {
          for (int w = 1; w <= 512; w *= 2) {
            PassPlan cand;
            if (!make_plan(c, mode, ax, E, w, cand)) continue;
            if (cand.E == best.E && cand.lpb == best.lpb && cand.tx == best.tx) continue;
            c->mplan[mode][ax] = cand;
            double t = 0.0;
            s = tune_time(c, mode, iters, g128, &t);
            ++r.candidates;
            if (s != GPE_OK) { c->mplan[mode][ax] = best; return s; }
            if (t < 0.98 * cur) { cur = t; best = cand; }
          }
        }
        c->mplan[mode][ax] = best;
      }
      r.us_after[mode] = cur;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      std::array<PassPlan, 3> pl;
      for (int ax = 0; ax < 3; ++ax) pl[ax] = c->mplan[mode][ax];
      g_tune_cache[key] = pl;
    }
    for (int ax = 0; ax < c->dim; ++ax) {
      r.E[mode][ax] = c->mplan[mode][ax].E;
      r.width[mode][ax] = ax == 0 ? c->mplan[mode][ax].lpb : c->mplan[mode][ax].tx;
    }
    plans_changed(c, mode);
  }
  if (rep) *rep = r;
  return GPE_OK;
}

extern "C" gpe_status gpe_pcg_solve(gpe_ctx* c, void* phi_inout, const gpe_solve_opts* opts, gpe_report* rep) {
  if (!c) return GPE_ERR_ARG;
  if (!phi_inout) { c->err = "null phi"; return GPE_ERR_ARG; }
  gpe_solve_opts o;
  gpe_solve_opts_default(&o);
  if (opts) o = *opts;
  if (check_opts(o, c->err) != GPE_OK) return GPE_ERR_ARG;
  const int log_cap = (rep && rep->log && rep->log_cap > 0) ? rep->log_cap : 0;
  if (log_cap > c->log_dev_cap) {
    cudaFree(c->log_dev);
    c->log_dev = nullptr;
    c->log_dev_cap = 0;
    GPE_CU(c, cudaMalloc(&c->log_dev, sizeof(double) * kLogFields * (size_t)log_cap));
    c->log_dev_cap = log_cap;
  }
  const bool dev = is_device_ptr(phi_inout);
  const size_t b128 = 16 * (size_t)c->N;
  GPE_CU(c, cudaMemcpyAsync(c->pb[1].phi, phi_inout, b128, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));

  Ctl h = solve_ctl(c, o, log_cap);
  int iters_lo = 0, iters_hi = 0;
  gpe_status s;
  if (c->prob.prec == GPE_MIXED) {
    GPE_CU(c, launch_convert_c128_to_c64(c->pb[1].phi, c->pb[0].phi, c->N, c->st));
    h.lo_phase = 1; h.phase = 0; h.iter_phase0 = 0; h.max_iter_phase = o.max_iter_lo;
    s = run_phase(c, 0, h, o);
    if (s != GPE_OK) return s;
    iters_lo = h.iter;
    const bool go_on = h.switch_req || h.status == 0;  // a complex64 "success" is refined too
    if (h.status == GPE_ERR_NONFINITE || h.status == GPE_ERR_PRECOND) {
      // keep the input in the complex128 buffer; report the failure
    } else {
      // the last complex64 iterate: the refinement's start, or the answer when
      // the iteration cap ended the solve in the complex64 phase
      GPE_CU(c, launch_convert_c64_to_c128(c->pb[0].phi, c->pb[1].phi, c->N, c->st));
    }
    if (go_on && h.iter < o.max_iter) {
      const bool keep = !o.refine_restart;
      h.done = 0; h.status = 0; h.switch_req = 0; h.lo_phase = 0; h.phase = 1; h.restart = keep ? 0 : 1;
      h.stop_dE = 0;
      h.iter_phase0 = h.iter; h.max_iter_phase = o.max_iter;
      h.stall_switch = 1; h.anchor_res = 1e300; h.anchor_iter = h.iter;
      // the refinement state lives in double-single: phi (and, when the
      // direction is kept, r_{n-1}; p is complex64 in both phases)
      GPE_CU(c, launch_convert_c64_to_ds(c->pb[0].phi, c->pb[2].phi, c->N, c->st));
      if (keep) GPE_CU(c, launch_convert_c64_to_ds(c->pb[0].r_prev, c->pb[2].r_prev, c->N, c->st));
      s = run_phase(c, 2, h, o, keep);  // refinement: double-single state, FP32 direction
      if (s != GPE_OK) return s;
      if (h.status != GPE_ERR_NONFINITE && h.status != GPE_ERR_PRECOND)
        GPE_CU(c, launch_convert_ds_to_c128(c->pb[2].phi, c->pb[1].phi, c->N, c->st));
      if (h.switch_req && h.stall_switch && h.iter < o.max_iter) {
        // the refinement stalled: complete the solve in FP64 from its last iterate
        iters_hi = h.iter;
        h.done = 0; h.status = 0; h.switch_req = 0; h.phase = 2; h.restart = 1; h.stop_dE = 0;
        h.iter_phase0 = h.iter; h.max_iter_phase = o.max_iter; h.stall_switch = 0;
        s = run_phase(c, 1, h, o);
        if (s != GPE_OK) return s;
      }
    }
  } else {
    h.lo_phase = 0; h.phase = 1; h.max_iter_phase = o.max_iter;
    s = run_phase(c, 1, h, o);
    if (s != GPE_OK) return s;
  }
  GPE_CU(c, cudaMemcpyAsync(phi_inout, c->pb[1].phi, b128, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  GPE_CU(c, cudaStreamSynchronize(c->st));
  if (rep) {
    rep->status = h.status; rep->iters = h.iter; rep->iters_lo = iters_lo;
    rep->fallbacks = h.fallbacks; rep->backtracks = h.backtracks_total;
    rep->E = h.E; rep->lambda = h.lam; rep->res_inf = h.res_inf; rep->res_l2 = h.res_l2;
    rep->loop_kind = c->last_loop;
    rep->iters_fp64 = iters_hi ? h.iter - iters_hi : 0;
    rep->log_len = 0;
    if (log_cap) {
      int nrows = h.iter + 1 < log_cap ? h.iter + 1 : log_cap;
      GPE_CU(c, cudaMemcpy(rep->log, c->log_dev, sizeof(double) * kLogFields * (size_t)nrows, cudaMemcpyDeviceToHost));
      rep->log_len = nrows;
    }
  }
  if (h.status != GPE_OK) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "solve ended with status %d after %d iterations (res_inf %.3e)", h.status, h.iter,
                  h.res_inf);
    c->err = buf;
  }
  return (gpe_status)h.status;
}

// ---------------------------------------------------------------------------
// Batched solves: one CUDA graph with one branch per instance
// ---------------------------------------------------------------------------
struct gpe_batch {
  std::vector<gpe_ctx*> ctx;
  std::vector<Ctl*> ctl_init;  // device copies of each solve's starting control block
  cudaStream_t st = nullptr;    // caller's stream
  cudaStream_t cap = nullptr;   // capture of the branches
  cudaStream_t body = nullptr;  // capture of the loop bodies
  cudaGraphExec_t exec = nullptr;
  std::string err;
};

static bool cluster_eligible(const gpe_ctx* c) {
  return c->dim == 2 && c->n[0] == c->n[1] && c->n[0] >= 32 && c->n[0] <= 256;
}

// Append a WHILE node after the nodes captured so far on st; its body, one
// iteration of launch mode `mode` whose last pass re-arms h, is captured on body_st.
static gpe_status capture_while(gpe_batch* B, gpe_ctx* c, int mode, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  GPE_CU(B, cudaStreamGetCaptureInfo(B->cap, &cs, nullptr, &graph, &deps, &ed, &nd));
  if (cs != cudaStreamCaptureStatusActive) { B->err = "batch capture is not active"; return GPE_ERR_CUDA; }
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  GPE_CU(B, cudaGraphAddNode(&node, graph, deps, ed, nd, &np));
  GPE_CU(B, cudaStreamUpdateCaptureDependencies(B->cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  GPE_CU(B, cudaStreamBeginCaptureToGraph(B->body, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed));
  gpe_status s = enqueue_iteration(c, mode, B->body, (unsigned long long)h);
  cudaGraph_t got = nullptr;
  cudaError_t e = cudaStreamEndCapture(B->body, &got);
  if (s != GPE_OK) { B->err = c->err; return s; }
  if (e != cudaSuccess) { B->err = std::string("loop body capture: ") + cudaGetErrorString(e); return GPE_ERR_CUDA; }
  return GPE_OK;
}

static gpe_status new_handle(gpe_batch* B, unsigned dflt, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  GPE_CU(B, cudaStreamGetCaptureInfo(B->cap, &cs, nullptr, &graph, nullptr, nullptr, nullptr));
  GPE_CU(B, cudaGraphConditionalHandleCreate(h, graph, dflt, cudaGraphCondAssignDefault));
  return GPE_OK;
}

// One instance's whole solve, captured on B->cap: the steps of gpe_pcg_solve
// with the host's decisions between the phases taken by batch kernels.
static gpe_status batch_enqueue(gpe_batch* B, gpe_ctx* c, Ctl* ctl_init) {
  cudaStream_t st = B->cap;
  const long long N = c->N;
  gpe_status s;
  GPE_CU(B, cudaMemcpyAsync(c->ctl_solve, ctl_init, sizeof(Ctl), cudaMemcpyDeviceToDevice, st));
  auto clear_dir = [&](const IterBufs& b) -> gpe_status {
    GPE_CU(B, cudaMemsetAsync(b.p, 0, (b.tab_d ? 16 : 8) * (size_t)N, st));
    GPE_CU(B, cudaMemsetAsync(b.r_prev, 0, (b.tab_h ? 16 : 8) * (size_t)N, st));
    return GPE_OK;
  };
  if (c->prob.prec != GPE_MIXED) {
    const IterBufs b1 = iter_bufs(c, 1);
    if ((s = clear_dir(b1)) != GPE_OK) return s;
    GPE_CU(B, launch_init_norm(b1.tab_h, b1.phi, N, c->weight, c->ctl_solve, c->partials, c->ticket, st));
    cudaGraphConditionalHandle h;
    if ((s = new_handle(B, 1, &h)) != GPE_OK) return s;
    return capture_while(B, c, 1, h);
  }
  const IterBufs b0 = iter_bufs(c, 0);
  GPE_CU(B, launch_convert_c128_to_c64(c->pb[1].phi, c->pb[0].phi, N, st));
  if ((s = clear_dir(b0)) != GPE_OK) return s;
  GPE_CU(B, launch_init_norm(b0.tab_h, b0.phi, N, c->weight, c->ctl_solve, c->partials, c->ticket, st));
  if (cluster_eligible(c)) {
    ClusterSolveArgs P;
    std::memset(&P, 0, sizeof(P));
    P.base = iter_args(c, 0, 0ull).hx;
    P.phi = static_cast<float2*>(b0.phi);
    P.V = static_cast<const float*>(b0.V);
    P.ctl = c->ctl_solve;
    GPE_CU(B, launch_cluster_solve(c->n[0], P, st));
  } else {
    cudaGraphConditionalHandle h0;
    if ((s = new_handle(B, 1, &h0)) != GPE_OK) return s;
    if ((s = capture_while(B, c, 0, h0)) != GPE_OK) return s;
  }
  const IterBufs b2 = iter_bufs(c, 2);
  GPE_CU(B, launch_batch_between(c->pb[0].phi, c->pb[1].phi, c->pb[2].phi, N, c->ctl_solve, st));
  if ((s = clear_dir(b2)) != GPE_OK) return s;
  GPE_CU(B, launch_init_norm(b2.tab_h, b2.phi, N, c->weight, c->ctl_solve, c->partials, c->ticket, st));
  cudaGraphConditionalHandle h2;
  if ((s = new_handle(B, 0, &h2)) != GPE_OK) return s;
  GPE_CU(B, launch_batch_gate(c->ctl_solve, (unsigned long long)h2, st));
  if ((s = capture_while(B, c, 2, h2)) != GPE_OK) return s;
  GPE_CU(B, launch_batch_final(c->pb[2].phi, c->pb[1].phi, N, c->ctl_solve, st));
  // FP64 completion when the refinement stalled
  const IterBufs b1 = iter_bufs(c, 1);
  if ((s = clear_dir(b1)) != GPE_OK) return s;
  GPE_CU(B, launch_init_norm(b1.tab_h, b1.phi, N, c->weight, c->ctl_solve, c->partials, c->ticket, st));
  cudaGraphConditionalHandle h3;
  if ((s = new_handle(B, 0, &h3)) != GPE_OK) return s;
  GPE_CU(B, launch_batch_gate64(c->ctl_solve, (unsigned long long)h3, st));
  return capture_while(B, c, 1, h3);
}

static gpe_status batch_build(gpe_batch* B) {
  if (B->exec) return GPE_OK;
  for (gpe_ctx* c : B->ctx) {  // kernel attributes are set outside capture
    gpe_status s = GPE_OK;
    if (c->prob.prec == GPE_MIXED) {
      if ((s = warm_kernels(c, 0)) == GPE_OK) s = warm_kernels(c, 2);
      if (s == GPE_OK) s = warm_kernels(c, 1);
      if (s == GPE_OK && cluster_eligible(c)) GPE_CU(B, prepare_cluster_solve(c->n[0]));
    } else {
      s = warm_kernels(c, 1);
    }
    if (s != GPE_OK) { B->err = c->err; return s; }
  }
  cudaGraph_t g = nullptr;
  GPE_CU(B, cudaGraphCreate(&g, 0));
  for (size_t i = 0; i < B->ctx.size(); ++i) {
    cudaError_t e = cudaStreamBeginCaptureToGraph(B->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { B->err = std::string("batch capture: ") + cudaGetErrorString(e); cudaGraphDestroy(g); return GPE_ERR_CUDA; }
    gpe_status s = batch_enqueue(B, B->ctx[i], B->ctl_init[i]);
    cudaGraph_t got = nullptr;
    e = cudaStreamEndCapture(B->cap, &got);
    if (s != GPE_OK) { cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) { B->err = std::string("batch capture: ") + cudaGetErrorString(e); cudaGraphDestroy(g); return GPE_ERR_CUDA; }
  }
  cudaError_t e = cudaGraphInstantiate(&B->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { B->exec = nullptr; B->err = std::string("batch instantiate: ") + cudaGetErrorString(e); return GPE_ERR_CUDA; }
  return GPE_OK;
}

extern "C" gpe_status gpe_batch_destroy(gpe_batch* B) {
  if (!B) return GPE_OK;
  if (B->st) cudaStreamSynchronize(B->st);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  for (Ctl* p : B->ctl_init) cudaFree(p);
  for (gpe_ctx* c : B->ctx) gpe_destroy(c);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->body) cudaStreamDestroy(B->body);
  delete B;
  return GPE_OK;
}

extern "C" gpe_status gpe_batch_create(int count, const gpe_problem* probs, const double* const* V, void* stream,
                                       gpe_batch** out) {
  if (!out) { g_create_error = "null argument"; return GPE_ERR_ARG; }
  *out = nullptr;
  if (count < 1 || !probs || !V) { g_create_error = "count >= 1, probs and V required"; return GPE_ERR_ARG; }
  gpe_batch* B = new gpe_batch();
  B->st = (cudaStream_t)stream;
  auto fail = [&](gpe_status s, const std::string& msg) {
    g_create_error = msg;
    gpe_batch_destroy(B);
    return s;
  };
  if (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&B->body, cudaStreamNonBlocking) != cudaSuccess)
    return fail(GPE_ERR_CUDA, "stream create failed");
  for (int i = 0; i < count; ++i) {
    gpe_ctx* c = nullptr;
    gpe_status s = gpe_create(&probs[i], V[i], stream, &c);
    if (s != GPE_OK) return fail(s, "instance " + std::to_string(i) + ": " + g_create_error);
    B->ctx.push_back(c);
    Ctl* p = nullptr;
    if (cudaMalloc(&p, sizeof(Ctl)) != cudaSuccess) return fail(GPE_ERR_CUDA, "cudaMalloc control block");
    B->ctl_init.push_back(p);
  }
  *out = B;
  return GPE_OK;
}

extern "C" gpe_status gpe_batch_solve(gpe_batch* B, void* const* phi_inout, const gpe_solve_opts* opts,
                                      gpe_report* reports) {
  if (!B) return GPE_ERR_ARG;
  if (!phi_inout) { B->err = "null phi array"; return GPE_ERR_ARG; }
  gpe_solve_opts o;
  gpe_solve_opts_default(&o);
  if (opts) o = *opts;
  if (check_opts(o, B->err) != GPE_OK) return GPE_ERR_ARG;
  const size_t n = B->ctx.size();
  for (size_t i = 0; i < n; ++i)
    if (!phi_inout[i]) { B->err = "null phi for instance " + std::to_string(i); return GPE_ERR_ARG; }
  std::vector<Ctl> init(n), fin(n);
  std::vector<char> on_dev(n);
  for (size_t i = 0; i < n; ++i) {
    gpe_ctx* c = B->ctx[i];
    init[i] = solve_ctl(c, o, 0);
    if (c->prob.prec == GPE_MIXED) {
      init[i].lo_phase = 1; init[i].phase = 0; init[i].max_iter_phase = o.max_iter_lo;
    } else {
      init[i].lo_phase = 0; init[i].phase = 1; init[i].max_iter_phase = o.max_iter;
    }
    on_dev[i] = is_device_ptr(phi_inout[i]);
    GPE_CU(B, cudaMemcpyAsync(B->ctl_init[i], &init[i], sizeof(Ctl), cudaMemcpyHostToDevice, B->st));
    GPE_CU(B, cudaMemcpyAsync(c->pb[1].phi, phi_inout[i], 16 * (size_t)c->N,
                              on_dev[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, B->st));
  }
  GPE_CU(B, cudaStreamSynchronize(B->st));
  gpe_status s = batch_build(B);
  if (s != GPE_OK) return s;
  GPE_CU(B, cudaGraphLaunch(B->exec, B->st));
  for (size_t i = 0; i < n; ++i) {
    gpe_ctx* c = B->ctx[i];
    GPE_CU(B, cudaMemcpyAsync(phi_inout[i], c->pb[1].phi, 16 * (size_t)c->N,
                              on_dev[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, B->st));
    GPE_CU(B, cudaMemcpyAsync(&fin[i], c->ctl_solve, sizeof(Ctl), cudaMemcpyDeviceToHost, B->st));
  }
  GPE_CU(B, cudaStreamSynchronize(B->st));
  int failed = 0, first_bad = GPE_OK;
  for (size_t i = 0; i < n; ++i) {
    const Ctl& h = fin[i];
    if (h.status != GPE_OK) {
      ++failed;
      if (first_bad == GPE_OK) first_bad = h.status;
    }
    if (reports) {
      gpe_report& r = reports[i];
      r.status = h.status; r.iters = h.iter;
      r.iters_lo = B->ctx[i]->prob.prec == GPE_MIXED ? h.iters_lo : 0;
      r.iters_fp64 = h.iters_hi ? h.iter - h.iters_hi : 0;
      r.fallbacks = h.fallbacks; r.backtracks = h.backtracks_total;
      r.E = h.E; r.lambda = h.lam; r.res_inf = h.res_inf; r.res_l2 = h.res_l2;
      r.log_len = 0;
      r.loop_kind = (B->ctx[i]->prob.prec == GPE_MIXED && cluster_eligible(B->ctx[i])) ? 3 : 1;
    }
  }
  if (failed) {
    B->err = std::to_string(failed) + " of " + std::to_string(n) + " solves did not meet the stopping rule";
    return (gpe_status)first_bad;
  }
  B->err.clear();
  return GPE_OK;
}

extern "C" gpe_status gpe_batch_autotune(gpe_batch* B, int iters) {
  if (!B) return GPE_ERR_ARG;
  for (gpe_ctx* c : B->ctx) {
    const gpe_status s = gpe_autotune(c, iters, 1, nullptr);
    if (s != GPE_OK) { B->err = c->err; return s; }
  }
  if (B->exec) cudaGraphExecDestroy(B->exec);  // rebuilt with the new plans by the next solve
  B->exec = nullptr;
  return GPE_OK;
}

extern "C" const char* gpe_batch_last_error(const gpe_batch* B) { return B ? B->err.c_str() : g_create_error.c_str(); }

