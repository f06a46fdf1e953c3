// gpe_noalloc.cu -- gpe_apply_H_noalloc: H_phi f without any device
// allocation, for callers that must not (or cannot) call cudaMalloc.
//
// Who needs this: code that runs where allocating device memory is not
// allowed or not possible -- inside a host callback or a library that
// promised its users never to touch the allocator, under an external memory
// manager that owns every byte of the device, or after the device memory is
// exhausted -- but that still wants one application of the mean-field
// Hamiltonian.  gpe_create cannot serve them: it allocates the context's
// fields, tables and reduction buffers.
//
// Instead, the intermediate field, the grid tables, the reduction partials
// and the control block live in one file-scope device array of fixed size
// (kScratchBytes below), which every GPU that loads libgpe keeps for the
// life of the process.  All calls share it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "../../include/gpe.h"
#include "gpe_internal.h"

using namespace gpe;

namespace {

// Capacity of the intermediate field: 16 MiB = 2^20 complex128 or 2^21
// complex64 points (512^2, 1024^2 in complex64, 128 x 128 x 64, ...).
constexpr size_t kFieldBytes = size_t(16) << 20;
// Control block, ticket, reduction partials (up to kMaxBlocks blocks) and
// tables (three axes of at most 512 points).
constexpr int kMaxBlocks = 8192;
constexpr size_t kCtlOff = 0;
constexpr size_t kTicketOff = 4096;
constexpr size_t kPartialsOff = 8192;
constexpr size_t kPartialsBytes = size_t(kMaxBlocks) * kMaxMoments * sizeof(double);
constexpr size_t kTablesOff = kPartialsOff + kPartialsBytes;
constexpr size_t kTablesBytes = size_t(3) * 4 * 512 * sizeof(double);  // xi, xc, tw(re, im) per axis
constexpr size_t kFieldOff = (kTablesOff + kTablesBytes + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kFieldOff + kFieldBytes;
static_assert(sizeof(Ctl) <= kTicketOff, "control block must fit before the ticket");

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};  // device address of g_scratch, per device

constexpr int kTargetBlocks = 2 * 152;

void set_err(char* err, size_t len, const char* msg) {
  if (err && len > 0) std::snprintf(err, len, "%s", msg);
}

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; the device address is obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// xi_p = p pi / L (p in DFT order), x_k = -L + k h, twiddles e^{-2 pi i m/M}
// for each axis, in the kernel precision T, from CUDA's sincospi.
template <typename T>
__global__ void k_noalloc_tables(T* base, int dim, int n0, int n1, int n2, double L0, double L1, double L2) {
  const int n[3] = {n0, n1, n2};
  const double L[3] = {L0, L1, L2};
  for (int ax = 0; ax < dim; ++ax) {
    T* xi = base + ax * 4 * 512;
    T* xc = xi + 512;
    T* tw = xc + 512;
    const int M = n[ax];
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
      const int pp = p < M / 2 ? p : p - M;
      xi[p] = (T)(pp * (M_PI / L[ax]));
      xc[p] = (T)(-L[ax] + p * (2.0 * L[ax] / M));
      double s, c;
      sincospi(2.0 * p / M, &s, &c);
      tw[2 * p] = (T)c;
      tw[2 * p + 1] = (T)(-s);
    }
  }
}

static bool pow2_in(int v) { return v >= 8 && v <= 512 && (v & (v - 1)) == 0; }

extern "C" gpe_status gpe_apply_H_noalloc(const gpe_problem* prob, const void* V_dev, const void* phi_dev,
                                          const void* f_dev, void* out_dev, void* stream, char* err,
                                          size_t err_len) {
  if (!prob || !V_dev || !phi_dev || !f_dev || !out_dev) {
    set_err(err, err_len, "null argument");
    return GPE_ERR_ARG;
  }
  if (prob->dim != 2 && prob->dim != 3) { set_err(err, err_len, "dim must be 2 or 3"); return GPE_ERR_ARG; }
  if (prob->prec != GPE_FP64 && prob->prec != GPE_MIXED) { set_err(err, err_len, "unknown precision"); return GPE_ERR_ARG; }
  long long N = 1;
  double weight = 1.0;
  int n[3] = {1, 1, 1};
  for (int i = 0; i < prob->dim; ++i) {
    if (!pow2_in(prob->n[i])) { set_err(err, err_len, "n[i] must be a power of two in [8, 512]"); return GPE_ERR_ARG; }
    if (!(prob->L[i] > 0.0) || !std::isfinite(prob->L[i])) { set_err(err, err_len, "L[i] must be finite and > 0"); return GPE_ERR_ARG; }
    n[i] = prob->n[i];
    N *= n[i];
    weight *= 2.0 * prob->L[i] / n[i];
  }
  if (!std::isfinite(prob->eta) || !std::isfinite(prob->omega)) { set_err(err, err_len, "eta/omega must be finite"); return GPE_ERR_ARG; }
  const int mode = prob->prec == GPE_FP64 ? 1 : 0;
  const size_t csz = mode ? 16 : 8;
  if ((size_t)N * csz > kFieldBytes) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "grid of %lld points needs %zu bytes of scratch; the limit is %zu bytes "
                  "(2^20 complex128 / 2^21 complex64 points)", N, (size_t)N * csz, kFieldBytes);
    set_err(err, err_len, msg);
    return GPE_ERR_UNSUPPORTED;
  }

  // Pass plans for every axis, checked before anything is queued: the same
  // rules as a context's default plans, with the FP64 thread cap.
  const int maxT = 256;
  int lpb = maxT / (n[0] / 8);
  if (lpb < 1) lpb = 1;
  const long long nlines = (long long)n[1] * (prob->dim == 3 ? n[2] : 1);
  while (lpb > 1 && (lpb > nlines || nlines / lpb < kTargetBlocks)) lpb >>= 1;
  int tx_ax[3] = {0, 0, 0};
  long long blocks_ax[3] = {nlines / lpb, 0, 0};
  for (int ax = 1; ax < prob->dim; ++ax) {
    const int nx = n[0];
    const long long outer = (ax == 1) ? (prob->dim == 3 ? n[2] : 1) : n[1];
    int tx = 16 < nx ? 16 : nx;
    while (tx > 1 && tx * (n[ax] / 8) > maxT) tx >>= 1;
    while (tx > 4 && (long long)(nx / tx) * outer < kTargetBlocks) tx >>= 1;
    tx_ax[ax] = tx;
    blocks_ax[ax] = (long long)(nx / tx) * outer;
  }
  for (int ax = 0; ax < prob->dim; ++ax) {
    if (blocks_ax[ax] > kMaxBlocks) {
      char msg[160];
      std::snprintf(msg, sizeof(msg), "axis %d needs %lld thread blocks; the scratch holds reduction partials for "
                    "at most %d", ax, blocks_ax[ax], kMaxBlocks);
      set_err(err, err_len, msg);
      return GPE_ERR_UNSUPPORTED;
    }
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) { set_err(err, err_len, "no usable CUDA device"); return GPE_ERR_CUDA; }
  cudaStream_t st = (cudaStream_t)stream;
  // The device address of the scratch symbol on this device (current).  It is
  // looked up again on every call outside a stream capture, so a module
  // reloaded after cudaDeviceReset is followed; inside a capture the address
  // from the last uncaptured call on this device is used.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;  // treat as capturing: no driver call that capture forbids
  }
  if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
    if (cap != cudaStreamCaptureStatusNone) {
      set_err(err, err_len, "first call on this device inside a stream capture: call once before capturing");
      return GPE_ERR_CUDA;
    }
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) {
      set_err(err, err_len, cudaGetErrorString(e));
      return GPE_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);

  // The reduction ticket must start at zero; the other contents are fully
  // rewritten before they are read.
  e = cudaMemsetAsync(base + kTicketOff, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) { set_err(err, err_len, cudaGetErrorString(e)); return GPE_ERR_CUDA; }
  if (mode)
    k_noalloc_tables<double><<<1, 256, 0, st>>>(reinterpret_cast<double*>(base + kTablesOff), prob->dim, n[0], n[1],
                                                 n[2], prob->L[0], prob->L[1], prob->L[2]);
  else
    k_noalloc_tables<float><<<1, 256, 0, st>>>(reinterpret_cast<float*>(base + kTablesOff), prob->dim, n[0], n[1],
                                                n[2], prob->L[0], prob->L[1], prob->L[2]);
  e = cudaGetLastError();
  if (e != cudaSuccess) { set_err(err, err_len, cudaGetErrorString(e)); return GPE_ERR_CUDA; }

  const size_t tsz = mode ? sizeof(double) : sizeof(float);
  for (int ax = 0; ax < prob->dim; ++ax) {
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.dim = prob->dim; a.nx = n[0]; a.ny = n[1]; a.nz = prob->dim == 3 ? n[2] : 1;
    a.axis = ax; a.M = n[ax];
    a.weight = weight; a.eta = prob->eta; a.omega = prob->omega;
    for (int i = 0; i < 3; ++i) {
      a.xi[i] = base + kTablesOff + (size_t)i * 4 * 512 * tsz;
      a.xc[i] = base + kTablesOff + ((size_t)i * 4 * 512 + 512) * tsz;
    }
    a.tw = base + kTablesOff + ((size_t)ax * 4 * 512 + 1024) * tsz;
    a.V = V_dev;
    a.phi = phi_dev;
    a.f = f_dev;
    a.t = base + kFieldOff;
    a.ctl = reinterpret_cast<Ctl*>(base + kCtlOff);
    a.partials = reinterpret_cast<double*>(base + kPartialsOff);
    a.ticket = reinterpret_cast<unsigned*>(base + kTicketOff);
    if (ax == 0) {
      a.lpb = lpb;
      a.nblocks = (int)blocks_ax[0];
      e = launch_pass(mode, P_HX, a, st);
    } else {
      const int nx = n[0];
      a.tx = tx_ax[ax];
      a.ntx = nx / a.tx;
      a.nblocks = (int)blocks_ax[ax];
      a.stride = (ax == 1) ? nx : (long long)nx * n[1];
      a.outer_stride = (ax == 1) ? (long long)nx * n[1] : nx;
      a.last_axis = (ax == prob->dim - 1);
      a.out = a.last_axis ? out_dev : nullptr;
      e = launch_pass(mode, P_HMID, a, st);
    }
    if (e != cudaSuccess) { set_err(err, err_len, cudaGetErrorString(e)); return GPE_ERR_CUDA; }
  }
  set_err(err, err_len, "");
  return GPE_OK;
}
