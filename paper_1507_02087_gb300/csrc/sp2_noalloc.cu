// An FP64 purification entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while another component owns
// the device memory budget (a framework with its own caching allocator, a plugin
// handed only the buffers it may touch), latency-critical loops that must not enter
// the driver's allocator, and environments where allocation is forbidden outright.
// sp2_run_fp64_noalloc serves them: its workspace is one fixed file-scope device
// array, created when the library's device code is loaded on a GPU and held until
// the process exits.  The caller still passes F and D (and, optionally, an info
// buffer), all in device memory it already owns.  With CUDA's lazy module loading
// (the default), that load may happen inside the first call on a device, which then
// allocates the array (about 4.2 MB); make that first call as a warm-up, outside any
// region where allocation is not allowed and before any stream capture.
//
// The workspace limits the problem size to N <= SP2_NOALLOC_MAX_N.  Every call shares
// the one array, so calls whose work overlaps on the GPU (on different streams, or
// from different threads without ordering) race with each other and must be
// serialised by the caller.  The array keeps what the last call left in it; each call
// zeroes the parts that must start at zero before it uses them.
#include <cuda_runtime.h>

#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sp2.h"
#include "sp2_common.cuh"
#include "sp2_kernels.h"

namespace {

using sp2::DevState;

constexpr int kMaxN = SP2_NOALLOC_MAX_N;
constexpr int kLd = (kMaxN + 63) / 64 * 64;        // padded size of the largest problem
constexpr int kT = kLd / 64;
constexpr int kTiles = kT * (kT + 1) / 2;
constexpr int kGersh = 1024;                       // Gershgorin partial slots
constexpr int kMaxIter = 200;                      // iteration cap (the default of sp2_opts)

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffState = 0;
constexpr size_t kOffLo = align256(kOffState + sizeof(DevState));
constexpr size_t kOffHi = align256(kOffLo + kGersh * sizeof(double));
constexpr size_t kOffBad = align256(kOffHi + kGersh * sizeof(double));
constexpr size_t kOffPart = align256(kOffBad + kGersh * sizeof(int));
constexpr size_t kOffBuf0 = align256(kOffPart + 2 * kTiles * sizeof(double));
constexpr size_t kOffBuf1 = align256(kOffBuf0 + (size_t)kLd * kLd * sizeof(double));
constexpr size_t kScratchBytes = align256(kOffBuf1 + (size_t)kLd * kLd * sizeof(double));

// The workspace.  In host code this name is only a host-side handle for the symbol,
// not a device address: the address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Fixed fields of the state for this call (written by a kernel: no host buffer).
__global__ void noalloc_setup_kernel(DevState* st, int N, int ld, int nocc, int max_iter) {
  st->N = N;
  st->ld = ld;
  st->nocc = nocc;
  st->max_iter = max_iter;
  st->guard = 1;
  st->qtilde = 1.8;
  st->round_fp32 = 0;
}

__global__ void noalloc_info_kernel(const DevState* st, int32_t* info) {
  info[0] = st->status;
  info[1] = st->n_out;
  info[2] = st->reason;
  info[3] = st->hist_len;
}

}  // namespace

static sp2_status run_noalloc(const double* F_dev, double* D_dev, int64_t N, int64_t n_occ, int32_t* info_dev,
                              void* stream);

extern "C" sp2_status sp2_run_fp64_noalloc(const double* F_dev, double* D_dev, int64_t N, int64_t n_occ,
                                           int32_t* info_dev, void* stream) {
  nvtxRangePushA("sp2_run_fp64_noalloc");
  const sp2_status st = run_noalloc(F_dev, D_dev, N, n_occ, info_dev, stream);
  nvtxRangePop();
  return st;
}

static sp2_status run_noalloc(const double* F_dev, double* D_dev, int64_t N, int64_t n_occ, int32_t* info_dev,
                              void* stream) {
  if (!F_dev || !D_dev || N < 1 || n_occ < 0 || n_occ > N) return SP2_ERR_INVALID_ARG;
  if (N > kMaxN) return SP2_ERR_INVALID_ARG;   // larger than the fixed workspace
  const size_t bytes = (size_t)N * N * sizeof(double);
  const char* f = (const char*)F_dev;
  const char* d = (const char*)D_dev;
  if (f < d + bytes && d < f + bytes) return SP2_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  {
    // Set-up, once per device, with that device current: the device address of the
    // workspace.  The first call on a device does this; make it before any stream
    // capture that the later calls may join.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return SP2_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    base = (unsigned char*)g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = (DevState*)(base + kOffState);
  double* lo = (double*)(base + kOffLo);
  double* hi = (double*)(base + kOffHi);
  int* bad = (int*)(base + kOffBad);
  double* part = (double*)(base + kOffPart);
  double* buf0 = (double*)(base + kOffBuf0);
  double* buf1 = (double*)(base + kOffBuf1);
  const int ld = (int)((N + 63) / 64 * 64);
  const int T = ld / 64;
  const int nparts = (int)((N + 7) / 8 < kGersh ? (N + 7) / 8 : kGersh);
  // The iterates need a zero border (rows and columns N .. ld-1); the last call may
  // have left other values there.
  if (cudaMemsetAsync(buf0, 0, (size_t)ld * ld * sizeof(double), s) != cudaSuccess ||
      cudaMemsetAsync(buf1, 0, (size_t)ld * ld * sizeof(double), s) != cudaSuccess) {
    (void)cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  noalloc_setup_kernel<<<1, 1, 0, s>>>(st, (int)N, ld, (int)n_occ, kMaxIter);
  if (cudaGetLastError() != cudaSuccess) return SP2_ERR_CUDA;
  if (sp2::launch_bounds_and_init(st, F_dev, N, (int)N, lo, hi, bad, nparts, s) != cudaSuccess ||
      sp2::launch_scale_f64(st, F_dev, N, (int)N, buf0, ld, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  // At most kMaxIter + 1 squares; once the stop test has fired every launch returns at once.
  for (int it = 0; it <= kMaxIter; ++it) {
    if (sp2::launch_f64_step_plain(st, buf0, buf1, part, T, s) != cudaSuccess) {
      (void)cudaGetLastError();
      return SP2_ERR_CUDA;
    }
  }
  if (sp2::launch_copy_out(st, buf0, buf1, ld, (int)N, D_dev, N, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  if (info_dev) {
    noalloc_info_kernel<<<1, 1, 0, s>>>(st, info_dev);
    if (cudaGetLastError() != cudaSuccess) return SP2_ERR_CUDA;
  }
  return SP2_OK;
}
