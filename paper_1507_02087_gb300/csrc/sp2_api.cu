// C-ABI layer: handles, workspace, the device-controlled loop as a CUDA graph with a
// conditional WHILE node, and the host-buffer entry point.
//
// A run is: bounds + init kernels, the scaling kernel, one launch of the loop graph
// (its body squares once and runs the stop test, which clears the loop condition on
// the device), then the output copy.  Nothing waits on the host in between.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <new>

#include "sp2_common.cuh"
#include "sp2_kernels.h"

using sp2::DevState;

struct sp2_ctx {
  int64_t N = 0, nocc = 0;
  int32_t precision = 0;
  sp2_opts opts{};
  int device = 0;
  int ld = 0, T = 0, nparts = 0;
  double* buf[2] = {nullptr, nullptr};
  double* part = nullptr;
  double* part_lo = nullptr;
  double* part_hi = nullptr;
  int* part_bad = nullptr;
  DevState* st_dev = nullptr;
  DevState* st_host = nullptr;   // pinned mirror for sp2_get_info
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaStream_t last_stream = nullptr;
  bool ran = false;
  double* stage_F = nullptr;     // device staging for sp2_run_host
  double* stage_D = nullptr;
  cudaEvent_t ev_loop[2] = {nullptr, nullptr};   // around the loop graph launch
};

#define SP2_TRY(expr)                              \
  do {                                             \
    if ((expr) != cudaSuccess) {                   \
      (void)cudaGetLastError();                    \
      return SP2_ERR_CUDA;                         \
    }                                              \
  } while (0)

extern "C" void sp2_default_opts(sp2_opts* o) {
  if (!o) return;
  o->max_iter = 200;
  o->guard = 1;
  o->qtilde = 1.8;
}

extern "C" const char* sp2_status_string(int32_t s) {
  switch (s) {
    case SP2_OK: return "ok";
    case SP2_ERR_INVALID_ARG: return "invalid argument";
    case SP2_ERR_CUDA: return "CUDA runtime error";
    case SP2_ERR_NONFINITE: return "non-finite value in F";
    case SP2_ERR_TIMEOUT: return "device-side wait timed out";
    case SP2_ERR_NOMEM: return "out of device memory";
    case SP2_ERR_NO_GAP: return "F has zero spectral width (no gap)";
    case SP2_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

static void free_ctx(sp2_ctx* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  cudaFree(h->part);
  cudaFree(h->part_lo);
  cudaFree(h->part_hi);
  cudaFree(h->part_bad);
  cudaFree(h->st_dev);
  cudaFree(h->stage_F);
  cudaFree(h->stage_D);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->ev_loop[0]) cudaEventDestroy(h->ev_loop[0]);
  if (h->ev_loop[1]) cudaEventDestroy(h->ev_loop[1]);
  (void)cudaGetLastError();
  cudaSetDevice(cur);
  delete h;
}

static sp2_status build_loop_graph(sp2_ctx* h) {
  SP2_TRY(cudaGraphCreate(&h->graph, 0));
  // Default value 1: the body runs at least once per launch; the finalize kernel sets
  // the condition to 0 when the stop test fires (or at once when a run is already done).
  SP2_TRY(cudaGraphConditionalHandleCreate(&h->cond, h->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h->cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  SP2_TRY(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  SP2_TRY(sp2::add_f64_loop_body(body, h->st_dev, h->buf[0], h->buf[1], h->part, h->T, h->cond));
  SP2_TRY(cudaGraphInstantiate(&h->exec, h->graph, 0));
  return SP2_OK;
}

extern "C" sp2_status sp2_create(int64_t N, int64_t nocc, int32_t precision, const sp2_opts* opts,
                                 sp2_handle* out) {
  if (!out) return SP2_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < 1 || N > 65536 || nocc < 0 || nocc > N) return SP2_ERR_INVALID_ARG;
  if (precision != SP2_PREC_FP64) return SP2_ERR_UNSUPPORTED;
  sp2_opts o;
  sp2_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_iter < 1 || o.max_iter > SP2_MAX_ITER || !(o.qtilde > 0.0) || (o.guard != 0 && o.guard != 1))
    return SP2_ERR_INVALID_ARG;

  sp2_ctx* h = new (std::nothrow) sp2_ctx();
  if (!h) return SP2_ERR_NOMEM;
  h->N = N; h->nocc = nocc; h->precision = precision; h->opts = o;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; (void)cudaGetLastError(); return SP2_ERR_CUDA; }
  h->ld = (int)((N + 63) / 64 * 64);
  h->T = h->ld / 64;
  h->nparts = (int)((N + 7) / 8 < 1024 ? (N + 7) / 8 : 1024);
  const size_t bytes = (size_t)h->ld * h->ld * sizeof(double);
  const size_t ntiles = (size_t)h->T * (h->T + 1) / 2;
  bool ok = cudaMalloc(&h->buf[0], bytes) == cudaSuccess && cudaMalloc(&h->buf[1], bytes) == cudaSuccess &&
            cudaMalloc(&h->part, ntiles * 2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_lo, h->nparts * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_hi, h->nparts * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_bad, h->nparts * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->st_dev, sizeof(DevState)) == cudaSuccess &&
            cudaMallocHost(&h->st_host, sizeof(DevState)) == cudaSuccess &&
            cudaEventCreate(&h->ev_loop[0]) == cudaSuccess && cudaEventCreate(&h->ev_loop[1]) == cudaSuccess;
  if (!ok) { (void)cudaGetLastError(); free_ctx(h); return SP2_ERR_NOMEM; }
  // Zero borders of the ping-pong buffers stay zero for the whole life of the handle.
  DevState init;
  std::memset(&init, 0, sizeof(init));
  init.N = (int32_t)N; init.ld = h->ld; init.nocc = (int32_t)nocc;
  init.max_iter = o.max_iter; init.guard = o.guard; init.qtilde = o.qtilde;
  if (cudaMemset(h->buf[0], 0, bytes) != cudaSuccess || cudaMemset(h->buf[1], 0, bytes) != cudaSuccess ||
      cudaMemcpy(h->st_dev, &init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess) {
    (void)cudaGetLastError(); free_ctx(h); return SP2_ERR_CUDA;
  }
  *h->st_host = init;
  sp2_status s = build_loop_graph(h);
  if (s != SP2_OK) { free_ctx(h); return s; }
  if (cudaDeviceSynchronize() != cudaSuccess) { (void)cudaGetLastError(); free_ctx(h); return SP2_ERR_CUDA; }
  *out = h;
  return SP2_OK;
}

static bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + bytes && y < x + bytes;
}

static sp2_status enqueue_run(sp2_ctx* h, const double* F, int64_t ldf, double* D, int64_t ldd,
                              cudaStream_t s) {
  const int N = (int)h->N;
  SP2_TRY(sp2::launch_bounds_and_init(h->st_dev, F, ldf, N, h->part_lo, h->part_hi, h->part_bad,
                                      h->nparts, s));
  SP2_TRY(sp2::launch_scale_f64(h->st_dev, F, ldf, N, h->buf[0], h->ld, s));
  SP2_TRY(cudaEventRecord(h->ev_loop[0], s));
  SP2_TRY(cudaGraphLaunch(h->exec, s));
  SP2_TRY(cudaEventRecord(h->ev_loop[1], s));
  SP2_TRY(sp2::launch_copy_out(h->st_dev, h->buf[0], h->buf[1], h->ld, N, D, ldd, s));
  SP2_TRY(cudaMemcpyAsync(h->st_host, h->st_dev, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  h->last_stream = s;
  h->ran = true;
  return SP2_OK;
}

extern "C" sp2_status sp2_run(sp2_handle h, const double* F_dev, double* D_dev, void* stream) {
  if (!h || !F_dev || !D_dev) return SP2_ERR_INVALID_ARG;
  const size_t bytes = (size_t)h->N * h->N * sizeof(double);
  if (overlaps(F_dev, D_dev, bytes)) return SP2_ERR_INVALID_ARG;
  return enqueue_run(h, F_dev, h->N, D_dev, h->N, (cudaStream_t)stream);
}

extern "C" sp2_status sp2_run_host(sp2_handle h, const double* F_host, double* D_host, void* stream) {
  if (!h || !F_host || !D_host) return SP2_ERR_INVALID_ARG;
  const size_t bytes = (size_t)h->N * h->N * sizeof(double);
  if (overlaps(F_host, D_host, bytes)) return SP2_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!h->stage_F) {
    if (cudaMalloc(&h->stage_F, bytes) != cudaSuccess || cudaMalloc(&h->stage_D, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaFree(h->stage_F); cudaFree(h->stage_D);
      h->stage_F = h->stage_D = nullptr;
      return SP2_ERR_NOMEM;
    }
  }
  SP2_TRY(cudaMemcpyAsync(h->stage_F, F_host, bytes, cudaMemcpyHostToDevice, s));
  sp2_status st = enqueue_run(h, h->stage_F, h->N, h->stage_D, h->N, s);
  if (st != SP2_OK) return st;
  SP2_TRY(cudaMemcpyAsync(D_host, h->stage_D, bytes, cudaMemcpyDeviceToHost, s));
  SP2_TRY(cudaStreamSynchronize(s));
  return SP2_OK;
}

extern "C" sp2_status sp2_get_info(sp2_handle h, sp2_info* out) {
  if (!h || !out) return SP2_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (h->ran) SP2_TRY(cudaStreamSynchronize(h->last_stream));
  const DevState* s = h->st_host;
  out->status = h->ran ? s->status : SP2_OK;
  out->n_iter = s->n_out;
  out->stop_reason = s->reason;
  out->hist_len = s->hist_len;
  out->lambda_min = s->lmin;
  out->lambda_max = s->lmax;
  float ms = 0.f;
  if (h->ran && cudaEventElapsedTime(&ms, h->ev_loop[0], h->ev_loop[1]) == cudaSuccess) out->loop_ms = ms;
  (void)cudaGetLastError();
  out->v = s->v;
  out->trace = s->tr;
  out->p = s->p;
  return SP2_OK;
}

extern "C" void sp2_destroy(sp2_handle h) { free_ctx(h); }
