// C-ABI layer: handles, workspace, and the device-controlled loops as CUDA graphs
// with conditional WHILE nodes, plus the host-buffer entry point.
//
// FP64 run:  bounds + init, scaling, [WHILE: FP64 square + stop test], output copy.
// Mixed run: bounds + init, scaling + piece split, [WHILE: tensor-core square + stop
//            test], correction GEMMs (M = P F, dX_0 from M + M^T - 2 M P),
//            [WHILE: derivative step], D = X_n + dX_n, optional FP64 refinement pair.
// Nothing waits on the host in between; the loop conditions are cleared on the device.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <new>

#include "sp2_common.cuh"
#include "sp2_kernels.h"
#include "sp2_tc.cuh"

using sp2::DevState;

struct sp2_ctx {
  int64_t N = 0, nocc = 0;
  int32_t precision = 0;
  sp2_opts opts{};
  int device = 0;
  int ld = 0, T = 0, nparts = 0;
  // FP64 path (and the mixed path's refinement)
  double* buf[2] = {nullptr, nullptr};
  double* part = nullptr;
  double* part_lo = nullptr;
  double* part_hi = nullptr;
  int* part_bad = nullptr;
  DevState* st_dev = nullptr;
  DevState* st_host = nullptr;   // pinned mirror for sp2_get_info
  int32_t* err_dev = nullptr;    // device-side wait failures
  int32_t* err_host = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0, cond2 = 0;
  cudaStream_t last_stream = nullptr;
  bool ran = false;
  double* stage_F = nullptr;     // device staging for sp2_run_host
  double* stage_D = nullptr;
  cudaEvent_t ev_loop[2] = {nullptr, nullptr};
  // mixed path
  void* arena = nullptr;
  int64_t slot_elems = 0;
  int nslots = 0, hist0 = 0, dx0 = 0, m_slot = 0, f_slot = 0, r0_slot = 0;
  CUtensorMap mapA, mapB;
  double* part_tc = nullptr;
  int tiles_upper = 0;
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
  o->corrections = 1;
  o->refine_steps = 2;
  o->refine_fp64 = 0;
  o->reserved = 0;
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
  cudaFree(h->err_dev);
  cudaFree(h->stage_F);
  cudaFree(h->stage_D);
  cudaFree(h->arena);
  cudaFree(h->part_tc);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->err_host) cudaFreeHost(h->err_host);
  if (h->ev_loop[0]) cudaEventDestroy(h->ev_loop[0]);
  if (h->ev_loop[1]) cudaEventDestroy(h->ev_loop[1]);
  (void)cudaGetLastError();
  cudaSetDevice(cur);
  delete h;
}

static sp2_status add_while(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, cudaGraphConditionalHandle* cond,
                            cudaGraphNode_t* node, cudaGraph_t* body) {
  // Default value 1: the body runs at least once per launch; a kernel in the body
  // clears the condition when its loop is finished (or at once if there is no work).
  SP2_TRY(cudaGraphConditionalHandleCreate(cond, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = *cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  SP2_TRY(cudaGraphAddNode(node, g, deps, nullptr, ndeps, &np));
  *body = np.conditional.phGraph_out[0];
  return SP2_OK;
}

static sp2_status build_graph_f64(sp2_ctx* h) {
  SP2_TRY(cudaGraphCreate(&h->graph, 0));
  cudaGraphNode_t node;
  cudaGraph_t body;
  sp2_status s = add_while(h->graph, nullptr, 0, &h->cond, &node, &body);
  if (s != SP2_OK) return s;
  SP2_TRY(sp2::add_f64_loop_body(body, h->st_dev, h->buf[0], h->buf[1], h->part, h->T, h->cond));
  SP2_TRY(cudaGraphInstantiate(&h->exec, h->graph, 0));
  return SP2_OK;
}

static sp2::tc::Job base_job(const sp2_ctx* h) {
  sp2::tc::Job j;
  std::memset(&j, 0, sizeof(j));
  j.ld = h->ld;
  j.arena = (__nv_bfloat16*)h->arena;
  j.slot_elems = h->slot_elems;
  j.st = h->st_dev;
  j.err = h->err_dev;
  j.hist0 = h->hist0;
  j.dx0 = h->dx0;
  j.m_slot = h->m_slot;
  j.f_slot = h->f_slot;
  j.r0_slot = h->r0_slot;
  j.nterms = 1;
  return j;
}

static sp2_status build_graph_mixed(sp2_ctx* h) {
  using namespace sp2::tc;
  SP2_TRY(cudaGraphCreate(&h->graph, 0));
  cudaGraphNode_t n_fwd, n_sq, n_fin;
  cudaGraph_t body;
  sp2_status s = add_while(h->graph, nullptr, 0, &h->cond, &n_fwd, &body);
  if (s != SP2_OK) return s;
  Job fwd = base_job(h);
  fwd.mode = MODE_SP2_STEP;
  fwd.upper = 1;
  fwd.rule = SLOTS_FORWARD;
  fwd.part = h->part_tc;
  SP2_TRY(sp2::tc_add_node(body, nullptr, 0, h->mapA, h->mapB, fwd, &n_sq));
  SP2_TRY(sp2::add_finalize_node(body, &n_sq, 1, h->st_dev, h->part_tc, 4 * h->tiles_upper, 4, h->cond, &n_fin));
  if (h->opts.corrections > 0) {
    cudaGraphNode_t n_m, n_df, n_der, n_dsq, n_dfin;
    Job jm = base_job(h);
    jm.mode = MODE_STORE_PIECES;
    jm.upper = 0;
    jm.rule = SLOTS_CORR_M;
    SP2_TRY(sp2::tc_add_node(h->graph, &n_fwd, 1, h->mapA, h->mapB, jm, &n_m));
    Job jd = base_job(h);
    jd.mode = MODE_DF_COMBINE;
    jd.upper = 1;
    jd.rule = SLOTS_CORR_DF;
    SP2_TRY(sp2::tc_add_node(h->graph, &n_m, 1, h->mapA, h->mapB, jd, &n_df));
    cudaGraph_t dbody;
    s = add_while(h->graph, &n_df, 1, &h->cond2, &n_der, &dbody);
    if (s != SP2_OK) return s;
    Job jv = base_job(h);
    jv.mode = MODE_DERIV_STEP;
    jv.upper = 1;
    jv.nterms = 2;
    jv.rule = SLOTS_DERIV;
    SP2_TRY(sp2::tc_add_node(dbody, nullptr, 0, h->mapA, h->mapB, jv, &n_dsq));
    SP2_TRY(sp2::add_deriv_finalize_node(dbody, &n_dsq, 1, h->st_dev, h->cond2, &n_dfin));
    n_fwd = n_der;
  }
  if (h->opts.refine_steps > 0 && !h->opts.refine_fp64) {
    cudaGraphNode_t n_piece, n_r0, n_r1;
    SP2_TRY(sp2::add_corrected_to_pieces_node(h->graph, &n_fwd, 1, h->st_dev, h->arena, h->slot_elems, h->ld,
                                              h->hist0, h->dx0, h->opts.corrections > 0, h->r0_slot, (int)h->N,
                                              &n_piece));
    Job jr = base_job(h);
    jr.mode = MODE_DERIV_STEP;   // new = p ? C : 2 in - C with C = in^2: one SP2 step
    jr.upper = 1;
    jr.rule = SLOTS_REFINE;
    jr.a_slot[0] = 0;
    SP2_TRY(sp2::tc_add_node(h->graph, &n_piece, 1, h->mapA, h->mapB, jr, &n_r0));
    jr.a_slot[0] = 1;
    SP2_TRY(sp2::tc_add_node(h->graph, &n_r0, 1, h->mapA, h->mapB, jr, &n_r1));
  }
  SP2_TRY(cudaGraphInstantiate(&h->exec, h->graph, 0));
  return SP2_OK;
}

extern "C" sp2_status sp2_create(int64_t N, int64_t nocc, int32_t precision, const sp2_opts* opts,
                                 sp2_handle* out) {
  if (!out) return SP2_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < 1 || N > 65536 || nocc < 0 || nocc > N) return SP2_ERR_INVALID_ARG;
  if (precision != SP2_PREC_FP64 && precision != SP2_PREC_MIXED) return SP2_ERR_UNSUPPORTED;
  sp2_opts o;
  sp2_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_iter < 1 || o.max_iter > SP2_MAX_ITER || !(o.qtilde > 0.0) || (o.guard != 0 && o.guard != 1) ||
      o.corrections < 0 || o.corrections > 1 || (o.refine_steps != 0 && o.refine_steps != 2) ||
      (o.refine_fp64 != 0 && o.refine_fp64 != 1) || o.reserved != 0)
    return SP2_ERR_INVALID_ARG;

  sp2_ctx* h = new (std::nothrow) sp2_ctx();
  if (!h) return SP2_ERR_NOMEM;
  h->N = N; h->nocc = nocc; h->precision = precision; h->opts = o;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; (void)cudaGetLastError(); return SP2_ERR_CUDA; }
  const bool mixed = precision == SP2_PREC_MIXED;
  const int align = mixed ? sp2::tc::LD_ALIGN : 64;
  h->ld = (int)((N + align - 1) / align * align);
  h->T = h->ld / 64;
  h->nparts = (int)((N + 7) / 8 < 1024 ? (N + 7) / 8 : 1024);
  const size_t bytes = (size_t)h->ld * h->ld * sizeof(double);
  const size_t ntiles = (size_t)h->T * (h->T + 1) / 2;
  const bool need_f64 = !mixed || (o.refine_steps > 0 && o.refine_fp64);
  bool ok = cudaMalloc(&h->part, ntiles * 2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_lo, h->nparts * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_hi, h->nparts * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_bad, h->nparts * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->st_dev, sizeof(DevState)) == cudaSuccess &&
            cudaMalloc(&h->err_dev, sizeof(int32_t)) == cudaSuccess &&
            cudaMallocHost(&h->st_host, sizeof(DevState)) == cudaSuccess &&
            cudaMallocHost(&h->err_host, sizeof(int32_t)) == cudaSuccess &&
            cudaEventCreate(&h->ev_loop[0]) == cudaSuccess && cudaEventCreate(&h->ev_loop[1]) == cudaSuccess;
  if (ok && need_f64)
    ok = cudaMalloc(&h->buf[0], bytes) == cudaSuccess && cudaMalloc(&h->buf[1], bytes) == cudaSuccess;
  if (ok && mixed) {
    h->hist0 = 0;
    const int H = o.max_iter + 2;
    h->dx0 = H;
    h->m_slot = H + 2;
    h->f_slot = H + 3;
    h->r0_slot = H + 4;
    h->nslots = H + 6;
    h->slot_elems = (int64_t)sp2::tc::NP * h->ld * h->ld;
    h->tiles_upper = sp2::tc_tiles(h->ld, 1);
    ok = cudaMalloc(&h->arena, (size_t)h->nslots * h->slot_elems * 2) == cudaSuccess &&
         cudaMalloc(&h->part_tc, (size_t)h->tiles_upper * 16 * sizeof(double)) == cudaSuccess;
  }
  if (!ok) { (void)cudaGetLastError(); free_ctx(h); return SP2_ERR_NOMEM; }
  // Zero borders stay zero for the whole life of the handle (every step maps 0 to 0).
  DevState init;
  std::memset(&init, 0, sizeof(init));
  init.N = (int32_t)N; init.ld = h->ld; init.nocc = (int32_t)nocc;
  init.max_iter = o.max_iter; init.guard = o.guard; init.qtilde = o.qtilde;
  init.round_fp32 = mixed ? 1 : 0;
  bool okz = cudaMemcpy(h->st_dev, &init, sizeof(init), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(h->err_dev, 0, sizeof(int32_t)) == cudaSuccess;
  if (okz && need_f64)
    okz = cudaMemset(h->buf[0], 0, bytes) == cudaSuccess && cudaMemset(h->buf[1], 0, bytes) == cudaSuccess;
  if (okz && mixed) okz = cudaMemset(h->arena, 0, (size_t)h->nslots * h->slot_elems * 2) == cudaSuccess;
  if (!okz) { (void)cudaGetLastError(); free_ctx(h); return SP2_ERR_CUDA; }
  *h->st_host = init;
  *h->err_host = 0;
  sp2_status s = SP2_OK;
  if (mixed) {
    if (sp2::tc_make_maps(h->arena, h->ld, h->nslots, &h->mapA, &h->mapB) != cudaSuccess) {
      (void)cudaGetLastError(); free_ctx(h); return SP2_ERR_CUDA;
    }
    s = build_graph_mixed(h);
  } else {
    s = build_graph_f64(h);
  }
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
  SP2_TRY(cudaMemsetAsync(h->err_dev, 0, sizeof(int32_t), s));
  SP2_TRY(sp2::launch_bounds_and_init(h->st_dev, F, ldf, N, h->part_lo, h->part_hi, h->part_bad,
                                      h->nparts, s));
  if (h->precision == SP2_PREC_MIXED) {
    SP2_TRY(sp2::launch_scale_split(h->st_dev, F, ldf, N, h->arena, h->slot_elems, h->ld, h->hist0, h->f_slot, s));
  } else {
    SP2_TRY(sp2::launch_scale_f64(h->st_dev, F, ldf, N, h->buf[0], h->ld, s));
  }
  SP2_TRY(cudaEventRecord(h->ev_loop[0], s));
  SP2_TRY(cudaGraphLaunch(h->exec, s));
  SP2_TRY(cudaEventRecord(h->ev_loop[1], s));
  if (h->precision == SP2_PREC_MIXED) {
    const int use_dx = h->opts.corrections > 0;
    if (h->opts.refine_steps > 0 && h->opts.refine_fp64) {
      SP2_TRY(sp2::launch_assemble(h->st_dev, h->arena, h->slot_elems, h->ld, h->hist0, h->dx0, use_dx, h->r0_slot,
                                   0, N, h->buf[0], h->ld, s));
      SP2_TRY(sp2::launch_refine_f64(h->st_dev, h->buf[0], h->buf[1], h->ld, 0, h->part, s));
      SP2_TRY(sp2::launch_refine_f64(h->st_dev, h->buf[1], h->buf[0], h->ld, 1, h->part, s));
      SP2_TRY(sp2::launch_copy_f64(h->st_dev, h->buf[0], h->ld, N, D, ldd, s));
    } else {
      const int from_r0 = h->opts.refine_steps > 0 ? 1 : 0;
      SP2_TRY(sp2::launch_assemble(h->st_dev, h->arena, h->slot_elems, h->ld, h->hist0, h->dx0, use_dx, h->r0_slot,
                                   from_r0, N, D, ldd, s));
    }
  } else {
    SP2_TRY(sp2::launch_copy_out(h->st_dev, h->buf[0], h->buf[1], h->ld, N, D, ldd, s));
  }
  SP2_TRY(cudaMemcpyAsync(h->st_host, h->st_dev, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  SP2_TRY(cudaMemcpyAsync(h->err_host, h->err_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
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
  if (h->ran && out->status == SP2_OK && *h->err_host != 0) out->status = *h->err_host;
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
