// C-ABI layer: handles, workspace, and the device-controlled loops as CUDA graphs
// with conditional WHILE nodes, plus the host-buffer and batch entry points.
//
// FP64 run:  bounds + init, scaling, [WHILE: FP64 square + stop test], output copy.
// Mixed run (a batch of one or more problems):
//   batched bounds + init + scaling/piece split,
//   [WHILE: one tensor-core launch squaring every live problem, per-problem stop test],
//   correction GEMMs (M = P F, dX_0 from M + M^T - 2 M P),
//   [WHILE: one derivative step for every problem short of its n],
//   refinement pair on the corrected D, output.
// Nothing waits on the host in between; the loop conditions are cleared on the device.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sp2_common.cuh"
#include "sp2_kernels.h"
#include "sp2_tc.cuh"

using sp2::DevState;
using sp2::tc::Instance;

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
  o->launch_mode = 0;
  o->history = 0;
  o->tile = 0;
  o->norm = 0;
  o->bsr_cuda_cores = 0;
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
    case SP2_ERR_BOUNDS: return "device-side bounds check failed (debug library)";
    default: return "unknown status";
  }
}

// Host-side NVTX range over an entry point (the enqueue, or the whole call for the synchronous
// host-buffer entry); a no-op unless a profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static bool opts_valid(const sp2_opts& o) {
  return o.max_iter >= 1 && o.max_iter <= SP2_MAX_ITER && o.qtilde > 0.0 && (o.guard == 0 || o.guard == 1) &&
         o.corrections >= 0 && o.corrections <= 1 && (o.refine_steps == 0 || o.refine_steps == 2) &&
         (o.refine_fp64 >= 0 && o.refine_fp64 <= 2) && (o.launch_mode == 0 || o.launch_mode == 1) &&
         o.history >= 0 && o.history <= 2 && o.tile >= 0 && o.tile <= 2 &&
         o.norm >= 0 && o.norm <= 2;
}

static DevState initial_state(int64_t N, int64_t nocc, const sp2_opts& o, int ld, int round_fp32) {
  DevState init;
  std::memset(&init, 0, sizeof(init));
  init.N = (int32_t)N; init.ld = ld; init.nocc = (int32_t)nocc;
  init.max_iter = o.max_iter; init.guard = o.guard; init.qtilde = o.qtilde;
  init.round_fp32 = round_fp32;
  init.norm = o.norm;
  return init;
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

// ---------------------------------------------------------------------------------------------
// Tile tuner for the mixed path: 1 = 128 x 128 tiles (ld a multiple of 128), 2 = 256 x 256
// CTA-pair tiles (ld a multiple of 256).  Each candidate runs the same product a forward
// square runs (every problem's upper tiles, pieces out, mirror written) on zeroed scratch
// shaped like the handle's problems, one launch untimed and three timed; the faster one is
// kept.  When the scratch would exceed kTuneBytes, a model of the kernels' measured
// algorithmic rates at large sizes (1200 and 1580 TFLOP/s) decides instead.
static constexpr size_t kTuneBytes = size_t(2) << 30;

static int round_up(int64_t n, int a) { return (int)((n + a - 1) / a * a); }

static int tune_tiles(const std::vector<int64_t>& N, int fmt, int lowprec) {
  using namespace sp2::tc;
  const int count = (int)N.size();
  const int np = np_of(fmt);
  double model[3] = {0.0, 0.0, 0.0};
  size_t bytes[3] = {0, 0, 0};
  for (int c = 1; c <= 2; ++c)
    for (int k = 0; k < count; ++k) {
      const double ld = round_up(N[k], c == 2 ? PT : LD_ALIGN);
      model[c] += ld * ld * ld / (c == 2 ? 1580.0 : 1200.0);
      bytes[c] += (size_t)2 * np * (size_t)ld * (size_t)ld * esize_of(fmt);
    }
  const int by_model = model[2] < model[1] ? 2 : 1;
  if (std::max(bytes[1], bytes[2]) > kTuneBytes) return by_model;

  float best[3] = {0.f, 0.f, 0.f};
  cudaStream_t s = nullptr;
  void* scratch = nullptr;
  Instance* dinst = nullptr;
  int32_t* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&scratch, std::max(bytes[1], bytes[2])) == cudaSuccess &&
            cudaMalloc(&dinst, sizeof(Instance) * count) == cudaSuccess &&
            cudaMalloc(&err, sizeof(int32_t)) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
            cudaEventCreate(&e1) == cudaSuccess &&
            cudaMemsetAsync(scratch, 0, std::max(bytes[1], bytes[2]), s) == cudaSuccess &&
            cudaMemsetAsync(err, 0, sizeof(int32_t), s) == cudaSuccess;
  std::vector<Instance> hinst(count);
  for (int c = 1; c <= 2 && ok; ++c) {
    const int pair = c == 2;
    size_t off = 0;
    int tiles = 0;
    for (int k = 0; k < count && ok; ++k) {
      Instance& I = hinst[k];
      std::memset(&I, 0, sizeof(I));
      const int ld = round_up(N[k], pair ? PT : LD_ALIGN);
      __nv_bfloat16* arena = (__nv_bfloat16*)((char*)scratch + off);
      off += (size_t)2 * np * (size_t)ld * (size_t)ld * esize_of(fmt);
      I.ld = ld;
      I.arena = arena;
      I.fmt = fmt;
      I.np = np;
      I.nslots = 2;
      I.slot_elems = sp2::tc::slot_units_of(fmt, ld);
      I.tile_off_upper = I.tile_off_upper2 = tiles;
      tiles += sp2::tc_tiles(ld, 1, pair);
      ok = sp2::tc_make_maps(arena, ld, 2, fmt, &I.mapA, &I.mapB) == cudaSuccess;
    }
    if (!ok) break;
    Job j;
    std::memset(&j, 0, sizeof(j));
    j.mode = MODE_STORE_PIECES;
    j.upper = 1;
    j.nterms = 1;
    j.rule = SLOTS_FIXED;
    j.count = count;
    j.total_tiles = tiles;
    j.inst = dinst;
    j.out_slot = 1;
    j.pair = pair;
    j.fmt = fmt;
    j.lowprec = lowprec;
    j.err = err;
    ok = cudaMemcpyAsync(dinst, hinst.data(), sizeof(Instance) * count, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         sp2::tc_launch(j, s) == cudaSuccess;
    float t = 1e30f;
    for (int r = 0; r < 3 && ok; ++r) {
      float ms = 0.f;
      ok = cudaEventRecord(e0, s) == cudaSuccess && sp2::tc_launch(j, s) == cudaSuccess &&
           cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      t = std::min(t, ms);
    }
    best[c] = t;
  }
  int32_t herr = 0;
  if (ok) ok = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
               cudaStreamSynchronize(s) == cudaSuccess && herr == 0;
  if (s) cudaStreamSynchronize(s);
  cudaFree(scratch);
  cudaFree(dinst);
  cudaFree(err);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  (void)cudaGetLastError();
  if (!ok) return by_model;
  return best[2] < best[1] ? 2 : 1;
}

// Mixed-precision engine: `count` problems, stored largest first (internal order).
// ---------------------------------------------------------------------------------------------
struct MixedEngine {
  int count = 0;
  sp2_opts opts{};
  int fmt = 0;                     // tc::Fmt of every arena
  int lp_main = 0;                 // 1: forward, correction and refinement products at low precision
                                   // (SP2_PREC_BF16X3); the derivative pass always is
  std::vector<int> user_of;        // internal index -> user index
  std::vector<int> internal_of;    // user index -> internal index
  std::vector<int64_t> N, nocc;    // internal order
  std::vector<Instance> inst_host;
  Instance* inst_dev = nullptr;
  DevState* st_dev = nullptr;
  DevState* st_host = nullptr;     // pinned mirror
  std::vector<void*> arenas;
  std::vector<double*> parts;
  std::vector<double*> mscrs;      // mixed-norm scratch per problem (norm = 1)
  void* lz = nullptr;              // Lanczos scratch of the spectral-norm stop (norm = 2, one problem)
  double* part_lo = nullptr;
  double* part_hi = nullptr;
  int* part_bad = nullptr;
  int pb = 1, sb = 1;
  int pair = 0;                    // tensor-core tiles: 1 = 256 x 256 per SM pair, 0 = 128 x 128 per SM
  int total_upper = 0, total_full = 0;   // tiles of one launch, in the unit above
  int32_t* err_dev = nullptr;
  int32_t* err_host = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0, cond2 = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double* fbuf[2] = {nullptr, nullptr};   // FP64 refinement (single problem only)
  double* fpart = nullptr;
  int fld = 0;

  ~MixedEngine() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFree(inst_dev);
    cudaFree(st_dev);
    for (void* a : arenas) cudaFree(a);
    for (double* p : parts) cudaFree(p);
    for (double* p : mscrs) cudaFree(p);
    cudaFree(lz);
    cudaFree(part_lo);
    cudaFree(part_hi);
    cudaFree(part_bad);
    cudaFree(err_dev);
    cudaFree(fbuf[0]);
    cudaFree(fbuf[1]);
    cudaFree(fpart);
    if (st_host) cudaFreeHost(st_host);
    if (err_host) cudaFreeHost(err_host);
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    (void)cudaGetLastError();
  }

  sp2::tc::Job job(int mode, int upper, int rule, int nterms = 1) const {
    sp2::tc::Job j;
    std::memset(&j, 0, sizeof(j));
    j.mode = mode;
    j.upper = upper;
    j.nterms = nterms;
    j.rule = rule;
    j.count = count;
    j.pair = pair;
    j.total_tiles = upper ? total_upper : total_full;
    j.inst = inst_dev;
    j.err = err_dev;
    j.fmt = fmt;
    j.lowprec = lp_main;
    return j;
  }

  // One derivative step: dX_j from X_{j-1} and dX_{j-1} (two products).  dX is a
  // first-order correction far smaller than X, so its products run at the format's low
  // precision: the two leading bf16 pieces (about 16 bits, half the work of a full product)
  // or the leading fp16 piece (11 bits, a third).
  sp2::tc::Job deriv_job() const {
    sp2::tc::Job j = job(sp2::tc::MODE_DERIV_STEP, 1, sp2::tc::SLOTS_DERIV, 2);
    j.lowprec = 1;
    j.whole_k = 1;
    return j;
  }

  sp2_status init(int cnt, const int64_t* Nu, const int64_t* noccu, const sp2_opts& o, int precision) {
    using namespace sp2::tc;
    count = cnt;
    opts = o;
    fmt = precision == SP2_PREC_FP16X3 ? FMT_FP16X2 : (precision == SP2_PREC_TF32X3 ? FMT_TF32X2 : FMT_BF16X3);
    lp_main = precision == SP2_PREC_BF16X3 ? 1 : 0;
    const int np = np_of(fmt);
    user_of.resize(count);
    std::iota(user_of.begin(), user_of.end(), 0);
    std::stable_sort(user_of.begin(), user_of.end(), [&](int a, int b) { return Nu[a] > Nu[b]; });
    internal_of.resize(count);
    for (int k = 0; k < count; ++k) internal_of[user_of[k]] = k;
    N.resize(count);
    nocc.resize(count);
    int64_t maxN = 1;
    for (int k = 0; k < count; ++k) {
      N[k] = Nu[user_of[k]];
      nocc[k] = noccu[user_of[k]];
      maxN = std::max(maxN, N[k]);
    }
    pb = (int)std::max<int64_t>(1, std::min<int64_t>((maxN + 7) / 8, std::max(4, 2048 / count)));
    sb = (int)std::max<int64_t>(1, std::min<int64_t>((maxN * maxN + 255) / 256, std::max(4, 2432 / count)));
    if (cudaMalloc(&inst_dev, sizeof(Instance) * count) != cudaSuccess ||
        cudaMalloc(&st_dev, sizeof(DevState) * count) != cudaSuccess ||
        cudaMallocHost(&st_host, sizeof(DevState) * count) != cudaSuccess ||
        cudaMalloc(&part_lo, sizeof(double) * count * pb) != cudaSuccess ||
        cudaMalloc(&part_hi, sizeof(double) * count * pb) != cudaSuccess ||
        cudaMalloc(&part_bad, sizeof(int) * count * pb) != cudaSuccess ||
        cudaMalloc(&err_dev, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&err_host, sizeof(int32_t)) != cudaSuccess || cudaEventCreate(&ev[0]) != cudaSuccess ||
        cudaEventCreate(&ev[1]) != cudaSuccess) {
      (void)cudaGetLastError();
      return SP2_ERR_NOMEM;
    }
    inst_host.resize(count);
    arenas.assign(count, nullptr);
    parts.assign(count, nullptr);
    const int H = o.max_iter + 2;
    pair = (o.tile == 0 ? tune_tiles(N, fmt, lp_main) : o.tile) == 2 ? 1 : 0;
    const int align = pair ? PT : LD_ALIGN;
    auto ld_of = [&](int64_t n) { return round_up(n, align); };
    // Keep every iterate (full history) or recompute them in the derivative pass; without
    // the correction no pass reads the history, so the rings suffice.
    int lowmem = (o.history == 2 || o.corrections == 0) ? 1 : 0;
    if (o.history == 0 && o.corrections > 0) {
      double full = 0.0;
      for (int k = 0; k < count; ++k) {
        const double ld = (double)ld_of(N[k]);
        full += (double)(H + 6) * np * ld * ld * esize_of(fmt);
      }
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { (void)cudaGetLastError(); free_b = 0; }
      lowmem = full > 0.6 * (double)free_b ? 1 : 0;
    }
    int off_u = 0, off_f = 0;
    for (int k = 0; k < count; ++k) {
      Instance& I = inst_host[k];
      std::memset(&I, 0, sizeof(I));
      const int ld = ld_of(N[k]);
      I.ld = ld;
      I.hist0 = 0;
      I.lowmem = lowmem;
      // full history: X_0..X_{H-1}, dX x2, M, F, refinement x2; low memory: X_0, two
      // forward slots, two recompute slots, then the same five
      const int base = lowmem ? 5 : H;
      I.dx0 = base;
      I.m_slot = base + 2;
      I.f_slot = base + 3;
      I.r0_slot = base + 4;
      const int nslots = base + 6;
      I.nslots = nslots;
      I.fmt = fmt;
      I.np = np;
      I.slot_elems = sp2::tc::slot_units_of(fmt, ld);
      I.st = st_dev + k;
      I.tile_off_upper = I.tile_off_upper2 = off_u;
      I.tile_off_full = I.tile_off_full2 = off_f;
      off_u += pair ? pair_tiles_of(ld, 1) : tiles_of(ld, 1);
      off_f += pair ? pair_tiles_of(ld, 0) : tiles_of(ld, 0);
      I.nparts = nparts_of(ld, pair);
      I.rec_pair = pair;
      const size_t abytes = (size_t)nslots * I.slot_elems * 2;
      if (cudaMalloc(&arenas[k], abytes) != cudaSuccess ||
          cudaMalloc(&parts[k], sizeof(double) * 4 * I.nparts) != cudaSuccess) {
        (void)cudaGetLastError();
        return SP2_ERR_NOMEM;
      }
      // zero borders stay zero for the life of the handle (every step maps 0 to 0)
      SP2_TRY(cudaMemset(arenas[k], 0, abytes));
      I.arena = (__nv_bfloat16*)arenas[k];
      I.part = parts[k];
      if (o.norm == 1) {
        const int nb = ld / BM;
        double* ms = nullptr;
        if (cudaMalloc(&ms, sizeof(double) * ((size_t)nb * nb + 2 * nb)) != cudaSuccess) {
          (void)cudaGetLastError();
          return SP2_ERR_NOMEM;
        }
        mscrs.push_back(ms);
        I.mscr = ms;
      }
      SP2_TRY(sp2::tc_make_maps(arenas[k], ld, nslots, fmt, &I.mapA, &I.mapB));
      if (o.norm == 2) {   // spectral-norm stop: single problems only (one Lanczos scratch)
        if (count != 1) return SP2_ERR_UNSUPPORTED;
        if (cudaMalloc(&lz, sp2::lanczos_scratch_bytes(ld)) != cudaSuccess) {
          (void)cudaGetLastError();
          return SP2_ERR_NOMEM;
        }
      }
      st_host[k] = initial_state(N[k], nocc[k], o, ld, 1);
    }
    total_upper = off_u;
    total_full = off_f;
    SP2_TRY(cudaMemcpy(inst_dev, inst_host.data(), sizeof(Instance) * count, cudaMemcpyHostToDevice));
    SP2_TRY(cudaMemcpy(st_dev, st_host, sizeof(DevState) * count, cudaMemcpyHostToDevice));
    SP2_TRY(cudaMemset(err_dev, 0, sizeof(int32_t)));
    *err_host = 0;
    if (o.refine_steps > 0 && o.refine_fp64) {
      if (count != 1) return SP2_ERR_UNSUPPORTED;
      fld = inst_host[0].ld;   // the FP64 buffers share the tensor-core layout's ld (a multiple of 64)
      const size_t fb = (size_t)fld * fld * sizeof(double);
      const int T = fld / 64;
      if (cudaMalloc(&fbuf[0], fb) != cudaSuccess || cudaMalloc(&fbuf[1], fb) != cudaSuccess ||
          cudaMalloc(&fpart, sizeof(double) * T * (T + 1)) != cudaSuccess) {
        (void)cudaGetLastError();
        return SP2_ERR_NOMEM;
      }
      SP2_TRY(cudaMemset(fbuf[0], 0, fb));
      SP2_TRY(cudaMemset(fbuf[1], 0, fb));
    }
    return build_graph();
  }

  sp2_status build_graph() {
    using namespace sp2::tc;
    SP2_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphNode_t n_fwd, n_sq, last;
    cudaGraph_t body;
    sp2_status s = add_while(graph, nullptr, 0, &cond, &n_fwd, &body);
    if (s != SP2_OK) return s;
    SP2_TRY(sp2::tc_add_node(body, nullptr, 0, job(MODE_SP2_STEP, 1, SLOTS_FORWARD), &n_sq));
    if (lz) {   // e_{k-1} (Lanczos) between the square and the stop test
      cudaGraphNode_t n_lz;
      SP2_TRY(sp2::add_lanczos_tc_nodes(body, n_sq, st_dev, inst_dev, parts[0], inst_host[0].nparts, lz, (int)N[0],
                                        inst_host[0].ld, &n_lz));
      n_sq = n_lz;
    }
    SP2_TRY(sp2::batch_add_forward_tail(body, &n_sq, inst_dev, count, cond));
    last = n_fwd;
    if (opts.corrections > 0) {
      cudaGraphNode_t n_m, n_df, n_der, n_dsq;
      SP2_TRY(sp2::tc_add_node(graph, &last, 1, job(MODE_STORE_PIECES, 0, SLOTS_CORR_M), &n_m));
      SP2_TRY(sp2::tc_add_node(graph, &n_m, 1, job(MODE_DF_COMBINE, 1, SLOTS_CORR_DF), &n_df));
      cudaGraph_t dbody;
      s = add_while(graph, &n_df, 1, &cond2, &n_der, &dbody);
      if (s != SP2_OK) return s;
      SP2_TRY(sp2::tc_add_node(dbody, nullptr, 0, deriv_job(), &n_dsq));
      cudaGraphNode_t n_tail = n_dsq;
      if (inst_host[0].lowmem) {   // low memory: X_j again, next to its derivative step
        SP2_TRY(sp2::tc_add_node(dbody, &n_dsq, 1, job(MODE_DERIV_STEP, 1, SLOTS_RECOMPUTE), &n_tail));
      }
      SP2_TRY(sp2::batch_add_deriv_tail(dbody, &n_tail, inst_dev, count, cond2));
      last = n_der;
    }
    if (opts.refine_steps > 0 && !opts.refine_fp64) {
      cudaGraphNode_t n_piece, n_r0, n_r1;
      SP2_TRY(sp2::batch_add_corrected_to_pieces(graph, &last, inst_dev, count, sb, opts.corrections > 0,
                                                 &n_piece));
      // one SP2 step each: new = p ? C : 2 in - C with C = in^2
      Job jr = job(MODE_DERIV_STEP, 1, SLOTS_REFINE);
      jr.a_slot[0] = 0;
      SP2_TRY(sp2::tc_add_node(graph, &n_piece, 1, jr, &n_r0));
      jr.a_slot[0] = 1;
      SP2_TRY(sp2::tc_add_node(graph, &n_r0, 1, jr, &n_r1));
    }
    SP2_TRY(cudaGraphInstantiate(&exec, graph, 0));
    return SP2_OK;
  }

  // The graph's loops as plain stream launches (launch_mode 1): every launch after the
  // device-side stop returns at once, so the work and the results are the same.
  sp2_status enqueue_loops_plain(cudaStream_t s) {
    using namespace sp2::tc;
    for (int it = 0; it <= opts.max_iter; ++it) {
      SP2_TRY(sp2::tc_launch(job(MODE_SP2_STEP, 1, SLOTS_FORWARD), s));
      if (lz)
        SP2_TRY(sp2::launch_lanczos_tc(st_dev, inst_dev, parts[0], inst_host[0].nparts, lz, (int)N[0],
                                       inst_host[0].ld, s));
      SP2_TRY(sp2::batch_launch_forward_tail(inst_dev, count, s));
    }
    if (opts.corrections > 0) {
      SP2_TRY(sp2::tc_launch(job(MODE_STORE_PIECES, 0, SLOTS_CORR_M), s));
      SP2_TRY(sp2::tc_launch(job(MODE_DF_COMBINE, 1, SLOTS_CORR_DF), s));
      for (int it = 0; it <= opts.max_iter + 1; ++it) {
        SP2_TRY(sp2::tc_launch(deriv_job(), s));
        if (inst_host[0].lowmem) SP2_TRY(sp2::tc_launch(job(MODE_DERIV_STEP, 1, SLOTS_RECOMPUTE), s));
        SP2_TRY(sp2::batch_launch_deriv_tail(inst_dev, count, s));
      }
    }
    if (opts.refine_steps > 0 && !opts.refine_fp64) {
      SP2_TRY(sp2::batch_launch_corrected_to_pieces(inst_dev, count, sb, opts.corrections > 0, s));
      Job jr = job(MODE_DERIV_STEP, 1, SLOTS_REFINE);
      jr.a_slot[0] = 0;
      SP2_TRY(sp2::tc_launch(jr, s));
      jr.a_slot[0] = 1;
      SP2_TRY(sp2::tc_launch(jr, s));
    }
    return SP2_OK;
  }

  // F/D in user order.
  sp2_status enqueue(const double* const* F, double* const* D, cudaStream_t s) {
    sp2::BatchPtrs ptrs;
    std::memset(&ptrs, 0, sizeof(ptrs));
    for (int k = 0; k < count; ++k) {
      ptrs.F[k] = F[user_of[k]];
      ptrs.D[k] = D[user_of[k]];
    }
    SP2_TRY(cudaMemsetAsync(err_dev, 0, sizeof(int32_t), s));
    SP2_TRY(sp2::batch_launch_prologue(inst_dev, count, pb, sb, ptrs, part_lo, part_hi, part_bad, s));
    SP2_TRY(cudaEventRecord(ev[0], s));
    if (opts.launch_mode == 0) {
      SP2_TRY(cudaGraphLaunch(exec, s));
    } else {
      sp2_status st = enqueue_loops_plain(s);
      if (st != SP2_OK) return st;
    }
    SP2_TRY(cudaEventRecord(ev[1], s));
    const int use_dx = opts.corrections > 0;
    if (opts.refine_steps > 0 && opts.refine_fp64 == 2) {
      // one McWeeny step: FP64 square, E = D^2 - D, D E on the tensor cores, D + E - 2 D E
      SP2_TRY(sp2::batch_launch_assemble(inst_dev, count, sb, use_dx, 0, ptrs, fbuf[0], s));
      SP2_TRY(sp2::launch_refine_f64(st_dev, fbuf[0], fbuf[1], fld, 2, fpart, s));
      SP2_TRY(sp2::launch_mcw_split(inst_dev, fbuf[0], fbuf[1], sb, s));
      sp2::tc::Job jm = job(sp2::tc::MODE_STORE_PIECES, 1, sp2::tc::SLOTS_FIXED);
      jm.a_slot[0] = inst_host[0].r0_slot;
      jm.b_slot[0] = inst_host[0].r0_slot + 1;
      jm.out_slot = inst_host[0].m_slot;
      SP2_TRY(sp2::tc_launch(jm, s));
      SP2_TRY(sp2::launch_mcw_out(inst_dev, fbuf[0], fbuf[1], ptrs, sb, s));
    } else if (opts.refine_steps > 0 && opts.refine_fp64) {
      SP2_TRY(sp2::batch_launch_assemble(inst_dev, count, sb, use_dx, 0, ptrs, fbuf[0], s));
      SP2_TRY(sp2::launch_refine_f64(st_dev, fbuf[0], fbuf[1], fld, 0, fpart, s));
      SP2_TRY(sp2::launch_refine_f64(st_dev, fbuf[1], fbuf[0], fld, 1, fpart, s));
      SP2_TRY(sp2::launch_copy_f64(st_dev, fbuf[0], fld, (int)N[0], ptrs.D[0], N[0], s));
    } else {
      SP2_TRY(sp2::batch_launch_assemble(inst_dev, count, sb, use_dx, opts.refine_steps > 0 ? 1 : 0, ptrs,
                                         nullptr, s));
    }
    SP2_TRY(cudaMemcpyAsync(st_host, st_dev, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
    SP2_TRY(cudaMemcpyAsync(err_host, err_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    return SP2_OK;
  }

  void info(int user_index, bool ran, sp2_info* out) const {
    const DevState* st = st_host + internal_of[user_index];
    out->status = ran ? st->status : SP2_OK;
    if (ran && out->status == SP2_OK && *err_host != 0) out->status = *err_host;
    out->n_iter = st->n_out;
    out->stop_reason = st->reason;
    out->hist_len = st->hist_len;
    out->lambda_min = st->lmin;
    out->lambda_max = st->lmax;
    float ms = 0.f;
    if (ran && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) out->loop_ms = ms;
    (void)cudaGetLastError();
    out->v = st->v;
    out->trace = st->tr;
    out->p = st->p;
    out->tile = pair ? 2 : 1;
  }
};

// ---------------------------------------------------------------------------------------------
// Single-problem handle
// ---------------------------------------------------------------------------------------------
struct sp2_ctx {
  int64_t N = 0, nocc = 0;
  int32_t precision = 0;
  sp2_opts opts{};
  int device = 0;
  cudaStream_t last_stream = nullptr;
  bool ran = false;
  double* stage_F = nullptr;     // device staging for sp2_run_host
  double* stage_D = nullptr;
  // FP64 path
  int ld = 0, T = 0, nparts = 0;
  double* buf[2] = {nullptr, nullptr};
  double* part = nullptr;
  double* part_lo = nullptr;
  double* part_hi = nullptr;
  int* part_bad = nullptr;
  double* mscr = nullptr;        // mixed-norm scratch (norm = 1): T^2 + 2T doubles
  void* lz = nullptr;            // Lanczos scratch (norm = 2): lanczos_scratch_bytes(ld)
  const double* pert = nullptr;  // prescribed perturbations E_0.. (caller-owned, testing hook)
  int64_t pert_count = 0;
  int mcw = 0;                   // 0: SP2, 1: McWeeny, 2: McW-ACC (FP64 path)
  double* sbuf = nullptr;        // McWeeny: the shifted square S_s (ld x ld)
  DevState* st_dev = nullptr;
  DevState* st_host = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaEvent_t ev_loop[2] = {nullptr, nullptr};
  // mixed path
  MixedEngine* mixed = nullptr;
};

static void free_ctx(sp2_ctx* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  delete h->mixed;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  cudaFree(h->part);
  cudaFree(h->mscr);
  cudaFree(h->lz);
  cudaFree(h->sbuf);
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

// The FP64 path's loop graph: a WHILE node around {square, stop test} (SP2) or {shifted
// square, stop test, product} (McWeeny).
static sp2_status build_f64_graph(sp2_ctx* h) {
  if (h->exec) { cudaGraphExecDestroy(h->exec); h->exec = nullptr; }
  if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
  SP2_TRY(cudaGraphCreate(&h->graph, 0));
  cudaGraphNode_t node;
  cudaGraph_t body;
  sp2_status s = add_while(h->graph, nullptr, 0, &h->cond, &node, &body);
  if (s != SP2_OK) return s;
  if (h->mcw)
    SP2_TRY(sp2::add_mcw_loop_body(body, h->st_dev, h->buf[0], h->buf[1], h->sbuf, h->part, h->T, h->cond,
                                   h->mscr, h->lz, (int)h->N));
  else
    SP2_TRY(sp2::add_f64_loop_body(body, h->st_dev, h->buf[0], h->buf[1], h->part, h->T, h->cond, h->mscr, h->lz,
                                   (int)h->N, h->pert, h->pert_count));
  SP2_TRY(cudaGraphInstantiate(&h->exec, h->graph, 0));
  return SP2_OK;
}

static sp2_status create_f64(sp2_ctx* h) {
  h->ld = (int)((h->N + 63) / 64 * 64);
  h->T = h->ld / 64;
  h->nparts = (int)((h->N + 7) / 8 < 1024 ? (h->N + 7) / 8 : 1024);
  const size_t bytes = (size_t)h->ld * h->ld * sizeof(double);
  const size_t ntiles = (size_t)h->T * (h->T + 1) / 2;
  bool ok = cudaMalloc(&h->part, ntiles * 2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_lo, h->nparts * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_hi, h->nparts * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->part_bad, h->nparts * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->st_dev, sizeof(DevState)) == cudaSuccess &&
            cudaMallocHost(&h->st_host, sizeof(DevState)) == cudaSuccess &&
            cudaEventCreate(&h->ev_loop[0]) == cudaSuccess && cudaEventCreate(&h->ev_loop[1]) == cudaSuccess &&
            cudaMalloc(&h->buf[0], bytes) == cudaSuccess && cudaMalloc(&h->buf[1], bytes) == cudaSuccess;
  if (ok && h->opts.norm == 1)
    ok = cudaMalloc(&h->mscr, sizeof(double) * ((size_t)h->T * h->T + 2 * h->T)) == cudaSuccess;
  if (ok && h->opts.norm == 2) ok = cudaMalloc(&h->lz, sp2::lanczos_scratch_bytes(h->ld)) == cudaSuccess;
  if (!ok) { (void)cudaGetLastError(); return SP2_ERR_NOMEM; }
  DevState init = initial_state(h->N, h->nocc, h->opts, h->ld, 0);
  SP2_TRY(cudaMemcpy(h->st_dev, &init, sizeof(init), cudaMemcpyHostToDevice));
  SP2_TRY(cudaMemset(h->buf[0], 0, bytes));
  SP2_TRY(cudaMemset(h->buf[1], 0, bytes));
  *h->st_host = init;
  return build_f64_graph(h);
}

extern "C" sp2_status sp2_create(int64_t N, int64_t nocc, int32_t precision, const sp2_opts* opts,
                                 sp2_handle* out) {
  if (!out) return SP2_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < 1 || N > 65536 || nocc < 0 || nocc > N) return SP2_ERR_INVALID_ARG;
  if (precision < SP2_PREC_FP64 || precision > SP2_PREC_TF32X3) return SP2_ERR_UNSUPPORTED;
  sp2_opts o;
  sp2_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_valid(o)) return SP2_ERR_INVALID_ARG;
  sp2_ctx* h = new (std::nothrow) sp2_ctx();
  if (!h) return SP2_ERR_NOMEM;
  h->N = N; h->nocc = nocc; h->precision = precision; h->opts = o;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; (void)cudaGetLastError(); return SP2_ERR_CUDA; }
  sp2_status s;
  if (precision != SP2_PREC_FP64) {
    h->mixed = new (std::nothrow) MixedEngine();
    s = h->mixed ? h->mixed->init(1, &N, &nocc, o, precision) : SP2_ERR_NOMEM;
  } else {
    s = create_f64(h);
  }
  if (s == SP2_OK && cudaDeviceSynchronize() != cudaSuccess) { (void)cudaGetLastError(); s = SP2_ERR_CUDA; }
  if (s != SP2_OK) { free_ctx(h); return s; }
  *out = h;
  return SP2_OK;
}

static bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + bytes && y < x + bytes;
}

static sp2_status enqueue_f64(sp2_ctx* h, const double* F, double* D, cudaStream_t s) {
  const int N = (int)h->N;
  SP2_TRY(sp2::launch_bounds_and_init(h->st_dev, F, N, N, h->part_lo, h->part_hi, h->part_bad, h->nparts, s));
  SP2_TRY(sp2::launch_scale_f64(h->st_dev, F, N, N, h->buf[0], h->ld, s));
  if (h->pert) SP2_TRY(sp2::launch_perturb(h->st_dev, h->buf[0], h->buf[1], h->pert, h->pert_count, N, 1, s));
  SP2_TRY(cudaEventRecord(h->ev_loop[0], s));
  if (h->opts.launch_mode == 0) {
    SP2_TRY(cudaGraphLaunch(h->exec, s));
  } else {
    for (int it = 0; it <= h->opts.max_iter; ++it)
      if (h->mcw)
        SP2_TRY(sp2::launch_mcw_step_plain(h->st_dev, h->buf[0], h->buf[1], h->sbuf, h->part, h->T, s, h->mscr,
                                           h->lz, N));
      else
        SP2_TRY(sp2::launch_f64_step_plain(h->st_dev, h->buf[0], h->buf[1], h->part, h->T, s, h->mscr, h->lz, N,
                                           h->pert, h->pert_count));
  }
  SP2_TRY(cudaEventRecord(h->ev_loop[1], s));
  SP2_TRY(sp2::launch_copy_out(h->st_dev, h->buf[0], h->buf[1], h->ld, N, D, N, s));
  SP2_TRY(cudaMemcpyAsync(h->st_host, h->st_dev, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  return SP2_OK;
}

static sp2_status enqueue_run(sp2_ctx* h, const double* F, double* D, cudaStream_t s) {
  sp2_status st = h->mixed ? h->mixed->enqueue(&F, &D, s) : enqueue_f64(h, F, D, s);
  if (st == SP2_OK) {
    h->last_stream = s;
    h->ran = true;
  }
  return st;
}

extern "C" sp2_status sp2_run(sp2_handle h, const double* F_dev, double* D_dev, void* stream) {
  NvtxRange range("sp2_run");
  if (!h || !F_dev || !D_dev) return SP2_ERR_INVALID_ARG;
  const size_t bytes = (size_t)h->N * h->N * sizeof(double);
  if (overlaps(F_dev, D_dev, bytes)) return SP2_ERR_INVALID_ARG;
  return enqueue_run(h, F_dev, D_dev, (cudaStream_t)stream);
}

extern "C" sp2_status sp2_run_host(sp2_handle h, const double* F_host, double* D_host, void* stream) {
  NvtxRange range("sp2_run_host");
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
  sp2_status st = enqueue_run(h, h->stage_F, h->stage_D, s);
  if (st != SP2_OK) return st;
  SP2_TRY(cudaMemcpyAsync(D_host, h->stage_D, bytes, cudaMemcpyDeviceToHost, s));
  SP2_TRY(cudaStreamSynchronize(s));
  return SP2_OK;
}

extern "C" sp2_status sp2_get_info(sp2_handle h, sp2_info* out) {
  if (!h || !out) return SP2_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (h->ran) SP2_TRY(cudaStreamSynchronize(h->last_stream));
  if (h->mixed) {
    h->mixed->info(0, h->ran, out);
    return SP2_OK;
  }
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

// ---------------------------------------------------------------------------------------------
// Batch handle
// ---------------------------------------------------------------------------------------------
// ---- SP2-ACC bounds -------------------------------------------------------------------------
// The accelerated path's inputs live in the device state; the schedule itself is computed
// by the init kernel of every run (the Gershgorin bounds it needs are found there).
struct AccFields {
  int32_t acc, n_min, n_max, pad;
  double hl[4];
};
static_assert(offsetof(DevState, n_min) == offsetof(DevState, acc) + 4 &&
                  offsetof(DevState, hl) == offsetof(DevState, acc) + 16,
              "AccFields mirrors the SP2-ACC fields of DevState");

static bool acc_bounds_valid(const double* b) {
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(b[i])) return false;
  return b[0] <= b[1] && b[1] < b[2] && b[2] <= b[3];
}

static sp2_status write_acc(DevState* st_dev, DevState* st_host, const double* bounds) {
  AccFields f;
  std::memset(&f, 0, sizeof(f));
  if (bounds) {
    f.acc = 1;
    for (int i = 0; i < 4; ++i) f.hl[i] = bounds[i];
  }
  SP2_TRY(cudaDeviceSynchronize());
  SP2_TRY(cudaMemcpy(reinterpret_cast<char*>(st_dev) + offsetof(DevState, acc), &f, sizeof(f),
                     cudaMemcpyHostToDevice));
  st_host->acc = f.acc;
  for (int i = 0; i < 4; ++i) st_host->hl[i] = f.hl[i];
  return SP2_OK;
}

static bool bounds_valid(const double* b) {
  return std::isfinite(b[0]) && std::isfinite(b[1]) && b[0] < b[1];
}

// Caller's outer bounds into one device state (and its host copy); NULL switches them off.
static sp2_status write_bounds(DevState* st_dev, DevState* st_host, const double* bounds) {
  const int32_t on = bounds ? 1 : 0;
  const double b[2] = {bounds ? bounds[0] : 0.0, bounds ? bounds[1] : 0.0};
  static_assert(offsetof(DevState, ub_hi) == offsetof(DevState, ub_lo) + sizeof(double), "ub_lo, ub_hi adjacent");
  char* base = reinterpret_cast<char*>(st_dev);
  SP2_TRY(cudaDeviceSynchronize());
  SP2_TRY(cudaMemcpy(base + offsetof(DevState, ubounds), &on, sizeof(on), cudaMemcpyHostToDevice));
  SP2_TRY(cudaMemcpy(base + offsetof(DevState, ub_lo), b, sizeof(b), cudaMemcpyHostToDevice));
  st_host->ubounds = on;
  st_host->ub_lo = b[0];
  st_host->ub_hi = b[1];
  return SP2_OK;
}

namespace sp2 {
int32_t write_bound_fields(DevState* st_dev, DevState* st_host, const double* bounds) {
  return write_bounds(st_dev, st_host, bounds);
}
bool acc_bounds_ok(const double* bounds) { return acc_bounds_valid(bounds); }
int32_t write_acc_fields(DevState* st_dev, DevState* st_host, const double* bounds) {
  return write_acc(st_dev, st_host, bounds);
}
}  // namespace sp2

extern "C" int32_t sp2_set_homo_lumo(sp2_handle h, const double* bounds) {
  if (!h || (bounds && !acc_bounds_valid(bounds))) return SP2_ERR_INVALID_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  sp2_status r = h->mixed ? write_acc(h->mixed->st_dev, h->mixed->st_host, bounds)
                          : write_acc(h->st_dev, h->st_host, bounds);
  cudaSetDevice(cur);
  return r;
}

// ---- McWeeny expansion (FP64 handles) -------------------------------------------------------
extern "C" int32_t sp2_set_mcweeny(sp2_handle h, int32_t mode, double mu, double xi) {
  if (!h || mode < 0 || mode > 2 || (mode > 0 && !std::isfinite(mu)) ||
      (mode == 2 && !(std::isfinite(xi) && xi > 0.0)))
    return SP2_ERR_INVALID_ARG;
  if (h->mixed || (mode > 0 && h->pert)) return SP2_ERR_UNSUPPORTED;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  sp2_status r = SP2_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) r = SP2_ERR_CUDA;
  if (r == SP2_OK && mode > 0 && !h->sbuf) {
    const size_t bytes = (size_t)h->ld * h->ld * sizeof(double);
    if (cudaMalloc(&h->sbuf, bytes) != cudaSuccess || cudaMemset(h->sbuf, 0, bytes) != cudaSuccess) r = SP2_ERR_NOMEM;
  }
  if (r == SP2_OK) {
    const int32_t m = mode;
    const double mx[2] = {mode > 0 ? mu : 0.0, mode == 2 ? xi : 0.0};
    static_assert(offsetof(DevState, xi) == offsetof(DevState, mu) + sizeof(double), "mu, xi adjacent");
    char* base = reinterpret_cast<char*>(h->st_dev);
    if (cudaMemcpy(base + offsetof(DevState, mcw), &m, sizeof(m), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + offsetof(DevState, mu), mx, sizeof(mx), cudaMemcpyHostToDevice) != cudaSuccess)
      r = SP2_ERR_CUDA;
  }
  if (r == SP2_OK) {
    h->st_host->mcw = mode;
    h->mcw = mode;
    if (h->opts.launch_mode == 0) r = build_f64_graph(h);
  }
  (void)cudaGetLastError();
  cudaSetDevice(cur);
  return r;
}

extern "C" int32_t sp2_set_bounds(sp2_handle h, const double* bounds) {
  if (!h || (bounds && !bounds_valid(bounds))) return SP2_ERR_INVALID_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  const sp2_status r = h->mixed ? write_bounds(h->mixed->st_dev, h->mixed->st_host, bounds)
                                : write_bounds(h->st_dev, h->st_host, bounds);
  (void)cudaGetLastError();
  cudaSetDevice(cur);
  return r;
}

extern "C" int32_t sp2_test_set_perturbation(sp2_handle h, const double* E_dev, int64_t count) {
  if (!h || count < 0 || (count > 0 && !E_dev)) return SP2_ERR_INVALID_ARG;
  if (h->mixed || (count > 0 && h->mcw)) return SP2_ERR_UNSUPPORTED;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  sp2_status r = cudaDeviceSynchronize() == cudaSuccess ? SP2_OK : SP2_ERR_CUDA;
  if (r == SP2_OK) {
    h->pert = count > 0 ? E_dev : nullptr;
    h->pert_count = count > 0 ? count : 0;
    if (h->opts.launch_mode == 0) r = build_f64_graph(h);
  }
  (void)cudaGetLastError();
  cudaSetDevice(cur);
  return r;
}

struct sp2_batch_ctx {
  int count = 0;
  int32_t precision = 0;
  int device = 0;
  std::vector<int64_t> N;
  MixedEngine* mixed = nullptr;          // SP2_PREC_MIXED
  std::vector<sp2_ctx*> singles;         // SP2_PREC_FP64: one handle per problem
  cudaStream_t last_stream = nullptr;
  bool ran = false;
};

extern "C" int32_t sp2_set_bounds_batch(sp2_batch hb, int32_t i, const double* bounds) {
  if (!hb || i < 0 || i >= hb->count || (bounds && !bounds_valid(bounds))) return SP2_ERR_INVALID_ARG;
  if (!hb->mixed) return sp2_set_bounds(hb->singles[i], bounds);
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(hb->device);
  const int k = hb->mixed->internal_of[i];
  const sp2_status r = write_bounds(hb->mixed->st_dev + k, hb->mixed->st_host + k, bounds);
  (void)cudaGetLastError();
  cudaSetDevice(cur);
  return r;
}

extern "C" int32_t sp2_set_homo_lumo_batch(sp2_batch hb, int32_t i, const double* bounds) {
  if (!hb || i < 0 || i >= hb->count || (bounds && !acc_bounds_valid(bounds))) return SP2_ERR_INVALID_ARG;
  if (!hb->mixed) return sp2_set_homo_lumo(hb->singles[i], bounds);
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(hb->device);
  const int k = hb->mixed->internal_of[i];
  sp2_status r = write_acc(hb->mixed->st_dev + k, hb->mixed->st_host + k, bounds);
  cudaSetDevice(cur);
  return r;
}

extern "C" void sp2_destroy_batch(sp2_batch hb) {
  if (!hb) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(hb->device);
  cudaDeviceSynchronize();
  delete hb->mixed;
  for (sp2_ctx* h : hb->singles) free_ctx(h);
  (void)cudaGetLastError();
  cudaSetDevice(cur);
  delete hb;
}

extern "C" sp2_status sp2_create_batch(int32_t count, const int64_t* N, const int64_t* nocc, int32_t precision,
                                       const sp2_opts* opts, sp2_batch* out) {
  if (!out) return SP2_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || count > SP2_MAX_BATCH || !N || !nocc) return SP2_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (N[i] < 1 || N[i] > 65536 || nocc[i] < 0 || nocc[i] > N[i]) return SP2_ERR_INVALID_ARG;
  if (precision < SP2_PREC_FP64 || precision > SP2_PREC_TF32X3) return SP2_ERR_UNSUPPORTED;
  sp2_opts o;
  sp2_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_valid(o)) return SP2_ERR_INVALID_ARG;
  if (precision != SP2_PREC_FP64 && o.refine_steps > 0 && o.refine_fp64 && count > 1) return SP2_ERR_UNSUPPORTED;
  if (o.norm == 2 && precision != SP2_PREC_FP64) return SP2_ERR_UNSUPPORTED;
  sp2_batch_ctx* hb = new (std::nothrow) sp2_batch_ctx();
  if (!hb) return SP2_ERR_NOMEM;
  hb->count = count;
  hb->precision = precision;
  hb->N.assign(N, N + count);
  if (cudaGetDevice(&hb->device) != cudaSuccess) { delete hb; (void)cudaGetLastError(); return SP2_ERR_CUDA; }
  sp2_status s = SP2_OK;
  if (precision != SP2_PREC_FP64) {
    hb->mixed = new (std::nothrow) MixedEngine();
    s = hb->mixed ? hb->mixed->init(count, N, nocc, o, precision) : SP2_ERR_NOMEM;
  } else {
    hb->singles.assign(count, nullptr);
    for (int i = 0; i < count && s == SP2_OK; ++i) s = sp2_create(N[i], nocc[i], SP2_PREC_FP64, &o, &hb->singles[i]);
  }
  if (s == SP2_OK && cudaDeviceSynchronize() != cudaSuccess) { (void)cudaGetLastError(); s = SP2_ERR_CUDA; }
  if (s != SP2_OK) { sp2_destroy_batch(hb); return s; }
  *out = hb;
  return SP2_OK;
}

extern "C" sp2_status sp2_run_batch(sp2_batch hb, const double* const* F_dev, double* const* D_dev, void* stream) {
  NvtxRange range("sp2_run_batch");
  if (!hb || !F_dev || !D_dev) return SP2_ERR_INVALID_ARG;
  for (int i = 0; i < hb->count; ++i) {
    if (!F_dev[i] || !D_dev[i]) return SP2_ERR_INVALID_ARG;
    if (overlaps(F_dev[i], D_dev[i], (size_t)hb->N[i] * hb->N[i] * sizeof(double))) return SP2_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  sp2_status st = SP2_OK;
  if (hb->mixed) {
    st = hb->mixed->enqueue(F_dev, D_dev, s);
  } else {
    for (int i = 0; i < hb->count && st == SP2_OK; ++i) st = enqueue_run(hb->singles[i], F_dev[i], D_dev[i], s);
  }
  if (st == SP2_OK) {
    hb->last_stream = s;
    hb->ran = true;
  }
  return st;
}

extern "C" sp2_status sp2_get_info_batch(sp2_batch hb, int32_t i, sp2_info* out) {
  if (!hb || !out || i < 0 || i >= hb->count) return SP2_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (hb->mixed) {
    if (hb->ran) SP2_TRY(cudaStreamSynchronize(hb->last_stream));
    hb->mixed->info(i, hb->ran, out);
    return SP2_OK;
  }
  return sp2_get_info(hb->singles[i], out);
}
