// batch.cuh -- ensembles of configurations of uneven lattice shapes fixed together (part of the
// lgf.cu translation unit: it uses the context internals defined there).
//
// Configurations are grouped by shape; each group is one context holding nb configurations stored one
// after the other, and every kernel of an iteration is launched once per group with gridDim.z = nb
// (each configuration has its own loop control, so a converged configuration's blocks return at once
// and every configuration's iteration count is exactly its own). K iterations of all groups -- in the
// mixed schedule both the float-stage and the double-stage kernels, each running only for the
// configurations in that stage -- are captured once in a CUDA graph and replayed until every
// configuration has stopped; between replays the host hands over each mixed configuration that has
// reached theta_switch, or whose float stage did not lower theta over the last replay. FFT pass shapes are chosen per (shape, precision) by a timing autotuner whose
// results are cached in a JSON file.

// ------------------------------------------------------------------------------------------------
// FFT autotuner: candidates are the generic passes and the specialised passes with 16- or 32-wide
// column tiles; each is timed on the context's own packed buffers and the fastest is kept. Results are
// cached in a JSON object {"<Nx>x<Ny>x<Nz>x<Nt>:<f64|f32>": {"plan": "...", "C": c, "ms": t}, ...} at
// $LGF_TUNE_CACHE (default $HOME/.cache/lgf_fft_tune.json).
// ------------------------------------------------------------------------------------------------
namespace {

struct TuneEntry {
  std::string plan;  // "fixed" or "generic"
  int C = 0;
  double ms = 0;
};

std::string tune_cache_path() {
  const char *p = std::getenv("LGF_TUNE_CACHE");
  if (p && *p) return p;
  const char *h = std::getenv("HOME");
  return std::string(h && *h ? h : "/tmp") + "/.cache/lgf_fft_tune.json";
}

std::map<std::string, TuneEntry> tune_cache_read() {
  std::map<std::string, TuneEntry> m;
  FILE *f = std::fopen(tune_cache_path().c_str(), "r");
  if (!f) return m;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
  std::fclose(f);
  size_t pos = 0;
  while ((pos = text.find('"', pos)) != std::string::npos) {
    const size_t end = text.find('"', pos + 1);
    if (end == std::string::npos) break;
    const std::string key = text.substr(pos + 1, end - pos - 1);
    const size_t brace = text.find('{', end), close = text.find('}', end);
    if (key.find(':') == std::string::npos || brace == std::string::npos || close == std::string::npos) {
      pos = end + 1;
      continue;
    }
    const std::string body = text.substr(brace, close - brace + 1);
    TuneEntry e;
    char plan[32] = {0};
    if (std::sscanf(body.c_str(), "{\"plan\": \"%31[a-z]\", \"C\": %d, \"ms\": %lf}", plan, &e.C, &e.ms) == 3) {
      e.plan = plan;
      m[key] = e;
    }
    pos = close + 1;
  }
  return m;
}

void tune_cache_write(const std::map<std::string, TuneEntry> &m) {
  const std::string path = tune_cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    mkdir(path.substr(0, slash).c_str(), 0755);  // the directory, one level deep, if missing
  }
  const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto &kv : m)
    std::fprintf(f, "  \"%s\": {\"plan\": \"%s\", \"C\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(),
                 kv.second.plan.c_str(), kv.second.C, kv.second.ms, ++i < m.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

template <typename T> std::string tune_key(const lgf_ctx *ctx) {
  return std::to_string(ctx->n[0]) + "x" + std::to_string(ctx->n[1]) + "x" + std::to_string(ctx->n[2]) + "x" +
         std::to_string(ctx->n[3]) + (sizeof(T) == 8 ? ":f64" : ":f32");
}

// Apply a candidate: re-plan the passes and opt the kernels in to their shared memory.
template <typename T> lgf_status apply_fft_choice(lgf_ctx *ctx, State<T> &S, bool generic, int C) {
  ctx->generic_fft = generic;
  ctx->fixed_cols[sizeof(T) == 8 ? 0 : 1] = C;
  plan_passes<T>(ctx, S);
  return opt_in_smem<T>(ctx, S);
}

// Time the filter passes of the current plan (ms per application, median of 5 after 2 warm-ups).
template <typename T> lgf_status time_fft(lgf_ctx *ctx, State<T> &S, double *ms_out) {
  const bool timing = ctx->timing;
  ctx->timing = false;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  std::vector<float> t;
  for (int rep = 0; rep < 7; ++rep) {
    CK(cudaEventRecord(a, ctx->stream));
    TRY(launch_filter<T>(ctx, S, S.P, 0));
    CK(cudaEventRecord(b, ctx->stream));
    CK(cudaEventSynchronize(b));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (rep >= 2) t.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  ctx->timing = timing;
  return LGF_OK;
}

template <typename T> lgf_status autotune_fft(lgf_ctx *ctx, State<T> &S, TuneEntry *chosen) {
  const std::string key = tune_key<T>(ctx);
  auto cache = tune_cache_read();
  auto it = cache.find(key);
  if (it != cache.end()) {
    TRY(apply_fft_choice<T>(ctx, S, it->second.plan == "generic", it->second.C));
    *chosen = it->second;
    return LGF_OK;
  }
  CK(cudaMemsetAsync(S.P, 0, sizeof(T) * 2 * 4 * (size_t)ctx->V * ctx->nb, ctx->stream));
  struct Cand {
    bool generic;
    int C;
  };
  const Cand cands[] = {{true, 0}, {false, 16}, {false, 32}};
  TuneEntry best;
  best.ms = 1e30;
  for (const Cand &c : cands) {
    TRY(apply_fft_choice<T>(ctx, S, c.generic, c.C));
    const bool fixed_plan = !S.passes.empty() && S.passes[0].kind != 0;
    if (!c.generic && !fixed_plan) continue;  // the specialised passes do not fit this shape
    double ms = 0;
    TRY(time_fft<T>(ctx, S, &ms));
    if (ms < best.ms) {
      best.ms = ms;
      best.plan = c.generic ? "generic" : "fixed";
      best.C = c.C;
    }
  }
  TRY(apply_fft_choice<T>(ctx, S, best.plan == "generic", best.C));
  cache = tune_cache_read();
  cache[key] = best;
  tune_cache_write(cache);
  *chosen = best;
  return LGF_OK;
}

}  // namespace

struct lgf_batch {
  int n = 0;
  std::vector<lgf_ctx *> groups;
  std::vector<int> group_of, index_of;  // configuration -> (group, index within group)
  cudaStream_t stream = nullptr;
  std::string err;
  bool poisoned = false;
  bool autotune = true;
  std::string tuned[2];  // description of the tuned FFT plans per group, double / float
  cudaStream_t body_stream = nullptr;  // captures the bodies of the graph's conditional nodes
  cudaGraphExec_t graph = nullptr;
  int graph_prec = -1, graph_chunk = 0;
  double graph_alpha = 0;
  int launches_per_replay = 0;  // kernels in the graph (those inside the IF bodies run only when guarded in)
  int guarded_stages = 0;       // IF nodes: one per (iteration, group, stage)
  long graph_replays = 0;
};

namespace {

// Condition of the IF node that guards one stage's iteration of a group in the replayed graph: 1 when some
// configuration of the group is active in that stage (0 float, 1 double, kStageResidual), else 0, and then
// none of that iteration's kernels is launched. The kernels inside still check each configuration.
__global__ void k_stage_condition(cudaGraphConditionalHandle h, const Ctrl *ctrl, int nb, int stage) {
  int any = 0;
  for (int j = threadIdx.x; j < nb; j += 32) any |= (ctrl[j].active && ctrl[j].stage == stage) ? 1 : 0;
  any = __any_sync(0xffffffffu, any);
  if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

lgf_status bfail(lgf_batch *b, lgf_status st, const std::string &msg) {
  if (b) {
    b->err = msg;
    if (st == LGF_ECUDA) b->poisoned = true;
  }
  return st;
}

// Appends to the graph being captured on b->stream one stage's iteration of group g, guarded by an IF node:
// a one-warp kernel sets the condition from the group's loop controls, and the iteration's kernels form the
// body (captured on b->body_stream), so a stage that no configuration of the group is in costs that one small
// launch instead of a full launch of every kernel of the iteration.
template <typename Fn> lgf_status add_guarded_stage(lgf_batch *b, lgf_ctx *g, int stage, Fn &&body) {
  lgf_ctx *ctx = g;
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(b->stream, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault));
  k_stage_condition<<<1, 32, 0, b->stream>>>(h, g->ctrl, g->nb, stage);
  CKL();
  CK(cudaStreamGetCaptureInfo(b->stream, &cs, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &p));
  CK(cudaStreamUpdateCaptureDependencies(b->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(b->body_stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaStream_t saved = g->stream;
  g->stream = b->body_stream;
  const lgf_status st = body();
  g->stream = saved;
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->body_stream, &out);
  if (st != LGF_OK) return st;
  if (e != cudaSuccess) return fail(ctx, LGF_ECUDA, std::string("body capture: ") + cudaGetErrorString(e));
  return LGF_OK;
}

#define BCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? LGF_ENOMEM : LGF_ECUDA,                   \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                           \
  } while (0)
#define BTRY(g, x)                                                                                \
  do {                                                                                            \
    lgf_status s_ = (x);                                                                          \
    if (s_ != LGF_OK) return bfail(b, s_, (g)->err);                                              \
  } while (0)

// Plane-offset helpers for configuration j of a group.
template <typename T> T *cfg_links(T *base, const lgf_ctx *g, int j) {
  return base + (int64_t)j * 4 * LinkStore<T>::planes * g->V * 2;
}
template <typename T> T *cfg_packed(T *base, const lgf_ctx *g, int j) { return base + (int64_t)j * 4 * g->V * 2; }
template <typename T> T *cfg_mat(T *base, const lgf_ctx *g, int j) { return base + (int64_t)j * 9 * g->V * 2; }
float *cfg_gacc(float *base, const lgf_ctx *g, int j) { return base + (int64_t)j * 6 * g->V * 2; }  // rows 0-1

// Delta, theta and F of configuration j alone (used at load and after a handover).
template <typename T> lgf_status delta_one(lgf_ctx *g, State<T> &S, int j) {
  lgf_ctx *ctx = g;
  return with_fft_type<T>(g, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    if constexpr (std::is_same<T, float>::value)
      k_delta_f32<NT><<<dim3(g->nblocks_site, 1, 1), NT, 0, g->stream>>>(
          cfg_links(S.U, g, j), cfg_packed(S.P, g, j), g->partials + (int64_t)j * 2 * g->nblocks_site, g->ctrl + j,
          g->L, 0, 0, 0);
    else
      k_delta<T, NT, FT><<<dim3(g->nblocks_site, 1, 1), NT, 0, g->stream>>>(
          cfg_links(S.U, g, j), reinterpret_cast<FT *>(cfg_packed(S.P, g, j)),
          g->partials + (int64_t)j * 2 * g->nblocks_site, g->ctrl + j, g->L, 0, 0, 0);
    CKL();
    return LGF_OK;
  });
}

// Handover of configuration j; with base, rows 0-1 of the new links rounded to float also go to its float
// link planes (the base of its residual stage).
lgf_status handover_one(lgf_ctx *g, int j, bool base) {
  lgf_ctx *ctx = g;
  k_gacc_to_double<NT><<<grid1(g->V, NT), NT, 0, g->stream>>>(cfg_gacc(g->Gacc, g, j), cfg_mat(g->s64.G, g, j), g->V);
  CKL();
  k_transform_from_q<NT><<<grid1(g->V, NT), NT, 0, g->stream>>>(cfg_links(g->U0, g, j), cfg_links(g->s64.U, g, j),
                                                                cfg_mat(g->s64.G, g, j), g->L,
                                                                base ? cfg_links(g->s32.U, g, j) : nullptr,
                                                                g->handover_split[0], g->handover_split[1]);
  CKL();
  return LGF_OK;
}

// Residual stage of configuration j (see lgf_iterate), entered after its double Delta, theta and F: the
// base links (narrowed from the double links unless the handover wrote them), R = K = 0, the loop
// control's transition (on the device) and the initial Delta.
lgf_status enter_residual_one(lgf_ctx *g, int j, double eps, bool narrow) {
  lgf_ctx *ctx = g;
  const int64_t V = g->V;
  if (narrow) {
    k_narrow_link_planes<<<grid1(4 * V, NT), NT, 0, g->stream>>>(cfg_links(g->s64.U, g, j), cfg_links(g->s32.U, g, j), V,
                                                                  0, 4 * V);
    CKL();
  }
  CK(cudaMemsetAsync(g->Rres + (int64_t)j * 72 * V, 0, sizeof(float) * 72 * (size_t)V, g->stream));
  CK(cudaMemsetAsync(g->Kres + (int64_t)j * 18 * V, 0, sizeof(float) * 18 * (size_t)V, g->stream));
  k_enter_residual<<<1, 1, 0, g->stream>>>(g->ctrl + j, 0.8 * eps);
  CKL();
  return with_fft_type<double>(g, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    k_delta_residual<NT, FT><<<dim3(g->nblocks_site, 1, 1), NT, 0, g->stream>>>(
        g->Rres + (int64_t)j * 72 * V, reinterpret_cast<const FT *>(cfg_packed(g->s64.P, g, j)),
        cfg_packed(g->s32.P, g, j), g->partials + (int64_t)j * 2 * g->nblocks_site, g->ctrl + j, g->L, 0, 0);
    CKL();
    return LGF_OK;
  });
}

// End of the residual stage of configuration j: H = proj(1 + K) in double and the double links rebuilt by
// the double update (small-step form), in place.
lgf_status rebuild_one(lgf_ctx *g, int j) {
  lgf_ctx *ctx = g;
  const int64_t V = g->V;
  float *A = g->s64.A + (int64_t)j * 9 * V * 4;
  k_residual_gauge<NT><<<grid1(V, NT), NT, 0, g->stream>>>(g->Kres + (int64_t)j * 18 * V, cfg_mat(g->s64.G, g, j), A, V);
  CKL();
  k_update<double, NT_UPDATE64><<<dim3(grid1(V, NT_UPDATE64), 1, 1), NT_UPDATE64, update_smem_bytes<NT_UPDATE64>(),
                                  g->stream>>>(cfg_links(g->s64.U, g, j), cfg_mat(g->s64.G, g, j), A, g->L, g->ctrl + j,
                                               0, 0, g->small_step ? 1 : 0, g->update_split[0], g->update_split[1]);
  CKL();
  return LGF_OK;
}

}  // namespace

extern "C" {

lgf_status lgf_batch_create(int n, const int *dims, lgf_batch **out) {
  if (!out || !dims || n < 1) return fail(nullptr, LGF_EINVAL, "lgf_batch_create: bad arguments");
  *out = nullptr;
  lgf_batch *b = new lgf_batch();
  b->n = n;
  std::vector<std::array<int, 4>> shapes;
  std::vector<int> counts;
  for (int i = 0; i < n; ++i) {
    std::array<int, 4> d = {dims[4 * i], dims[4 * i + 1], dims[4 * i + 2], dims[4 * i + 3]};
    int g = -1;
    for (size_t k = 0; k < shapes.size(); ++k)
      if (shapes[k] == d) g = (int)k;
    if (g < 0) {
      shapes.push_back(d);
      counts.push_back(0);
      g = (int)shapes.size() - 1;
    }
    b->group_of.push_back(g);
    b->index_of.push_back(counts[g]++);
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->body_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return fail(nullptr, LGF_ECUDA, "cudaStreamCreate failed");
  }
  for (size_t g = 0; g < shapes.size(); ++g) {
    lgf_ctx *c = nullptr;
    const lgf_status st = create_ctx(shapes[g].data(), counts[g], &c);
    if (st != LGF_OK) {
      lgf_batch_destroy(b);
      return st;
    }
    c->stream = b->stream;
    b->groups.push_back(c);
  }
  const char *t = std::getenv("LGF_AUTOTUNE");
  b->autotune = !(t && t[0] == '0');
  *out = b;
  return LGF_OK;
}

void lgf_batch_destroy(lgf_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (lgf_ctx *c : b->groups) {
    c->stream = c->own_stream;
    lgf_destroy(c);
  }
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->body_stream) cudaStreamDestroy(b->body_stream);
  delete b;
}

const char *lgf_batch_last_error(const lgf_batch *b) { return b ? b->err.c_str() : ""; }

lgf_status lgf_batch_fix(lgf_batch *b, double *const *links, double alpha, double eps, const lgf_options *opt,
                         double *theta, double *F, int *iters, int *status) {
  if (!b) return fail(nullptr, LGF_EINVAL, "null batch");
  if (b->poisoned) return LGF_ECUDA;
  if (!links || !(alpha > 0) || !(eps >= 0)) return bfail(b, LGF_EINVAL, "bad links, alpha or eps");
  lgf_options o;
  lgf_default_options(&o);
  if (opt) o = *opt;
  if (o.reunit_period < 1) o.reunit_period = 1;
  const int prec = o.precision;
  if (prec != LGF_FP64 && prec != LGF_MIXED && prec != LGF_FP32) return bfail(b, LGF_EINVAL, "unknown precision");
  const bool has_float = prec != LGF_FP64, has_double = prec != LGF_FP32;
  // buffers, FFT plans (autotuned) and loads
  b->tuned[0].clear();
  b->tuned[1].clear();
  for (lgf_ctx *g : b->groups) {
    BTRY(g, check_ctx(g));
    BTRY(g, ensure_common(g));
    if (has_double) {
      BTRY(g, setup_precision<double>(g, g->s64));
      TuneEntry e;
      if (b->autotune) BTRY(g, autotune_fft<double>(g, g->s64, &e));
      b->tuned[0] += tune_key<double>(g) + "=" + (b->autotune ? e.plan + "/" + std::to_string(e.C) : "default") + " ";
    }
    if (has_float) {
      BTRY(g, setup_precision<float>(g, g->s32));
      BTRY(g, alloc(g, &g->Gacc, (size_t)g->nb * 6 * g->V * 2));
      if (prec == LGF_MIXED) BTRY(g, alloc(g, &g->U0, (size_t)g->nb * 4 * 9 * g->V * 2));
      if (prec == LGF_MIXED && g->residual) {
        BTRY(g, alloc(g, &g->Rres, (size_t)g->nb * 72 * g->V));
        BTRY(g, alloc(g, &g->Kres, (size_t)g->nb * 18 * g->V));
      }
      TuneEntry e;
      if (b->autotune) BTRY(g, autotune_fft<float>(g, g->s32, &e));
      b->tuned[1] += tune_key<float>(g) + "=" + (b->autotune ? e.plan + "/" + std::to_string(e.C) : "default") + " ";
    }
  }
  for (int i = 0; i < b->n; ++i) {
    lgf_ctx *g = b->groups[b->group_of[i]];
    lgf_ctx *ctx = g;
    const int j = b->index_of[i];
    const double *src = nullptr;
    BTRY(g, input_ptr(g, links[i], (size_t)4 * g->V * 144, &g->staging, &g->staging_bytes, &src));
    if (prec == LGF_FP64) {
      BTRY(g, to_planes<double>(g, src, cfg_links(g->s64.U, g, j), 4));
    } else {
      if (prec == LGF_MIXED) BTRY(g, to_planes<double>(g, src, cfg_links(g->U0, g, j), 4));
      BTRY(g, to_planes<float>(g, src, cfg_links(g->s32.U, g, j), 4));
      k_set_identity<<<grid1(g->V, NT), NT, 0, g->stream>>>(cfg_gacc(g->Gacc, g, j), g->V);
      CKL();
    }
  }
  // loop control of every configuration, then Delta/theta/F of the inputs
  const double thr0 = prec == LGF_MIXED ? std::max(eps, o.theta_switch) : eps;
  std::vector<std::vector<Ctrl>> host(b->groups.size());
  for (size_t k = 0; k < b->groups.size(); ++k) {
    lgf_ctx *g = b->groups[k];
    host[k].assign(g->nb, Ctrl{});
    for (Ctrl &c : host[k]) {
      c.threshold = thr0;
      c.limit = o.max_iter;
      c.active = 1;
      c.stage = prec == LGF_FP64 ? 1 : 0;
    }
    BCK(cudaMemcpyAsync(g->ctrl, host[k].data(), sizeof(Ctrl) * g->nb, cudaMemcpyHostToDevice, b->stream));
    if (prec == LGF_FP64) BTRY(g, launch_delta<double>(g, g->s64, 0, 0));
    else BTRY(g, launch_delta<float>(g, g->s32, 0, 0));
  }
  // the captured chunk: reunit_period iterations of every group (the last one reprojects the float links)
  const int chunk = o.reunit_period;
  if (!b->graph || b->graph_prec != prec || b->graph_chunk != chunk || b->graph_alpha != alpha) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    for (lgf_ctx *g : b->groups) g->timing = false;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    b->guarded_stages = 0;
    int launches = 0;
    lgf_status cst = LGF_OK;
    std::string cmsg;
    for (int k = 0; k < chunk && cst == LGF_OK; ++k)
      for (lgf_ctx *g : b->groups) {
        if (has_float && cst == LGF_OK) {
          cst = add_guarded_stage(b, g, 0, [&]() { return launch_iteration_float(g, alpha, k == chunk - 1); });
          launches += (int)g->s32.passes.size() + 3;
        }
        if (has_double && cst == LGF_OK) {
          cst = add_guarded_stage(b, g, 1, [&]() { return launch_iteration<double>(g, g->s64, alpha); });
          launches += (int)g->s64.passes.size() + 4;
        }
        if (prec == LGF_MIXED && g->residual && cst == LGF_OK) {
          cst = add_guarded_stage(b, g, kStageResidual, [&]() { return launch_iteration_residual(g, alpha); });
          launches += (int)g->s32.passes.size() + 3;
        }
        if (cst != LGF_OK && cmsg.empty()) cmsg = g->err;
        b->guarded_stages += (has_float ? 1 : 0) + (has_double ? 1 : 0) + (prec == LGF_MIXED && g->residual ? 1 : 0);
      }
    if (cst != LGF_OK) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(b->stream, &junk);
      if (junk) cudaGraphDestroy(junk);
      return bfail(b, cst, cmsg.empty() ? "graph capture failed" : cmsg);
    }
    cudaGraph_t graph;
    BCK(cudaStreamEndCapture(b->stream, &graph));
    BCK(cudaGraphInstantiate(&b->graph, graph, 0));
    cudaGraphDestroy(graph);
    b->graph_prec = prec;
    b->graph_chunk = chunk;
    b->graph_alpha = alpha;
    b->launches_per_replay = launches;
  }
  b->graph_replays = 0;
  // replay until every configuration has stopped. Mixed configurations hand over at theta_switch, or
  // when a replay of the float stage did not lower theta (the resolution of float links is reached),
  // then run the residual stage; at its end (or when a replay of it did not lower theta) the double
  // links are rebuilt and theta is recomputed in double, and the stage starts again from the rebuilt
  // links while theta >= eps -- after three rebuilds double iterations take over instead.
  std::vector<std::vector<std::pair<double, int>>> last(b->groups.size());
  std::vector<std::vector<int>> rebuilds(b->groups.size());
  for (size_t k = 0; k < b->groups.size(); ++k) {
    last[k].assign(b->groups[k]->nb, {0.0, -1});
    rebuilds[k].assign(b->groups[k]->nb, 0);
  }
  for (;;) {
    bool pending = false;
    for (size_t k = 0; k < b->groups.size(); ++k) {
      lgf_ctx *g = b->groups[k];
      BCK(cudaMemcpyAsync(host[k].data(), g->ctrl, sizeof(Ctrl) * g->nb, cudaMemcpyDeviceToHost, b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));
    for (size_t k = 0; k < b->groups.size(); ++k) {
      lgf_ctx *g = b->groups[k];
      for (int j = 0; j < g->nb; ++j) {
        Ctrl &c = host[k][j];
        if (c.status == 5) continue;
        const bool residual = prec == LGF_MIXED && g->residual;
        const bool stalled = prec == LGF_MIXED && (c.stage == 0 || c.stage == kStageResidual) && c.active &&
                             last[k][j].second >= 0 && last[k][j].second < c.iters &&
                             !(c.theta < last[k][j].first);
        last[k][j] = {c.theta, c.iters};
        if (c.active && !stalled) {
          pending = true;
        } else if (prec == LGF_MIXED && c.stage == 0 && (c.theta < thr0 || stalled) && c.iters < c.limit) {
          BTRY(g, setup_precision<double>(g, g->s64));
          BTRY(g, handover_one(g, j, residual));
          c.stage = 1;
          c.threshold = eps;
          c.active = 1;
          BCK(cudaMemcpyAsync(g->ctrl + j, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, b->stream));
          BTRY(g, delta_one<double>(g, g->s64, j));
          if (residual) BTRY(g, enter_residual_one(g, j, eps, false));
          last[k][j] = {0.0, -1};
          pending = true;
        } else if (c.stage == kStageResidual) {
          BTRY(g, rebuild_one(g, j));
          c.stage = 1;
          c.threshold = eps;
          c.active = 1;
          BCK(cudaMemcpyAsync(g->ctrl + j, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, b->stream));
          BTRY(g, delta_one<double>(g, g->s64, j));
          k_set_active<<<1, 1, 0, b->stream>>>(g->ctrl + j, 0);  // the host decides what follows
          BCK(cudaGetLastError());
          ++rebuilds[k][j];
          last[k][j] = {0.0, -1};
          pending = true;
        } else if (residual && c.stage == 1 && rebuilds[k][j] > 0 && !(c.theta < eps) && c.iters < c.limit) {
          if (rebuilds[k][j] < 4) {
            BTRY(g, enter_residual_one(g, j, eps, true));
          } else {
            c.active = 1;
            BCK(cudaMemcpyAsync(g->ctrl + j, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, b->stream));
          }
          last[k][j] = {0.0, -1};
          pending = true;
        }
      }
    }
    if (!pending) break;
    BCK(cudaGraphLaunch(b->graph, b->stream));
    ++b->graph_replays;
  }
  // results and store
  lgf_status result = LGF_OK;
  for (int i = 0; i < b->n; ++i) {
    const int k = b->group_of[i], j = b->index_of[i];
    lgf_ctx *g = b->groups[k];
    const Ctrl &c = host[k][j];
    const lgf_status st = c.status == 5 ? LGF_ENONFINITE : (c.theta < eps ? LGF_OK : LGF_ENOCONV);
    if (theta) theta[i] = c.theta;
    if (F) F[i] = c.F;
    if (iters) iters[i] = c.iters;
    if (status) status[i] = st;
    if (st != LGF_OK && result == LGF_OK) result = st;
    if (st == LGF_ENONFINITE) continue;
    double *dst = nullptr;
    bool hostp = false;
    BTRY(g, output_ptr(g, links[i], (size_t)4 * g->V * 144, &g->staging, &g->staging_bytes, &dst, &hostp));
    if (c.stage == 1) {
      BTRY(g, from_planes<double>(g, cfg_links(g->s64.U, g, j), dst, 4));
    } else if (prec == LGF_MIXED) {
      BTRY(g, setup_precision<double>(g, g->s64));
      BTRY(g, handover_one(g, j, false));
      BTRY(g, from_planes<double>(g, cfg_links(g->s64.U, g, j), dst, 4));
    } else {
      BTRY(g, from_planes<float>(g, cfg_links(g->s32.U, g, j), dst, 4));
    }
    if (hostp) BCK(cudaMemcpyAsync(links[i], dst, (size_t)4 * g->V * 144, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
  }
  if (result == LGF_ENONFINITE) return bfail(b, result, "theta or F is not finite for a configuration");
  return result;
}

lgf_status lgf_batch_describe(const lgf_batch *b, char *buf, int len) {
  if (!b || !buf || len < 1) return LGF_EINVAL;
  std::string s = "{\"configs\": " + std::to_string(b->n) + ", \"groups\": [";
  for (size_t k = 0; k < b->groups.size(); ++k) {
    const lgf_ctx *g = b->groups[k];
    s += std::string(k ? ", " : "") + "{\"dims\": [" + std::to_string(g->n[0]) + ", " + std::to_string(g->n[1]) +
         ", " + std::to_string(g->n[2]) + ", " + std::to_string(g->n[3]) + "], \"configs\": " + std::to_string(g->nb) +
         "}";
  }
  s += "], \"fft_f64\": \"" + b->tuned[0] + "\", \"fft_f32\": \"" + b->tuned[1] +
       "\", \"launches_per_replay\": " + std::to_string(b->launches_per_replay) +
       ", \"guarded_stages\": " + std::to_string(b->guarded_stages) +
       ", \"graph_replays\": " + std::to_string(b->graph_replays) + "}";
  std::snprintf(buf, (size_t)len, "%s", s.c_str());
  return LGF_OK;
}

}  // extern "C"
