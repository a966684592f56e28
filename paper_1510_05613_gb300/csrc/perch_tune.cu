// Launch-configuration autotuner and CUDA-graph capture of the evaluation.
//
// The evaluation runs one persistent launch per mesh (its own shared-memory
// tile, sized by the mesh's largest screen box over the pose grid). The
// autotuner times the CTA widths the kernel is compiled for on a sample of
// each mesh's hypotheses and keeps the fastest per mesh; results are cached
// in the process by (triangle count, vertex count, tile), so contexts with the
// same meshes and camera reuse them. The graph entry point captures the whole
// evaluation sequence (parent z-buffers, residual sets, grouping, the
// per-mesh launches and optionally the record download) once per argument set
// and replays it.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "perch_ctx.h"
#include "perch_internal.h"

using namespace perch;

namespace {

using TuneKey = std::tuple<int, int, int, int, int, int>;  // device, tris, verts, tile_w, tile_h, shared renders
std::mutex g_tune_mu;
struct TuneChoice {
  int threads, inline_px, cost_threads, bin_depth, cost_stages;
};
std::map<TuneKey, TuneChoice> g_tune_cache;

constexpr int kWidths[3] = {128, 256, 512};
constexpr int kInline[3] = {8, 16, 32};  // k_render's inline limit (candidate pixel centres per lane)
constexpr int kCostWidths[2] = {128, 256};
constexpr int kBinDepths[3] = {32, 64, 128};  // the render's shared bin of larger triangles

}  // namespace

#define CK(expr, what)                 \
  do {                                 \
    int rc_ = ctx->cuda((expr), what); \
    if (rc_ != PERCH_OK) return rc_;   \
  } while (0)

extern "C" int perch_autotune(perch_ctx* ctx, int32_t n_sample, int32_t* threads_out) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  if (n_sample < 1 || n_sample > (1 << 22)) return ctx->fail(PERCH_E_ARG, "n_sample out of range");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  // time throughput, not latency: the sample must keep every SM busy for
  // many items, or wide CTAs win by finishing a near-empty launch sooner
  n_sample = std::max(n_sample, 32 * ctx->sm_count);
  const int n_mesh = ctx->n_mesh;
  const long long n_poses = (long long)ctx->nx * ctx->ny * ctx->n_yaw;
  // children of two empty parents, alternating (a batch of two parents takes
  // the shared-render path when it is on; every pose appears once)
  std::vector<perch_obj> hyps(n_sample);
  std::vector<int32_t> hp(n_sample, 0);
  for (int i = 0; i < n_sample; ++i) hp[i] = i & 1;
  const int32_t plen[2] = {0, 0};
  CK(ctx->b_parents.ensure(2 * sizeof(perch_obj)), "alloc");
  CK(ctx->b_plen.ensure(8), "alloc");
  CK(ctx->b_hp.ensure(4 * (size_t)n_sample), "alloc");
  CK(ctx->b_hyp.ensure(sizeof(perch_obj) * (size_t)n_sample), "alloc");
  CK(ctx->b_out.ensure(sizeof(perch_cost) * (size_t)n_sample), "alloc");
  CK(cudaMemcpyAsync(ctx->b_plen.p, plen, 8, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->b_hp.p, hp.data(), 4 * (size_t)n_sample, cudaMemcpyHostToDevice, ctx->stream), "copy");
  const std::vector<int> saved = ctx->mesh_threads;
  // time the rasteriser itself: the exact shortcut would skip most root
  // children, and the render cache every render after the first
  struct ShortcutOff {
    perch_ctx* c;
    bool was, cache;
    ~ShortcutOff() {
      c->shortcut = was;
      c->render_cache = cache;
    }
  } shortcut_off{ctx, ctx->shortcut, ctx->render_cache};
  ctx->shortcut = false;
  ctx->render_cache = false;
  const bool shared = ctx->share_renders && ctx->store_ok;
  const std::vector<int> saved_cost = ctx->mesh_cost_threads, saved_inline = ctx->mesh_inline,
                         saved_bins = ctx->mesh_queue, saved_stages = ctx->mesh_cost_stages;
  auto restore = [&]() {
    ctx->mesh_threads = saved;
    ctx->mesh_cost_threads = saved_cost;
    ctx->mesh_inline = saved_inline;
    ctx->mesh_queue = saved_bins;
    ctx->mesh_cost_stages = saved_stages;
  };
  for (int m = 0; m < n_mesh; ++m) {
    const TuneKey key{ctx->device,          ctx->h_meshes[m].n_tris, ctx->h_meshes[m].n_verts,
                      ctx->mesh_tile_w[m], ctx->mesh_tile_h[m],     shared ? 1 : 0};
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        ctx->mesh_threads[m] = it->second.threads;
        ctx->mesh_inline[m] = it->second.inline_px;
        ctx->mesh_cost_threads[m] = it->second.cost_threads;
        ctx->mesh_queue[m] = it->second.bin_depth;
        ctx->mesh_cost_stages[m] = it->second.cost_stages;
        continue;
      }
    }
    // a spread of poses of mesh m (a fixed stride through the pose grid)
    const long long stride = std::max(1LL, n_poses / n_sample) | 1LL;
    for (int i = 0; i < n_sample; ++i) {
      const long long q = (i * stride) % n_poses;
      perch_obj o;
      o.mesh = (uint16_t)m;
      o.iyaw = (uint16_t)(q % ctx->n_yaw);
      o.iy = (int16_t)((q / ctx->n_yaw) % ctx->ny);
      o.ix = (int16_t)(q / ((long long)ctx->n_yaw * ctx->ny));
      hyps[i] = o;
    }
    CK(cudaMemcpyAsync(ctx->b_hyp.p, hyps.data(), sizeof(perch_obj) * (size_t)n_sample, cudaMemcpyHostToDevice,
                       ctx->stream),
       "copy");
    // time one phase (ev[a] -> ev[a + 1]) of the sample's evaluation: the
    // render launches (k_render, or k_eval when every hypothesis is
    // rendered) or the cost launches (k_cost)
    auto time_phase = [&](int a, float& out) -> int {
      float ms = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        int rc = ctx->enqueue_eval(ctx->b_parents.as<perch_obj>(), 1, ctx->b_plen.as<int32_t>(), 2,
                                   ctx->b_hp.as<int32_t>(), ctx->b_hyp.as<perch_obj>(), n_sample, 1,
                                   ctx->b_out.as<perch_cost>());
        if (rc != PERCH_OK) return rc;
        float b = 0.0f;
        CK(cudaEventSynchronize(ctx->ev[4]), "event sync");
        CK(cudaEventElapsedTime(&b, ctx->ev[a], ctx->ev[a + 1]), "event time");
        if (rep > 0) ms = std::min(ms, b);  // the first launch of a width also loads its code
      }
      out = ms;
      return PERCH_OK;
    };
    // the render: CTA width x inline limit (the limit only applies to
    // k_render; the per-hypothesis kernel keeps kInlinePixels)
    int best = 256, best_inline = ctx->mesh_inline[m], best_cost = ctx->mesh_cost_threads[m];
    float best_ms = 1e30f;
    for (int w : kWidths)
      for (int il : kInline) {
        if (!shared && il != kInlinePixels) continue;
        ctx->mesh_threads[m] = w;
        ctx->mesh_inline[m] = il;
        float ms = 0.0f;
        const int rc = time_phase(2, ms);
        if (rc != PERCH_OK) {
          restore();
          return rc;
        }
        if (ms < best_ms) {
          best_ms = ms;
          best = w;
          best_inline = il;
        }
      }
    ctx->mesh_threads[m] = best;
    ctx->mesh_inline[m] = best_inline;
    // then the depth of the bin of larger triangles, at that width and limit
    int best_bins = ctx->mesh_queue[m];
    best_ms = 1e30f;
    for (int d : kBinDepths) {
      ctx->mesh_queue[m] = d;
      float ms = 0.0f;
      const int rc = time_phase(2, ms);
      if (rc != PERCH_OK) {
        restore();
        return rc;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best_bins = d;
      }
    }
    ctx->mesh_queue[m] = best_bins;
    int best_stages = ctx->mesh_cost_stages[m];
    if (shared) {
      // the cost: CTA width x stage buffers (two only where they fit)
      best_ms = 1e30f;
      for (int w : kCostWidths)
        for (int ns = 1; ns <= 2; ++ns) {
          if (ns == 2 && !cost_stages_fit(ctx->device, ctx->mesh_tile_w[m], ctx->mesh_tile_h[m], 2)) continue;
          ctx->mesh_cost_threads[m] = w;
          ctx->mesh_cost_stages[m] = ns;
          float ms = 0.0f;
          const int rc = time_phase(3, ms);
          if (rc != PERCH_OK) {
            restore();
            return rc;
          }
          if (ms < best_ms) {
            best_ms = ms;
            best_cost = w;
            best_stages = ns;
          }
        }
      ctx->mesh_cost_threads[m] = best_cost;
      ctx->mesh_cost_stages[m] = best_stages;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {best, best_inline, best_cost, best_bins, best_stages};
  }
  if (threads_out)
    for (int m = 0; m < n_mesh; ++m) threads_out[m] = ctx->mesh_threads[m];
  return PERCH_OK;
}

extern "C" int perch_eval_graph(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                                const int32_t* parent_len, int32_t n_par, const int32_t* hyp_parent,
                                const perch_obj* hyp, int64_t n_hyp, int32_t K_total, perch_cost* out,
                                perch_cost* out_host) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  if (n_hyp < 1 || n_hyp > 0x7fffffffLL) return ctx->fail(PERCH_E_ARG, "n_hyp out of range");
  if (!parent_len || !hyp_parent || !hyp || !out || n_par < 1 || parent_stride < 0 || K_total < 1 ||
      (parent_stride > 0 && !parents))
    return ctx->fail(PERCH_E_ARG, "null pointer or bad sizes");
  if (n_par > 65535 || (long long)n_par * std::max(parent_stride, 1) > 65535)
    return ctx->fail(PERCH_E_ARG, "too many parents in one batch (n_par x stride <= 65535)");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  GraphKey key{parents, parent_stride, parent_len, n_par, hyp_parent, hyp, n_hyp, K_total, out, out_host,
               ctx->tables_version, DevBuf::reallocs};
  if (!ctx->graph_exec || std::memcmp(&key, &ctx->graph_key, sizeof key) != 0) {
    if (ctx->graph_exec) {
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
    // one plain run sizes every buffer and sets kernel attributes, so the
    // capture below records only stream work (no allocation)
    int rc = ctx->enqueue_eval(parents, parent_stride, parent_len, n_par, hyp_parent, hyp, n_hyp, K_total, out);
    if (rc != PERCH_OK) return rc;
    CK(cudaStreamSynchronize(ctx->stream), "graph warm-up");
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    ctx->capturing = true;
    rc = ctx->enqueue_eval(parents, parent_stride, parent_len, n_par, hyp_parent, hyp, n_hyp, K_total, out);
    if (rc == PERCH_OK && out_host)
      rc = ctx->cuda(cudaMemcpyAsync(out_host, out, sizeof(perch_cost) * (size_t)n_hyp, cudaMemcpyDeviceToHost,
                                     ctx->stream),
                     "record download");
    ctx->capturing = false;
    const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
    if (rc != PERCH_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    CK(ec, "end capture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei, "graph instantiate");
    ctx->graph_exec = exec;
    key.reallocs = DevBuf::reallocs;  // the warm-up run may have grown buffers; the capture uses those
    ctx->graph_key = key;
  }
  CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream), "graph launch");
  return PERCH_OK;
}

extern "C" int perch_launch_config(perch_ctx* ctx, int32_t* render_threads, int32_t* inline_pixels,
                                   int32_t* cost_threads) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if ((int)ctx->mesh_threads.size() != ctx->n_mesh || (int)ctx->mesh_cost_threads.size() != ctx->n_mesh ||
      (int)ctx->mesh_inline.size() != ctx->n_mesh)
    return ctx->fail(PERCH_E_STATE, "no meshes and camera yet");
  for (int m = 0; m < ctx->n_mesh; ++m) {
    if (render_threads) render_threads[m] = ctx->mesh_threads[m];
    if (inline_pixels) inline_pixels[m] = ctx->mesh_inline[m];
    if (cost_threads) cost_threads[m] = ctx->mesh_cost_threads[m];
  }
  return PERCH_OK;
}

extern "C" int perch_set_inline_pixels(perch_ctx* ctx, int32_t mesh, int32_t inline_pixels) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (inline_pixels != 8 && inline_pixels != 16 && inline_pixels != 32)
    return ctx->fail(PERCH_E_ARG, "inline limit must be 8, 16 or 32");
  if (mesh < -1 || mesh >= ctx->n_mesh) return ctx->fail(PERCH_E_ARG, "mesh %d out of range", mesh);
  if ((int)ctx->mesh_inline.size() != ctx->n_mesh) ctx->mesh_inline.assign(ctx->n_mesh, kInlinePixels);
  for (int m = 0; m < ctx->n_mesh; ++m)
    if (mesh < 0 || m == mesh) ctx->mesh_inline[m] = inline_pixels;
  ctx->tables_version++;  // a captured graph holds the old launch
  return PERCH_OK;
}

extern "C" int perch_set_bin_depth(perch_ctx* ctx, int32_t mesh, int32_t depth) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (depth != 32 && depth != 64 && depth != 128) return ctx->fail(PERCH_E_ARG, "bin depth must be 32, 64 or 128");
  if (mesh < -1 || mesh >= ctx->n_mesh) return ctx->fail(PERCH_E_ARG, "mesh %d out of range", mesh);
  if ((int)ctx->mesh_queue.size() != ctx->n_mesh) ctx->mesh_queue.assign(ctx->n_mesh, kBigQueue);
  for (int m = 0; m < ctx->n_mesh; ++m)
    if (mesh < 0 || m == mesh) ctx->mesh_queue[m] = depth;
  ctx->tables_version++;  // a captured graph holds the old launch
  return PERCH_OK;
}

extern "C" int perch_set_cost_stages(perch_ctx* ctx, int32_t mesh, int32_t stages) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (stages != 1 && stages != 2) return ctx->fail(PERCH_E_ARG, "cost stages must be 1 or 2");
  if (mesh < -1 || mesh >= ctx->n_mesh) return ctx->fail(PERCH_E_ARG, "mesh %d out of range", mesh);
  if ((int)ctx->mesh_cost_stages.size() != ctx->n_mesh) ctx->mesh_cost_stages.assign(ctx->n_mesh, 1);
  for (int m = 0; m < ctx->n_mesh; ++m)
    if (mesh < 0 || m == mesh) ctx->mesh_cost_stages[m] = stages;
  ctx->tables_version++;  // a captured graph holds the old launch
  return PERCH_OK;
}

extern "C" int perch_launch_cost_stages(perch_ctx* ctx, int32_t* stages) {
  if (!ctx || !stages) return PERCH_E_ARG;
  ctx->err.clear();
  if ((int)ctx->mesh_cost_stages.size() != ctx->n_mesh) return ctx->fail(PERCH_E_STATE, "no geometry yet");
  for (int m = 0; m < ctx->n_mesh; ++m)
    stages[m] = ctx->mesh_cost_stages[m] == 2 &&
                        cost_stages_fit(ctx->device, ctx->mesh_tile_w[m], ctx->mesh_tile_h[m], 2)
                    ? 2
                    : 1;
  return PERCH_OK;
}

extern "C" int perch_launch_bin_depths(perch_ctx* ctx, int32_t* depths) {
  if (!ctx || !depths) return PERCH_E_ARG;
  ctx->err.clear();
  if ((int)ctx->mesh_queue.size() != ctx->n_mesh) return ctx->fail(PERCH_E_STATE, "no geometry yet");
  for (int m = 0; m < ctx->n_mesh; ++m) depths[m] = ctx->mesh_queue[m];
  return PERCH_OK;
}

extern "C" int perch_set_threads(perch_ctx* ctx, int32_t mesh, int32_t threads) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (threads != 128 && threads != 256 && threads != 512)
    return ctx->fail(PERCH_E_ARG, "threads must be 128, 256 or 512");
  if (mesh < -1 || mesh >= ctx->n_mesh) return ctx->fail(PERCH_E_ARG, "mesh %d out of range", mesh);
  if ((int)ctx->mesh_threads.size() != ctx->n_mesh) ctx->mesh_threads.assign(ctx->n_mesh, 256);
  for (int m = 0; m < ctx->n_mesh; ++m)
    if (mesh < 0 || m == mesh) ctx->mesh_threads[m] = threads;
  ctx->tables_version++;  // a captured graph holds the old widths
  return PERCH_OK;
}
