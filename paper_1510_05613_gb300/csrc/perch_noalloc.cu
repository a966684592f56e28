// perch_eval_successors_noalloc: successor evaluation whose scratch memory
// (the parent z-buffers and the residual sets) lives in one fixed device
// array compiled into the library, so the call itself allocates nothing.
//
// Some callers cannot allocate device memory at the moment they evaluate
// successors: a real-time perception loop that must not stall on
// cudaMalloc/cudaFree (which can synchronise the device), or a host process
// whose GPU memory is handed out once at start-up by its own pool and may not
// grow afterwards. They set the context up first (meshes, pose grid,
// observation) and then call this entry point with their own device buffers.
//
// The array below is held by every GPU that loads the library, until the
// process exits; every call shares it and it keeps the previous call's
// contents, so each call re-initialises what must start empty (z-buffers to
// +inf, residual-set counters to zero). Two calls whose work overlaps on the
// GPU (different streams, or two contexts on one device) race on it.
#include <cstring>
#include <mutex>

#include "perch_ctx.h"
#include "perch_internal.h"

using namespace perch;

// 8 MiB: the parent z-buffers, residual sets and their counters of one call
static constexpr size_t kNoallocBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

// Device address of the array on `device` (which must be current), resolved
// once per device.
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace

// Set-up of the allocation-free entry point on the context's device (called
// by perch_set_observation, which allocates anyway): resolves the array's
// address, which loads this file's module and with it the array, loads the
// kernels the entry point launches, and creates the timing events. After it
// the entry point only enqueues work.
int noalloc_prepare(perch_ctx* ctx) {
  void* base = nullptr;
  cudaError_t e = scratch_address(ctx->device, &base);
  if (e != cudaSuccess) return ctx->cuda(e, "cudaGetSymbolAddress(noalloc scratch)");
  e = preload_eval_kernels();
  if (e != cudaSuccess) return ctx->cuda(e, "load evaluation kernels");
  return ctx->create_events();
}

extern "C" int perch_eval_successors_noalloc(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                                             const int32_t* parent_len, int32_t n_par, const int32_t* hyp_parent,
                                             const perch_obj* hyp, int64_t n_hyp, int32_t K_total,
                                             perch_cost* out) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  if (n_hyp < 0 || n_hyp > 0x7fffffffLL) return ctx->fail(PERCH_E_ARG, "n_hyp out of range");
  if (n_hyp == 0) return PERCH_OK;
  if (!parent_len || !hyp_parent || !hyp || !out || n_par < 1 || parent_stride < 0 || K_total < 1 ||
      (parent_stride > 0 && !parents))
    return ctx->fail(PERCH_E_ARG, "null pointer or bad sizes");
  if (n_par > 65535 || (long long)n_par * (parent_stride > 0 ? parent_stride : 1) > 65535)
    return ctx->fail(PERCH_E_ARG, "too many parents in one batch (n_par x stride <= 65535)");
  const size_t npx = (size_t)ctx->cam.W * ctx->cam.H;
  const size_t n_obs = (size_t)(ctx->obs.n > 0 ? ctx->obs.n : 1);
  const size_t z_bytes = round256(4 * npx * (size_t)n_par);
  const size_t u_bytes = round256(4 * n_obs * (size_t)n_par);
  const size_t c_bytes = round256(4 * (size_t)n_par + 8);  // residual-set counters, item count and cursor
  if (z_bytes + u_bytes + c_bytes > kNoallocBytes)
    return ctx->fail(PERCH_E_RANGE,
                     "noalloc scratch: %d parents at %dx%d with %d observed points need %zu bytes, limit %zu",
                     n_par, ctx->cam.W, ctx->cam.H, ctx->obs.n, z_bytes + u_bytes + c_bytes, kNoallocBytes);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx->cuda(e, "cudaSetDevice");
  void* base = nullptr;
  e = scratch_address(ctx->device, &base);  // resolved by perch_set_observation: a table lookup here
  if (e != cudaSuccess) return ctx->cuda(e, "cudaGetSymbolAddress(noalloc scratch)");
  if (!ctx->ev[0]) return ctx->fail(PERCH_E_STATE, "noalloc: set an observation first");
  unsigned char* p = static_cast<unsigned char*>(base);
  float* parent_z = reinterpret_cast<float*>(p);
  int* uset = reinterpret_cast<int*>(p + z_bytes);
  int* uset_count = reinterpret_cast<int*>(p + z_bytes + u_bytes);
  int* item_count = uset_count + n_par;  // the evaluation's work counter pair
  int* item_next = item_count + 1;

  e = cudaEventRecord(ctx->ev[0], ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "event");
  e = launch_fill_u32(reinterpret_cast<uint32_t*>(parent_z), kInfBits, (long long)npx * n_par, ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "clear parents");
  e = cudaMemsetAsync(uset_count, 0, 4 * (size_t)n_par, ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "clear residual-set counters");
  Batch b;
  std::memset(&b, 0, sizeof b);
  b.parents = parents;
  b.parent_stride = parent_stride;
  b.parent_len = parent_len;
  b.n_par = n_par;
  b.parent_z = parent_z;
  b.uset = uset;
  b.uset_count = uset_count;
  b.uset_stride = (int)n_obs;
  b.hyp_parent = hyp_parent;
  b.hyp = hyp;
  b.n_hyp = n_hyp;
  b.K_total = K_total;
  b.out = out;
  b.tile_w = ctx->tile_w;
  b.tile_h = ctx->tile_h;
  b.wait_polls = ctx->wait_polls;
  const Geometry g = ctx->geometry();
  e = launch_render_parents(ctx->cam, g, b, ctx->max_chunks, nullptr, ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "render parents");
  e = launch_uset(ctx->cam, g, ctx->obs, b, ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "residual sets");
  e = cudaEventRecord(ctx->ev[1], ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "event");
  e = cudaEventRecord(ctx->ev[2], ctx->stream);  // no grouping: every hypothesis in one launch
  if (e != cudaSuccess) return ctx->cuda(e, "event");
  e = launch_fill_u32(reinterpret_cast<uint32_t*>(item_count), (uint32_t)n_hyp, 1, ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "item count");
  e = launch_fill_u32(reinterpret_cast<uint32_t*>(item_next), 0u, 1, ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "item cursor");
  e = launch_eval_group(ctx->cam, g, ctx->obs, b, nullptr, nullptr, item_count, item_next, n_hyp, 256,
                        ctx->sm_count, ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "eval kernel");
  e = cudaEventRecord(ctx->ev[3], ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "event");
  e = cudaEventRecord(ctx->ev[4], ctx->stream);
  if (e != cudaSuccess) return ctx->cuda(e, "event");
  ctx->timed = true;  // perch_last_timing: prep = clears, parent renders, U sets; eval = the kernel
  ctx->last_path = 1;
  return PERCH_OK;
}
