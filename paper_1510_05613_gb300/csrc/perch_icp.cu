// ICP refinement of successors (include/perch.h: perch_icp_refine): the
// observed cloud's world-frame grid, the parents' renders and the batch
// launch of k_icp.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "perch_ctx.h"

using namespace perch;

#define CK(expr, what)                 \
  do {                                 \
    int rc_ = ctx->cuda((expr), what); \
    if (rc_ != PERCH_OK) return rc_;   \
  } while (0)

static float icp_ordered_to_float(int i) {
  int b = i >= 0 ? i : i ^ 0x7fffffff;
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

// Bucket scene 0's observed world points by a 3D grid of cells of half the
// radius (at least 2.5 mm), grown by 1.25 until it has at most 16M cells.
// The kernel scans the cells that meet its search cube, found with the same
// monotone cell function, so any cell size gives the exact nearest point;
// half the radius keeps the scanned volume close to the search ball.
int perch_ctx::ensure_icp_grid(float radius) {
  perch_ctx* ctx = this;
  if (icp_serial == obs_serial && icp_radius == radius) return PERCH_OK;
  const SceneBufs& sc = scenes[0];
  const int n = sc.idx.n;
  CK(icp_src.ensure(16 * (size_t)std::max(n, 1)), "alloc");
  CK(icp_pts.ensure(16 * (size_t)std::max(n, 1)), "alloc");
  CK(scratch_small.ensure(64), "alloc");
  IcpGrid q{};
  q.pts = icp_pts.as<float4>();
  if (n == 0) {  // one empty cell
    CK(icp_start.ensure(8), "alloc");
    CK(cudaMemsetAsync(icp_start.p, 0, 8, stream), "memset");
    q.start = icp_start.as<int>();
    q.inv = 1.0f;
    q.nx = q.ny = q.nz = 1;
  } else {
    int binit[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    int* bounds = scratch_small.as<int>();
    CK(cudaMemcpyAsync(bounds, binit, sizeof binit, cudaMemcpyHostToDevice, stream), "copy");
    CK(launch_icp_points(sc.world2.as<float4>(), sc.cam2.as<float4>(), n, icp_src.as<float4>(), bounds, stream),
       "icp points kernel");
    int hb[6];
    CK(cudaMemcpyAsync(hb, bounds, sizeof hb, cudaMemcpyDeviceToHost, stream), "copy");
    CK(cudaStreamSynchronize(stream), "icp bounds");
    float lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = icp_ordered_to_float(hb[k]);
      hi[k] = icp_ordered_to_float(hb[3 + k]);
    }
    double h = std::max(0.5 * (double)radius, 0.0025);
    long long cells;
    int dims[3];
    for (;;) {
      cells = 1;
      for (int k = 0; k < 3; ++k) {
        dims[k] = (int)std::floor(((double)hi[k] - lo[k]) / h) + 3;
        cells *= dims[k];
      }
      if (cells <= (16LL << 20)) break;
      h *= 1.25;
    }
    q.gx = (float)(lo[0] - h);
    q.gy = (float)(lo[1] - h);
    q.gz = (float)(lo[2] - h);
    q.inv = (float)(1.0 / h);
    q.nx = dims[0];
    q.ny = dims[1];
    q.nz = dims[2];
    CK(keys.ensure(4 * (size_t)n), "alloc");
    CK(counts.ensure(4 * ((size_t)cells + 1)), "alloc");
    CK(cursor.ensure(4 * ((size_t)cells + 1)), "alloc");
    CK(icp_start.ensure(4 * ((size_t)cells + 1)), "alloc");
    CK(scan_tmp.ensure(4 * ((size_t)cells / 1024 + 2)), "alloc");
    CK(cudaMemsetAsync(counts.p, 0, 4 * (size_t)cells, stream), "memset");
    CK(launch_grid3_keys(icp_src.as<float4>(), n, q.gx, q.gy, q.gz, q.inv, q.nx, q.ny, q.nz, keys.as<int>(),
                         counts.as<int>(), stream),
       "icp grid keys");
    CK(launch_exclusive_scan(counts.as<int>(), icp_start.as<int>(), (int)cells, scan_tmp.as<int>(), stream),
       "icp scan");
    CK(cudaMemcpyAsync(cursor.p, icp_start.p, 4 * (size_t)cells, cudaMemcpyDeviceToDevice, stream), "copy");
    CK(launch_scatter(keys.as<int>(), n, cursor.as<int>(), icp_src.as<float4>(), icp_pts.as<float4>(), nullptr,
                      nullptr, stream),
       "icp scatter");
    q.start = icp_start.as<int>();
  }
  CK(cudaStreamSynchronize(stream), "icp grid");
  icp_grid = q;
  icp_serial = obs_serial;
  icp_radius = radius;
  return PERCH_OK;
}

// Render the parents into parent_z and launch k_icp over the batch (device
// arrays; enqueued on the context's stream).
int perch_ctx::enqueue_icp(const perch_obj* d_parents, int parent_stride, const int32_t* d_plen, int n_par,
                           const int32_t* d_hp, const perch_obj* d_hyp, long long n_hyp, float radius, int max_iter,
                           perch_icp* d_out) {
  perch_ctx* ctx = this;
  const size_t npx = (size_t)cam.W * cam.H;
  CK(parent_z.ensure(4 * npx * std::max(n_par, 1)), "alloc parent z-buffers");
  CK(icp_next.ensure(4), "alloc");
  // each CTA's model list and pair memory: 4 CTAs per SM at most (k_icp's registers)
  const long long prev_elems = 8LL * sm_count * tile_w * tile_h;
  CK(icp_prev.ensure(4 * (size_t)std::max(prev_elems, 1LL)), "alloc");
  Batch b;
  std::memset(&b, 0, sizeof b);
  b.parents = d_parents;
  b.parent_stride = parent_stride;
  b.parent_len = d_plen;
  b.n_par = n_par;
  b.parent_z = parent_z.as<float>();
  b.hyp_parent = d_hp;
  b.hyp = d_hyp;
  b.n_hyp = n_hyp;
  b.K_total = parent_stride + 1;  // unused by ICP
  b.tile_w = tile_w;
  b.tile_h = tile_h;
  b.wait_polls = wait_polls;
  const Geometry g = geometry();
  CK(launch_fill_u32(parent_z.as<uint32_t>(), kInfBits, (long long)npx * n_par, stream), "clear parents");
  CK(launch_render_parents(cam, g, b, max_chunks, nullptr, stream), "render parents");
  CK(cudaMemsetAsync(icp_next.p, 0, 4, stream), "memset");
  IcpWork w;
  w.r2 = (float)((double)radius * (double)radius);
  w.rwin = (float)(1.01 * (double)radius + 1e-6);
  w.max_iter = max_iter;
  w.out = d_out;
  w.prev = icp_prev.as<int>();
  CK(launch_icp(cam, g, b, icp_grid, w, prev_elems, icp_next.as<int>(), sm_count, stream), "icp kernel");
  return PERCH_OK;
}

constexpr int kNothingToDo = 1;  // icp_check_args: a valid call with no hypothesis

static int icp_check_args(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride, const int32_t* parent_len,
                          int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp, int64_t n_hyp,
                          float radius, int32_t max_iter, const perch_icp* out) {
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  if (n_hyp < 0 || n_hyp > 0x7fffffffLL) return ctx->fail(PERCH_E_ARG, "n_hyp out of range");
  if (!(radius >= 0.0f && radius <= 1.0f)) return ctx->fail(PERCH_E_ARG, "radius must lie in [0, 1] m");
  if (max_iter < 0 || max_iter > 1000) return ctx->fail(PERCH_E_ARG, "max_iter must lie in [0, 1000]");
  if (n_hyp == 0) return kNothingToDo;
  if (!parent_len || !hyp_parent || !hyp || !out || n_par < 1 || parent_stride < 0 ||
      (parent_stride > 0 && !parents))
    return ctx->fail(PERCH_E_ARG, "null pointer or bad sizes");
  if (n_par > 65535 || (long long)n_par * std::max(parent_stride, 1) > 65535)
    return ctx->fail(PERCH_E_ARG, "too many parents in one batch (n_par x stride <= 65535)");
  return PERCH_OK;
}

static int icp_obj_ok(perch_ctx* ctx, const perch_obj& o, const char* what, long long i) {
  if (o.mesh >= ctx->n_mesh || o.ix < 0 || o.ix >= ctx->nx || o.iy < 0 || o.iy >= ctx->ny || o.iyaw >= ctx->n_yaw)
    return ctx->fail(PERCH_E_ARG, "%s %lld: object (%d, %d, %d, %d) outside meshes / pose grid", what, i, o.mesh,
                     o.ix, o.iy, o.iyaw);
  return PERCH_OK;
}

extern "C" {

int perch_icp_refine(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride, const int32_t* parent_len,
                     int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp, int64_t n_hyp, float radius,
                     int32_t max_iter, perch_icp* out) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  int rc = icp_check_args(ctx, parents, parent_stride, parent_len, n_par, hyp_parent, hyp, n_hyp, radius, max_iter,
                          out);
  if (rc == kNothingToDo) return PERCH_OK;
  if (rc) return rc;
  for (int i = 0; i < n_par; ++i) {
    if (parent_len[i] < 0 || parent_len[i] > parent_stride)
      return ctx->fail(PERCH_E_ARG, "parent %d: length %d outside [0, stride]", i, parent_len[i]);
    for (int k = 0; k < parent_len[i]; ++k) {
      rc = icp_obj_ok(ctx, parents[(long long)i * parent_stride + k], "parent object", i);
      if (rc) return rc;
    }
  }
  for (long long h = 0; h < n_hyp; ++h) {
    if (hyp_parent[h] < 0 || hyp_parent[h] >= n_par)
      return ctx->fail(PERCH_E_ARG, "hypothesis %lld: parent %d out of range", h, hyp_parent[h]);
    rc = icp_obj_ok(ctx, hyp[h], "hypothesis", h);
    if (rc) return rc;
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  rc = ctx->ensure_tables();
  if (rc) return rc;
  rc = ctx->ensure_icp_grid(radius);
  if (rc) return rc;
  const size_t pbytes = sizeof(perch_obj) * std::max<size_t>((size_t)n_par * parent_stride, 1);
  CK(ctx->b_parents.ensure(pbytes), "alloc");
  CK(ctx->b_plen.ensure(4 * (size_t)n_par), "alloc");
  CK(ctx->b_hp.ensure(4 * (size_t)n_hyp), "alloc");
  CK(ctx->b_hyp.ensure(sizeof(perch_obj) * (size_t)n_hyp), "alloc");
  CK(ctx->icp_out.ensure(sizeof(perch_icp) * (size_t)n_hyp), "alloc");
  if (parent_stride > 0)
    CK(cudaMemcpyAsync(ctx->b_parents.p, parents, sizeof(perch_obj) * (size_t)n_par * parent_stride,
                       cudaMemcpyHostToDevice, ctx->stream),
       "copy parents");
  CK(cudaMemcpyAsync(ctx->b_plen.p, parent_len, 4 * (size_t)n_par, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->b_hp.p, hyp_parent, 4 * (size_t)n_hyp, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->b_hyp.p, hyp, sizeof(perch_obj) * (size_t)n_hyp, cudaMemcpyHostToDevice, ctx->stream),
     "copy");
  rc = ctx->enqueue_icp(ctx->b_parents.as<perch_obj>(), parent_stride, ctx->b_plen.as<int32_t>(), n_par,
                        ctx->b_hp.as<int32_t>(), ctx->b_hyp.as<perch_obj>(), n_hyp, radius, max_iter,
                        ctx->icp_out.as<perch_icp>());
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, ctx->icp_out.p, sizeof(perch_icp) * (size_t)n_hyp, cudaMemcpyDeviceToHost, ctx->stream),
     "copy results");
  CK(cudaStreamSynchronize(ctx->stream), "icp");
  for (long long h = 0; h < n_hyp; ++h)
    if ((uint32_t)out[h].status & (kFlagTimeout | kFlagBadIndex))
      return ctx->fail(PERCH_E_DEVICE, "ICP record %lld: %s", h,
                       ((uint32_t)out[h].status & kFlagBadIndex) ? "device index check failed"
                                                                 : "a bounded wait in the kernel gave up");
  return PERCH_OK;
}

int perch_icp_refine_dev(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                         const int32_t* parent_len, int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp,
                         int64_t n_hyp, float radius, int32_t max_iter, perch_icp* out) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  int rc = icp_check_args(ctx, parents, parent_stride, parent_len, n_par, hyp_parent, hyp, n_hyp, radius, max_iter,
                          out);
  if (rc == kNothingToDo) return PERCH_OK;
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  rc = ctx->ensure_tables();
  if (rc) return rc;
  rc = ctx->ensure_icp_grid(radius);
  if (rc) return rc;
  return ctx->enqueue_icp(parents, parent_stride, parent_len, n_par, hyp_parent, hyp, n_hyp, radius, max_iter, out);
}

}  // extern "C"
