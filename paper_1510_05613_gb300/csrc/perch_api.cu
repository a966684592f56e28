// C-ABI entry points of the PERCH successor-evaluation library (host side).
//
// Owns the context's device memory and orchestrates the kernels in
// perch_kernels.cu. Host arithmetic that feeds the device (camera transform,
// squared thresholds) is done in double and rounded once to binary32, as the
// arithmetic contract in include/perch.h states; this file is compiled with
// -ffp-contract=off so no fused multiply-add changes those roundings.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "perch_internal.h"
#include "perch_ctx.h"

using namespace perch;

// ------------------------------------------------------------------ helpers
long long DevBuf::reallocs = 0;

cudaError_t DevBuf::ensure(size_t bytes) {
  if (bytes <= cap) return cudaSuccess;
  ++reallocs;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  size_t nb = std::max<size_t>(bytes, 256);
  cudaError_t e = cudaMalloc(&p, nb);
  if (e != cudaSuccess) {
    p = nullptr;
    return e;
  }
  cap = nb;
  return cudaSuccess;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
}

int perch_ctx::fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  err = buf;
  return code;
}

int perch_ctx::cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PERCH_OK;
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return fail(PERCH_E_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(PERCH_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int perch_ctx::check_records(const perch_cost* out, long long n) {
  long long bad = 0, first = -1;
  for (long long h = 0; h < n; ++h)
    if (out[h].flags & (kFlagTimeout | kFlagBadIndex)) {
      if (first < 0) first = h;
      ++bad;
    }
  if (!bad) return PERCH_OK;
  return fail(PERCH_E_DEVICE,
              "%lld records (the first: hypothesis %lld, flags 0x%08x) carry no cost: a bounded wait in the "
              "evaluation kernel gave up or an index was out of range",
              bad, first, out[first].flags);
}

Geometry perch_ctx::geometry() const {
  Geometry g;
  g.meshes = meshes.as<DevMesh>();
  g.n_mesh = n_mesh;
  g.chunk_info = chunk_info.as<int4>();
  g.chunk_tris = chunk_tris.as<uint32_t>();
  g.chunk_verts = chunk_verts.as<float4>();
  g.n_cverts = n_cverts;
  g.vtab = vtab.as<float4>();
  g.pose_off = pose_off.as<float4>();
  g.xs = xs.as<float>();
  g.ys = ys.as<float>();
  g.cs = cs.as<float2>();
  g.nx = nx;
  g.ny = ny;
  g.n_yaw = n_yaw;
  g.pose_bbox = pose_bbox.as<int4>();
  g.rx = rx.as<float>();
  g.ry = ry.as<float>();
  g.vol_normals = vol_normals.as<float2>();
  return g;
}

// radius of the footprint disk the exact shortcut and the dJ_o candidate
// search use: it must hold every vertex and all of V(O)
static float footprint_radius(double vert_r, double vol_rmax) {
  return (float)(std::max(vert_r, vol_rmax) * (1.0 + 1e-6)) + 1e-6f;
}

#define CK(expr, what)                          \
  do {                                          \
    int rc_ = ctx->cuda((expr), what);          \
    if (rc_ != PERCH_OK) return rc_;            \
  } while (0)

static float ordered_to_float(int i) {
  int b = i >= 0 ? i : i ^ 0x7fffffff;
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

// Camera-frame pose tables (per-yaw matrices, per-(ix, iy) offsets, per-yaw
// vertex tables) and the screen box of every (mesh, pose), which sets the
// shared-memory tile size. Rebuilt when the meshes, the pose grid or the
// camera change.
int perch_ctx::ensure_tables() {
  perch_ctx* ctx = this;
  if (tables_valid) return PERCH_OK;
  if (!has_cam || n_mesh == 0 || nx == 0) return PERCH_OK;
  const long long n = (long long)n_mesh * nx * ny * n_yaw;
  CK(yaw_mats.ensure(sizeof(float) * 9 * n_yaw), "alloc yaw matrices");
  CK(pose_off.ensure(sizeof(float4) * nx * ny), "alloc pose offsets");
  CK(vtab.ensure(sizeof(float4) * (size_t)n_yaw * n_cverts), "alloc vertex tables");
  CK(pose_bbox.ensure(sizeof(int4) * n), "alloc pose boxes");
  CK(scratch_small.ensure(64), "alloc");
  DevBuf& wh = g_cursor;  // per-mesh tile sizes (scratch until the first batch)
  CK(wh.ensure(sizeof(int) * (2 * (size_t)n_mesh + 1)), "alloc");
  int* d = wh.as<int>();
  CK(cudaMemsetAsync(d, 0, sizeof(int) * (2 * (size_t)n_mesh + 1), stream), "memset");
  const Geometry g = geometry();
  CK(launch_pose_tables(cam, g, yaw_mats.as<float>(), pose_off.as<float4>(), vtab.as<float4>(), stream),
     "pose tables kernel");
  CK(launch_pose_bbox(cam, g, yaw_mats.as<float>(), pose_bbox.as<int4>(), d, d + 2 * n_mesh, stream),
     "pose_bbox kernel");
  std::vector<int> h(2 * (size_t)n_mesh + 1);
  CK(cudaMemcpyAsync(h.data(), d, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, stream), "copy pose boxes");
  CK(cudaStreamSynchronize(stream), "pose tables sync");
  const int bad = h[2 * n_mesh];
  if (bad & 1) return fail(PERCH_E_RANGE, "a (mesh, pose) projects behind the near plane or far off-screen");
  if (bad & 2)
    return fail(PERCH_E_RANGE, "an object's screen box exceeds %d pixels (too close to the camera)", kMaxObjectPixels);
  mesh_tile_w.assign(n_mesh, 1);
  mesh_tile_h.assign(n_mesh, 1);
  tile_w = tile_h = 1;
  for (int m = 0; m < n_mesh; ++m) {
    mesh_tile_w[m] = std::max(h[2 * m], 1);
    mesh_tile_h[m] = std::max(h[2 * m + 1], 1);
    tile_w = std::max(tile_w, mesh_tile_w[m]);
    tile_h = std::max(tile_h, mesh_tile_h[m]);
  }
  if (!eval_tile_fits(device, tile_w, tile_h))
    return fail(PERCH_E_RANGE, "object screen box %dx%d does not fit in shared memory", tile_w, tile_h);
  if ((int)mesh_threads.size() != n_mesh) mesh_threads.assign(n_mesh, 256);
  if ((int)mesh_cost_threads.size() != n_mesh) mesh_cost_threads.assign(n_mesh, 128);
  if ((int)mesh_cost_stages.size() != n_mesh) mesh_cost_stages.assign(n_mesh, 1);
  if ((int)mesh_inline.size() != n_mesh) mesh_inline.assign(n_mesh, kInlinePixels);
  if ((int)mesh_queue.size() != n_mesh) mesh_queue.assign(n_mesh, kBigQueue);
  const int rc = ensure_tile_store();
  if (rc != PERCH_OK) return rc;
  tables_valid = true;
  return PERCH_OK;
}

// The tile store of shared renders: per pose, its screen box's 1/z bits
// (rows of its width, rounded up to 16 bytes), at the offsets the scan of
// the box areas gives. Left out (store_ok = false, every hypothesis rendered
// by k_eval) when the pose grid is too large for int32 offsets or the store
// would take more than a quarter of the free device memory.
int perch_ctx::ensure_tile_store() {
  perch_ctx* ctx = this;
  store_ok = false;
  const long long per_mesh = (long long)nx * ny * n_yaw, P = per_mesh * n_mesh;
  long long bound = 0;  // 16-byte units, from the per-mesh tiles (each box fits its mesh's tile)
  for (int m = 0; m < n_mesh; ++m) bound += per_mesh * (((long long)mesh_tile_w[m] * mesh_tile_h[m] + 3) / 4);
  if (P > (1LL << 28) || bound >= (1LL << 31)) return PERCH_OK;
  CK(tile_sizes.ensure(4 * (size_t)P), "alloc tile sizes");
  CK(tile_off.ensure(4 * ((size_t)P + 1)), "alloc tile offsets");
  CK(pg_tmp.ensure(4 * ((size_t)P / 1024 + 2)), "alloc");
  CK(pose_flags.ensure((size_t)P), "alloc pose flags");
  CK(tile_box.ensure(16 * (size_t)P), "alloc stored boxes");
  CK(pose_valid.ensure(4 * (size_t)P), "alloc render cache tags");
  CK(cudaMemsetAsync(pose_valid.p, 0, 4 * (size_t)P, stream), "memset");  // no tag is 0
  ++render_epoch;
  CK(launch_tile_offsets(geometry(), tile_sizes.as<int>(), tile_off.as<int>(), pg_tmp.as<int>(), stream),
     "tile offsets");
  int total = 0;
  CK(cudaMemcpyAsync(&total, tile_off.as<int>() + P, 4, cudaMemcpyDeviceToHost, stream), "copy tile total");
  CK(cudaStreamSynchronize(stream), "tile offsets");
  const size_t bytes = 16 * (size_t)std::max(total, 1);
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
  if (bytes > tile_store.cap && bytes - tile_store.cap > free_b / 4) return PERCH_OK;
  CK(tile_store.ensure(bytes), "alloc tile store");
  store_ok = true;
  return PERCH_OK;
}

int perch_ctx::create_events() {
  perch_ctx* ctx = this;
  if (!ev[0])
    for (int k = 0; k < kEvents; ++k) CK(cudaEventCreate(&ev[k]), "cudaEventCreate");
  return PERCH_OK;
}

// Observed cloud of one scene and its two indices (A0). Every scene shares
// the camera and delta of the last perch_set_observation.
int perch_ctx::build_scene(int s, const float* depth_host) {
  perch_ctx* ctx = this;
  const Camera& c = cam;
  const int W = c.W, H = c.H;
  const float delta = c.delta;
  if ((int)scenes.size() <= s) scenes.resize(s + 1);
  SceneBufs& sc = scenes[s];
  ++render_epoch;  // stored renders with the explained bit belong to the old cloud
  if (s == 0) ++obs_serial;  // the ICP grid belongs to the old cloud
  const int npx = W * H;
  const int nblk = (npx + 255) / 256;
  CK(ctx->depth.ensure(4 * (size_t)npx), "alloc depth");
  CK(ctx->blockcnt.ensure(4 * ((size_t)nblk + 1)), "alloc");
  CK(ctx->scan_tmp.ensure(4 * ((size_t)npx / 1024 + 2 + 4096)), "alloc");
  CK(ctx->cam_pts.ensure(16 * (size_t)npx), "alloc");
  CK(ctx->world_pts.ensure(16 * (size_t)npx), "alloc");
  CK(ctx->scratch_small.ensure(64), "alloc");
  CK(cudaMemcpyAsync(ctx->depth.p, depth_host, 4 * (size_t)npx, cudaMemcpyHostToDevice, ctx->stream), "copy depth");
  CK(sc.img.ensure(4 * (size_t)npx), "alloc scene image");
  CK(cudaMemcpyAsync(sc.img.p, ctx->depth.p, 4 * (size_t)npx, cudaMemcpyDeviceToDevice, ctx->stream), "copy depth");
  int binit[10] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN, INT_MAX, INT_MAX, INT_MIN, INT_MIN};
  int* bounds = ctx->scratch_small.as<int>();
  CK(cudaMemcpyAsync(bounds, binit, sizeof binit, cudaMemcpyHostToDevice, ctx->stream), "copy");
  int* offs = ctx->blockcnt.as<int>();
  CK(ctx->blockoff.ensure(4 * ((size_t)nblk + 1)), "alloc");
  CK(launch_obs_count(ctx->depth.as<float>(), W, H, offs, ctx->stream), "obs count kernel");
  CK(launch_exclusive_scan(offs, ctx->blockoff.as<int>(), nblk, ctx->scan_tmp.as<int>(), ctx->stream), "scan");
  CK(launch_obs_write(ctx->depth.as<float>(), c, ctx->rx.as<float>(), ctx->ry.as<float>(), ctx->blockoff.as<int>(),
                      ctx->cam_pts.as<float4>(), ctx->world_pts.as<float4>(), bounds, ctx->stream),
     "obs write kernel");
  int hb[11];
  CK(cudaMemcpyAsync(hb, bounds, 10 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "copy");
  CK(cudaMemcpyAsync(hb + 10, ctx->blockoff.as<int>() + nblk, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
     "copy");
  CK(cudaStreamSynchronize(ctx->stream), "observation sync");
  const int n = hb[10];
  ObsIndex& o = sc.idx;
  std::memset(&o, 0, sizeof o);
  o.n = n;
  if (n > 0) {
    float lo[3], hi[3], wlo[2], whi[2];
    for (int k = 0; k < 3; ++k) {
      lo[k] = ordered_to_float(hb[k]);
      hi[k] = ordered_to_float(hb[3 + k]);
    }
    for (int k = 0; k < 2; ++k) {
      wlo[k] = ordered_to_float(hb[6 + k]);
      whi[k] = ordered_to_float(hb[8 + k]);
    }
    // 3D camera-frame grid, cells >= 1.02 delta (Eq. (1) neighbourhood = 3x3x3)
    double h = 1.02 * (double)delta;
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
    o.g3x = (float)(lo[0] - h);
    o.g3y = (float)(lo[1] - h);
    o.g3z = (float)(lo[2] - h);
    o.inv3 = (float)(1.0 / h);
    o.n3x = dims[0];
    o.n3y = dims[1];
    o.n3z = dims[2];
    // 2D world grid for V(O) candidates
    double g2 = 0.01;
    int d2[2];
    for (;;) {
      for (int k = 0; k < 2; ++k) d2[k] = (int)std::floor(((double)whi[k] - wlo[k]) / g2) + 3;
      if ((long long)d2[0] * d2[1] <= (4LL << 20)) break;
      g2 *= 1.5;
    }
    o.g2x = (float)(wlo[0] - g2);
    o.g2y = (float)(wlo[1] - g2);
    o.inv2 = (float)(1.0 / g2);
    o.n2x = d2[0];
    o.n2y = d2[1];
    const long long c2 = (long long)d2[0] * d2[1];
    const long long cmax = std::max(cells, c2);
    CK(ctx->keys.ensure(4 * (size_t)n), "alloc");
    CK(ctx->counts.ensure(4 * ((size_t)cmax + 1)), "alloc");
    CK(ctx->cursor.ensure(4 * ((size_t)cmax + 1)), "alloc");
    CK(sc.start3.ensure(4 * ((size_t)cells + 1)), "alloc");
    CK(sc.start2.ensure(4 * ((size_t)c2 + 1)), "alloc");
    CK(sc.obs3.ensure(16 * (size_t)n), "alloc");
    CK(sc.dil3.ensure(4 * ((size_t)cells / 32 + 1)), "alloc");
    CK(sc.world2.ensure(16 * (size_t)n), "alloc");
    CK(sc.cam2.ensure(16 * (size_t)n), "alloc");
    CK(ctx->scan_tmp.ensure(4 * ((size_t)cmax / 1024 + 2)), "alloc");
    // bucket the camera-frame cloud
    CK(cudaMemsetAsync(ctx->counts.p, 0, 4 * (size_t)cells, ctx->stream), "memset");
    CK(launch_grid3_keys(ctx->cam_pts.as<float4>(), n, o.g3x, o.g3y, o.g3z, o.inv3, o.n3x, o.n3y, o.n3z,
                         ctx->keys.as<int>(), ctx->counts.as<int>(), ctx->stream), "grid3 keys");
    CK(launch_exclusive_scan(ctx->counts.as<int>(), sc.start3.as<int>(), (int)cells, ctx->scan_tmp.as<int>(),
                             ctx->stream), "scan3");
    CK(cudaMemcpyAsync(ctx->cursor.p, sc.start3.p, 4 * (size_t)cells, cudaMemcpyDeviceToDevice, ctx->stream),
       "copy");
    CK(launch_scatter(ctx->keys.as<int>(), n, ctx->cursor.as<int>(), ctx->cam_pts.as<float4>(),
                      sc.obs3.as<float4>(), nullptr, nullptr, ctx->stream), "scatter3");
    CK(cudaMemsetAsync(sc.dil3.p, 0, 4 * ((size_t)cells / 32 + 1), ctx->stream), "memset");
    CK(launch_dilate3(sc.start3.as<int>(), o.n3x, o.n3y, o.n3z, sc.dil3.as<uint32_t>(), ctx->stream),
       "dilate3");
    // bucket the world-frame cloud (with its camera-frame copy)
    CK(cudaMemsetAsync(ctx->counts.p, 0, 4 * (size_t)c2, ctx->stream), "memset");
    CK(launch_grid2_keys(ctx->world_pts.as<float4>(), n, o.g2x, o.g2y, o.inv2, o.n2x, o.n2y, ctx->keys.as<int>(),
                         ctx->counts.as<int>(), ctx->stream), "grid2 keys");
    CK(launch_exclusive_scan(ctx->counts.as<int>(), sc.start2.as<int>(), (int)c2, ctx->scan_tmp.as<int>(),
                             ctx->stream), "scan2");
    CK(cudaMemcpyAsync(ctx->cursor.p, sc.start2.p, 4 * (size_t)c2, cudaMemcpyDeviceToDevice, ctx->stream),
       "copy");
    CK(launch_scatter(ctx->keys.as<int>(), n, ctx->cursor.as<int>(), ctx->world_pts.as<float4>(),
                      sc.world2.as<float4>(), ctx->cam_pts.as<float4>(), sc.cam2.as<float4>(), ctx->stream),
       "scatter2");
    // summed-area table of points per 2D cell (the exact shortcut's emptiness test)
    CK(sc.sat2.ensure(4 * ((size_t)d2[0] + 1) * ((size_t)d2[1] + 1)), "alloc");
    CK(launch_grid2_sat(sc.start2.as<int>(), d2[0], d2[1], ctx->counts.as<int>(), sc.sat2.as<int>(), ctx->stream),
       "grid2 table");
    o.sat2 = sc.sat2.as<int>();
    o.cam3 = sc.obs3.as<float4>();
    o.start3 = sc.start3.as<int>();
    o.dil3 = sc.dil3.as<uint32_t>();
    o.world2 = sc.world2.as<float4>();
    o.cam2 = sc.cam2.as<float4>();
    o.start2 = sc.start2.as<int>();
  }
  if (s == 0) obs = sc.idx;
  // device copy of every scene's index, for batches that mix scenes
  CK(d_scenes.ensure(sizeof(ObsIndex) * scenes.size()), "alloc scene table");
  std::vector<ObsIndex> all(scenes.size());
  for (size_t k = 0; k < scenes.size(); ++k) all[k] = scenes[k].idx;
  CK(cudaMemcpyAsync(d_scenes.p, all.data(), sizeof(ObsIndex) * all.size(), cudaMemcpyHostToDevice, stream),
     "copy scene table");
  CK(d_scene_img.ensure(sizeof(float*) * scenes.size()), "alloc scene image table");
  std::vector<const float*> imgs(scenes.size());
  for (size_t k = 0; k < scenes.size(); ++k) imgs[k] = scenes[k].img.as<float>();
  CK(cudaMemcpyAsync(d_scene_img.p, imgs.data(), sizeof(float*) * imgs.size(), cudaMemcpyHostToDevice, stream),
     "copy scene image table");
  CK(cudaStreamSynchronize(stream), "scene index");
  max_obs = 0;
  for (auto& x : scenes) max_obs = std::max(max_obs, x.idx.n);
  return PERCH_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int perch_create(perch_ctx** out, int device, void* cuda_stream) {
  if (!out) return PERCH_E_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return PERCH_E_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return PERCH_E_CUDA;
  perch_ctx* ctx = new (std::nothrow) perch_ctx();
  if (!ctx) return PERCH_E_OOM;
  ctx->device = device;
  if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete ctx;
    return PERCH_E_CUDA;
  }
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return PERCH_E_CUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return PERCH_OK;
}

int perch_destroy(perch_ctx* ctx) {
  if (!ctx) return PERCH_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (DevBuf* b : ctx->all_buffers()) b->release();
  for (SceneBufs& sc : ctx->scenes) sc.release();
  for (int k = 0; k < perch_ctx::kEvents; ++k)
    if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return PERCH_OK;
}

const char* perch_last_error(const perch_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int perch_load_meshes(perch_ctx* ctx, const perch_mesh* meshes, int32_t n) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!meshes || n < 1 || n > 65535) return ctx->fail(PERCH_E_ARG, "need 1..65535 meshes, got %d", n);
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  std::vector<DevMesh> dm(n);
  std::vector<double> vert_r(n, 0.0);
  std::vector<float4> verts;
  std::vector<int4> info;
  std::vector<uint32_t> tris;
  int max_ml = 0, max_tris = 0;
  for (int i = 0; i < n; ++i) {
    const perch_mesh& m = meshes[i];
    if (!m.verts || !m.tris || m.n_verts < 3 || m.n_tris < 1)
      return ctx->fail(PERCH_E_ARG, "mesh %d: empty or null arrays", i);
    if (!(m.vol_r >= 0.0f) || !std::isfinite(m.vol_zlo) || !std::isfinite(m.vol_zhi))
      return ctx->fail(PERCH_E_ARG, "mesh %d: bad volume parameters", i);
    DevMesh& d = dm[i];
    d.n_tris = m.n_tris;
    d.n_verts = m.n_verts;
    d.vol_r2 = (float)((double)m.vol_r * (double)m.vol_r);
    d.vol_zlo = m.vol_zlo;
    d.vol_zhi = m.vol_zhi;
    for (int k = 0; k < 3; ++k) {
      d.lo[k] = INFINITY;
      d.hi[k] = -INFINITY;
    }
    double vr2 = 0.0;
    for (int v = 0; v < m.n_verts; ++v)
      vr2 = std::max(vr2, (double)m.verts[3 * v] * m.verts[3 * v] + (double)m.verts[3 * v + 1] * m.verts[3 * v + 1]);
    vert_r[i] = std::sqrt(vr2);
    d.vol_kind = 0;
    d.vol_n = 0;
    d.vol_nrm = 0;
    d.vol_z0 = d.vol_z1 = 0.0f;
    for (int k = 0; k < 4; ++k) d.vol_p[k] = 0.0f;
    d.vol_rmax = m.vol_r;
    d.fp_r = footprint_radius(vert_r[i], m.vol_r);
    for (int v = 0; v < m.n_verts; ++v)
      for (int k = 0; k < 3; ++k) {
        float x = m.verts[3 * v + k];
        if (!std::isfinite(x)) return ctx->fail(PERCH_E_ARG, "mesh %d: non-finite vertex %d", i, v);
        d.lo[k] = std::min(d.lo[k], x);
        d.hi[k] = std::max(d.hi[k], x);
      }
    // greedy chunks in triangle order: <= 1024 vertices, <= 2048 triangles
    d.chunk_begin = (int)info.size();
    std::vector<int> local(m.n_verts, -1);
    std::vector<int> cur_v;
    std::vector<uint32_t> cur_t;
    auto flush = [&]() {
      if (cur_t.empty()) return;
      int4 in = make_int4((int)verts.size(), (int)cur_v.size(), (int)tris.size(), (int)cur_t.size());
      for (int gv : cur_v) {
        verts.push_back(make_float4(m.verts[3 * gv], m.verts[3 * gv + 1], m.verts[3 * gv + 2], 0.0f));
        local[gv] = -1;
      }
      tris.insert(tris.end(), cur_t.begin(), cur_t.end());
      while (tris.size() % 4) tris.push_back(0xffffffffu);  // 16-byte aligned chunk lists (bulk copies)
      info.push_back(in);
      cur_v.clear();
      cur_t.clear();
    };
    for (int t = 0; t < m.n_tris; ++t) {
      int idx[3];
      for (int k = 0; k < 3; ++k) {
        idx[k] = m.tris[3 * t + k];
        if (idx[k] < 0 || idx[k] >= m.n_verts)
          return ctx->fail(PERCH_E_ARG, "mesh %d: triangle %d has vertex index %d out of range", i, t, idx[k]);
      }
      int need = 0;
      for (int k = 0; k < 3; ++k) {
        bool dup = false;
        for (int j = 0; j < k; ++j) dup |= idx[j] == idx[k];
        if (!dup && local[idx[k]] < 0) need++;
      }
      if ((int)cur_v.size() + need > kChunkMaxVerts || (int)cur_t.size() + 1 > kChunkMaxTris) flush();
      uint32_t pk = 0;
      for (int k = 0; k < 3; ++k) {
        if (local[idx[k]] < 0) {
          local[idx[k]] = (int)cur_v.size();
          cur_v.push_back(idx[k]);
        }
        pk |= (uint32_t)local[idx[k]] << (10 * k);
      }
      cur_t.push_back(pk);
    }
    flush();
    d.chunk_count = (int)info.size() - d.chunk_begin;
    max_ml = std::max(max_ml, d.chunk_count);
    max_tris = std::max(max_tris, m.n_tris);
  }
  CK(ctx->meshes.ensure(sizeof(DevMesh) * n), "alloc meshes");
  CK(ctx->chunk_verts.ensure(sizeof(float4) * verts.size()), "alloc chunk vertices");
  CK(ctx->chunk_info.ensure(sizeof(int4) * info.size()), "alloc chunks");
  CK(ctx->chunk_tris.ensure(sizeof(uint32_t) * tris.size()), "alloc chunk triangles");
  CK(cudaMemcpyAsync(ctx->meshes.p, dm.data(), sizeof(DevMesh) * n, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->chunk_verts.p, verts.data(), sizeof(float4) * verts.size(), cudaMemcpyHostToDevice,
                     ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->chunk_info.p, info.data(), sizeof(int4) * info.size(), cudaMemcpyHostToDevice,
                     ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->chunk_tris.p, tris.data(), sizeof(uint32_t) * tris.size(), cudaMemcpyHostToDevice,
                     ctx->stream), "copy");
  CK(cudaStreamSynchronize(ctx->stream), "load meshes");
  ctx->h_meshes = dm;
  ctx->base_meshes = dm;
  ctx->vert_r = vert_r;
  ctx->n_mesh = n;
  ctx->mesh_sym.assign(n, 1);
  ctx->update_search_yaws();
  ctx->max_chunks = max_ml;
  ctx->max_tris = max_tris;
  ctx->n_cverts = (int)verts.size();
  ctx->tables_valid = false;
  ctx->tables_version++;
  ctx->geom_version++;
  return ctx->ensure_tables();
}

// Yaw k of a mesh with rotational symmetry order s is searched only if no
// smaller index k' differs from it by a multiple of 2 pi / s (angles from the
// pose table in double, to 1e-6 of a period): the mesh turned by that
// difference is the same vertex set, so the two yaws are one pose.
void perch_ctx::update_search_yaws() {
  search_yaws.assign(n_mesh, {});
  for (int m = 0; m < n_mesh; ++m) {
    const int sym = m < (int)mesh_sym.size() ? std::max(mesh_sym[m], 1) : 1;
    for (int k = 0; k < n_yaw; ++k) {
      bool dup = false;
      for (int j : search_yaws[m]) {
        const double dk = std::atan2((double)h_cos_sin[2 * k + 1], (double)h_cos_sin[2 * k]);
        const double dj = std::atan2((double)h_cos_sin[2 * j + 1], (double)h_cos_sin[2 * j]);
        const double t = (dk - dj) * sym / (2.0 * M_PI);
        if (std::fabs(t - std::nearbyint(t)) < 1e-6) {
          dup = true;
          break;
        }
      }
      if (!dup) search_yaws[m].push_back(k);
    }
  }
}

int perch_set_symmetry(perch_ctx* ctx, const int32_t* sym, int32_t n) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (ctx->n_mesh == 0) return ctx->fail(PERCH_E_STATE, "load meshes first");
  if (sym && n != ctx->n_mesh) return ctx->fail(PERCH_E_ARG, "%d symmetry orders for %d meshes", n, ctx->n_mesh);
  for (int m = 0; sym && m < n; ++m)
    if (sym[m] < 0 || sym[m] > (1 << 20)) return ctx->fail(PERCH_E_ARG, "mesh %d: bad symmetry order %d", m, sym[m]);
  ctx->mesh_sym.assign(ctx->n_mesh, 1);
  for (int m = 0; sym && m < n; ++m) ctx->mesh_sym[m] = std::max(sym[m], 1);
  ctx->update_search_yaws();
  return PERCH_OK;
}

int perch_set_volumes(perch_ctx* ctx, const perch_volume* volumes, int32_t n) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (ctx->n_mesh == 0) return ctx->fail(PERCH_E_STATE, "load meshes first");
  if (volumes && n != ctx->n_mesh) return ctx->fail(PERCH_E_ARG, "%d volumes for %d meshes", n, ctx->n_mesh);
  std::vector<DevMesh> dm = ctx->base_meshes;
  std::vector<float2> normals;
  auto fin = [](float x) { return std::isfinite(x); };
  for (int i = 0; volumes && i < n; ++i) {
    const perch_volume& v = volumes[i];
    DevMesh& d = dm[i];
    if (v.kind == 0) continue;
    if (!fin(v.zlo) || !fin(v.zhi) || !(v.zlo <= v.zhi))
      return ctx->fail(PERCH_E_ARG, "volume %d: bad height range", i);
    double rmax = 0.0;
    if (v.kind == 1) {
      if (!(v.p[0] > 0.0f) || !(v.p[1] > 0.0f) || !fin(v.p[0]) || !fin(v.p[1]))
        return ctx->fail(PERCH_E_ARG, "volume %d: box half extents must be finite and > 0", i);
      d.vol_p[0] = v.p[0];
      d.vol_p[1] = v.p[1];
      rmax = std::hypot((double)v.p[0], (double)v.p[1]);
    } else if (v.kind == 2) {
      if (v.n < 3 || v.n > kMaxPrismSides || !v.normals)
        return ctx->fail(PERCH_E_ARG, "volume %d: a prism needs 3..%d sides and their normals", i, kMaxPrismSides);
      if (!(v.p[1] > 0.0f) || !fin(v.p[1])) return ctx->fail(PERCH_E_ARG, "volume %d: apothem must be > 0", i);
      // the quick accept / reject circles of in_volume hold for a regular polygon:
      // unit normals in order of angle, 2 pi / n apart
      const double step = 2.0 * M_PI / v.n, a0 = std::atan2((double)v.normals[1], (double)v.normals[0]);
      for (int k = 0; k < v.n; ++k) {
        const double c = v.normals[2 * k], sn = v.normals[2 * k + 1];
        const double da = std::remainder(std::atan2(sn, c) - (a0 + k * step), 2.0 * M_PI);
        if (std::fabs(std::hypot(c, sn) - 1.0) > 1e-6 || std::fabs(da) > 2e-7)
          return ctx->fail(PERCH_E_ARG, "volume %d: prism normal %d is not that of a regular %d-gon", i, k, v.n);
      }
      const double A = v.p[1], R = A / std::cos(M_PI / v.n);
      d.vol_p[0] = v.p[1];
      d.vol_p[1] = (float)(A * A * (1.0 - std::ldexp(1.0, -12)));
      d.vol_p[2] = (float)(R * R * (1.0 + std::ldexp(1.0, -12)));
      d.vol_n = v.n;
      d.vol_nrm = (int)normals.size();
      for (int k = 0; k < v.n; ++k) normals.push_back(make_float2(v.normals[2 * k], v.normals[2 * k + 1]));
      rmax = R;
    } else if (v.kind == 3) {
      if (v.n != 1 && v.n != 2) return ctx->fail(PERCH_E_ARG, "volume %d: superquadric exponent pair must be 1 or 2", i);
      for (int k = 0; k < 3; ++k)
        if (!(v.p[k] > 0.0f) || !fin(v.p[k])) return ctx->fail(PERCH_E_ARG, "volume %d: bad semi-axis", i);
      if (!fin(v.p[3])) return ctx->fail(PERCH_E_ARG, "volume %d: bad centre height", i);
      for (int k = 0; k < 3; ++k) d.vol_p[k] = (float)(1.0 / (double)v.p[k]);
      d.vol_p[3] = v.p[3];
      d.vol_n = v.n;
      rmax = std::max((double)v.p[0], (double)v.p[1]);
    } else {
      return ctx->fail(PERCH_E_ARG, "volume %d: unknown kind %d", i, v.kind);
    }
    d.vol_kind = v.kind;
    d.vol_z0 = v.zlo;
    d.vol_z1 = v.zhi;
    d.vol_rmax = (float)(rmax * (1.0 + 1e-5));
    d.fp_r = footprint_radius(ctx->vert_r[i], d.vol_rmax);
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(ctx->vol_normals.ensure(sizeof(float2) * std::max<size_t>(normals.size(), 1)), "alloc normals");
  if (!normals.empty())
    CK(cudaMemcpyAsync(ctx->vol_normals.p, normals.data(), sizeof(float2) * normals.size(), cudaMemcpyHostToDevice,
                       ctx->stream), "copy normals");
  CK(cudaMemcpyAsync(ctx->meshes.p, dm.data(), sizeof(DevMesh) * dm.size(), cudaMemcpyHostToDevice, ctx->stream),
     "copy meshes");
  CK(cudaStreamSynchronize(ctx->stream), "set volumes");
  ctx->h_meshes = dm;
  ctx->tables_version++;  // a captured graph holds the old geometry
  return PERCH_OK;
}

int perch_set_pose_grid(perch_ctx* ctx, const float* xs, int32_t nx, const float* ys, int32_t ny,
                        const float* cos_sin, int32_t n_yaw) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!xs || !ys || !cos_sin || nx < 1 || ny < 1 || n_yaw < 1 || nx > 32767 || ny > 32767 || n_yaw > 65535)
    return ctx->fail(PERCH_E_ARG, "pose grid: bad sizes %d x %d x %d", nx, ny, n_yaw);
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(ctx->xs.ensure(4 * nx), "alloc");
  CK(ctx->ys.ensure(4 * ny), "alloc");
  CK(ctx->cs.ensure(8 * n_yaw), "alloc");
  CK(cudaMemcpyAsync(ctx->xs.p, xs, 4 * nx, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->ys.p, ys, 4 * ny, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->cs.p, cos_sin, 8 * n_yaw, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaStreamSynchronize(ctx->stream), "set pose grid");
  ctx->nx = nx;
  ctx->ny = ny;
  ctx->n_yaw = n_yaw;
  ctx->h_cos_sin.assign(cos_sin, cos_sin + 2 * (size_t)n_yaw);
  ctx->update_search_yaws();
  ctx->tables_valid = false;
  ctx->tables_version++;
  ctx->geom_version++;
  return ctx->ensure_tables();
}

int perch_set_observation(perch_ctx* ctx, const float* depth, int32_t W, int32_t H, const float fxfycxcy[4],
                          const float T_world_cam[12], float delta) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!depth || !fxfycxcy || !T_world_cam || W < 1 || H < 1 || (long long)W * H > (1LL << 28))
    return ctx->fail(PERCH_E_ARG, "observation: bad image %d x %d or null pointer", W, H);
  if (!(delta > 0.0f) || !std::isfinite(delta)) return ctx->fail(PERCH_E_ARG, "delta must be finite and > 0");
  if (!(fxfycxcy[0] > 0.0f) || !(fxfycxcy[1] > 0.0f)) return ctx->fail(PERCH_E_ARG, "focal lengths must be > 0");
  if (ctx->n_mesh == 0 || ctx->nx == 0) return ctx->fail(PERCH_E_STATE, "load meshes and the pose grid first");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  ctx->has_obs = false;
  Camera& c = ctx->cam;
  c.W = W;
  c.H = H;
  c.fx = fxfycxcy[0];
  c.fy = fxfycxcy[1];
  c.cx = fxfycxcy[2];
  c.cy = fxfycxcy[3];
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) c.Rwc[r * 3 + k] = T_world_cam[r * 4 + k];
    c.twc[r] = T_world_cam[r * 4 + 3];
  }
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) c.Rcw[r * 3 + k] = c.Rwc[k * 3 + r];
    double acc = (double)c.Rwc[0 * 3 + r] * (double)c.twc[0];
    acc = acc + (double)c.Rwc[1 * 3 + r] * (double)c.twc[1];
    acc = acc + (double)c.Rwc[2 * 3 + r] * (double)c.twc[2];
    c.tcw[r] = (float)(-acc);
  }
  c.delta = delta;
  c.delta2 = (float)((double)delta * (double)delta);
  ctx->has_cam = true;
  ctx->tables_valid = false;
  ctx->tables_version++;

  CK(ctx->rx.ensure(4 * (size_t)W), "alloc");
  CK(ctx->ry.ensure(4 * (size_t)H), "alloc");
  CK(launch_rays(c, ctx->rx.as<float>(), ctx->ry.as<float>(), ctx->stream), "rays kernel");
  int brc = ctx->build_scene(0, depth);
  if (brc != PERCH_OK) return brc;
  int rc = ctx->ensure_tables();
  if (rc != PERCH_OK) return rc;
  rc = noalloc_prepare(ctx);
  if (rc != PERCH_OK) return rc;
  CK(cudaStreamSynchronize(ctx->stream), "observation index");
  ctx->has_obs = true;
  return PERCH_OK;
}

}  // extern "C"

// The exact shortcut's solo table: every (mesh, pose) evaluated once against
// an empty parent and an empty observation (its record's |dR| is then the
// number of covered pixels, its flags the cull bit). Rebuilt when the
// meshes, the pose grid or the camera (not delta or the depth) change.
int perch_ctx::ensure_solo() {
  perch_ctx* ctx = this;
  auto same_camera = [&]() {
    return solo_cam.W == cam.W && solo_cam.H == cam.H && solo_cam.fx == cam.fx && solo_cam.fy == cam.fy &&
           solo_cam.cx == cam.cx && solo_cam.cy == cam.cy && !std::memcmp(solo_cam.Rwc, cam.Rwc, sizeof cam.Rwc) &&
           !std::memcmp(solo_cam.twc, cam.twc, sizeof cam.twc);
  };
  if (solo_version == geom_version && same_camera()) return PERCH_OK;
  const long long n = (long long)n_mesh * nx * ny * n_yaw;
  std::vector<perch_obj> all((size_t)n);
  long long h = 0;
  for (int m = 0; m < n_mesh; ++m)
    for (int ix = 0; ix < nx; ++ix)
      for (int iy = 0; iy < ny; ++iy)
        for (int k = 0; k < n_yaw; ++k) all[h++] = perch_obj{(uint16_t)m, (uint16_t)k, (int16_t)ix, (int16_t)iy};
  CK(solo.ensure(sizeof(int2) * (size_t)n), "alloc solo table");
  CK(solo_rec.ensure(sizeof(perch_cost) * (size_t)n), "alloc");
  CK(solo_hyp.ensure(sizeof(perch_obj) * (size_t)n), "alloc");
  CK(solo_hp.ensure(4 * (size_t)n), "alloc");
  CK(solo_parent.ensure(16), "alloc");
  CK(cudaMemcpyAsync(solo_hyp.p, all.data(), sizeof(perch_obj) * (size_t)n, cudaMemcpyHostToDevice, stream), "copy");
  CK(cudaMemsetAsync(solo_hp.p, 0, 4 * (size_t)n, stream), "memset");
  CK(cudaMemsetAsync(solo_parent.p, 0, 16, stream), "memset");
  const ObsIndex saved = obs;
  std::memset(&obs, 0, sizeof obs);  // the empty observation
  building_solo = true;
  const int rc = enqueue_eval(solo_parent.as<perch_obj>(), 1, solo_parent.as<int32_t>() + 2, 1, solo_hp.as<int32_t>(),
                              solo_hyp.as<perch_obj>(), n, 2, solo_rec.as<perch_cost>());
  building_solo = false;
  obs = saved;
  if (rc != PERCH_OK) return rc;
  CK(launch_solo_pack(solo_rec.as<perch_cost>(), n, solo.as<int2>(), stream), "solo table");
  CK(cudaStreamSynchronize(stream), "solo table");
  solo_version = geom_version;
  solo_cam = cam;
  return PERCH_OK;
}

// Enqueue parent preparation and successor evaluation for device-resident
// batch arrays (no host synchronisation).
int perch_ctx::enqueue_eval(const perch_obj* d_parents, int parent_stride, const int32_t* d_plen, int n_par,
                            const int32_t* d_hp, const perch_obj* d_hyp, long long n_hyp, int K_total,
                            perch_cost* d_out, const int32_t* d_parent_scene, const int32_t* d_parent_K) {
  perch_ctx* ctx = this;
  bool use_short = shortcut && !building_solo && n_hyp > 0;
  if (use_short && !capturing) {
    const int rc = ensure_solo();
    if (rc != PERCH_OK) return rc;
  }
  use_short = use_short && solo_version == geom_version;  // while capturing: only with a ready table
  const size_t npx = (size_t)cam.W * cam.H;
  CK(parent_z.ensure(4 * npx * std::max(n_par, 1)), "alloc parent z-buffers");
  const int ustride = std::max(d_parent_scene ? max_obs : obs.n, 1);
  CK(uset.ensure(4 * (size_t)ustride * std::max(n_par, 1)), "alloc U sets");
  CK(uset_count.ensure(4 * (size_t)std::max(n_par, 1)), "alloc");
  Batch b;
  std::memset(&b, 0, sizeof b);
  b.parents = d_parents;
  b.parent_stride = parent_stride;
  b.parent_len = d_plen;
  b.n_par = n_par;
  b.parent_z = parent_z.as<float>();
  b.uset = uset.as<int>();
  b.uset_count = uset_count.as<int>();
  b.uset_stride = ustride;
  b.scenes = d_scenes.as<ObsIndex>();
  b.n_scenes = (int)scenes.size();
  b.parent_scene = d_parent_scene;
  b.parent_K = d_parent_K;
  b.hyp_parent = d_hp;
  b.hyp = d_hyp;
  b.n_hyp = n_hyp;
  b.K_total = K_total;
  b.out = d_out;
  b.tile_w = tile_w;
  b.tile_h = tile_h;
  b.wait_polls = building_solo ? kWaitSpins : wait_polls;
  const Geometry g = geometry();
  {
    const int rc = create_events();
    if (rc != PERCH_OK) return rc;
  }
  if (!capturing) CK(cudaEventRecord(ev[0], stream), "event");
  CK(launch_fill_u32(parent_z.as<uint32_t>(), kInfBits, (long long)npx * n_par, stream), "clear parents");
  CK(cudaMemsetAsync(uset_count.p, 0, 4 * (size_t)std::max(n_par, 1), stream), "memset");
  CK(launch_render_parents(cam, g, b, max_chunks, nullptr, stream), "render parents");
  CK(launch_uset(cam, g, obs, b, stream), "U sets");
  if (use_short) {  // records fixed by the solo render, written now and left out of the evaluation
    b.tiles_w = (cam.W + 7) / 8;
    b.tiles_h = (cam.H + 7) / 8;
    const size_t per = (size_t)b.tiles_w * b.tiles_h, per_sat = (size_t)(b.tiles_w + 1) * (b.tiles_h + 1);
    CK(ptile_counts.ensure(4 * per * std::max(n_par, 1)), "alloc");
    CK(ptile_sat.ensure(4 * per_sat * std::max(n_par, 1)), "alloc");
    CK(skip.ensure((size_t)n_hyp), "alloc");
    CK(n_short.ensure(8), "alloc");
    CK(cudaMemsetAsync(n_short.p, 0, 8, stream), "memset");
    b.solo = solo.as<int2>();
    b.parent_sat = ptile_sat.as<int>();
    b.skip = skip.as<uint8_t>();
    b.n_short = n_short.as<unsigned long long>();
    CK(launch_parent_tiles(cam, b, ptile_counts.as<int>(), ptile_sat.as<int>(), stream), "parent tiles");
    CK(launch_shortcut(cam, g, obs, b, stream), "shortcut");
  }
  short_counted = use_short;
  last_total = n_hyp;
  if (!capturing) CK(cudaEventRecord(ev[1], stream), "event");
  // a batch of one parent repeats no pose: rendering per hypothesis skips the
  // tile store's round trip
  const bool cache = render_cache && !capturing;  // a captured graph would keep one epoch's tag
  if (share_renders && store_ok && (n_par >= 2 || cache)) {
    // shared renders: group by pose; per mesh one persistent launch renders
    // its distinct poses into the tile store, then one costs its hypotheses
    const int per_mesh = nx * ny * n_yaw, P = per_mesh * n_mesh;
    CK(pg_cnt.ensure(4 * (size_t)P), "alloc");
    CK(pg_start.ensure(4 * ((size_t)P + 1)), "alloc");
    CK(pg_flag.ensure(4 * (size_t)P), "alloc");
    CK(pg_gix.ensure(4 * ((size_t)P + 1)), "alloc");
    CK(pg_gpose.ensure(4 * (size_t)P), "alloc");
    CK(pg_tmp.ensure(4 * ((size_t)P / 1024 + 2)), "alloc");
    CK(pg_ranges.ensure(16 * (size_t)n_mesh), "alloc");
    CK(g_order.ensure(sizeof(int) * (size_t)std::max(n_hyp, 1LL)), "alloc");
    CK(g_next.ensure(sizeof(int) * 2 * (size_t)n_mesh), "alloc");
    PoseGroups pg{pg_cnt.as<int>(),   pg_start.as<int>(), pg_flag.as<int>(),   pg_gix.as<int>(),
                  pg_gpose.as<int>(), pg_tmp.as<int>(),   pg_ranges.as<int>(), g_order.as<int>()};
    const uint32_t tag = 2u * render_epoch + (b.parent_scene ? 0u : 1u);
    uint32_t* valid = cache ? pose_valid.as<uint32_t>() : nullptr;
    CK(launch_group_by_pose(g, b, pg, valid, tag, stream), "group by pose");
    CK(cudaMemsetAsync(g_next.p, 0, sizeof(int) * 2 * (size_t)n_mesh, stream), "memset");
    if (!capturing) CK(cudaEventRecord(ev[2], stream), "event");
    int* rg = pg.ranges;
    for (int m = 0; m < n_mesh; ++m) {
      Batch bm = b;
      bm.tile_w = mesh_tile_w[m];
      bm.tile_h = mesh_tile_h[m];
      bm.queue_cap = mesh_queue[m];
      const RenderWork w{pg.gpose, rg + 4 * m + 2, rg + 4 * m + 3, g_next.as<int>() + m, tile_store.as<uint32_t>(),
                         tile_off.as<int>(), pose_flags.as<uint8_t>(), valid, tag, tile_box.as<int4>()};
      CK(launch_render_group(cam, g, obs, bm, w, std::min<long long>(n_hyp, per_mesh), mesh_threads[m],
                             mesh_inline[m], sm_count, stream),
         "render kernel");
    }
    if (!capturing) CK(cudaEventRecord(ev[3], stream), "event");
    for (int m = 0; m < n_mesh; ++m) {
      Batch bm = b;
      bm.tile_w = mesh_tile_w[m];
      bm.tile_h = mesh_tile_h[m];
      const CostWork c{pg.order, rg + 4 * m, rg + 4 * m + 1, g_next.as<int>() + n_mesh + m, tile_store.as<uint32_t>(),
                       tile_off.as<int>(), pose_flags.as<uint8_t>(), tile_box.as<int4>()};
      CK(launch_cost_group(cam, g, obs, bm, c, n_hyp, mesh_cost_threads[m], mesh_cost_stages[m], sm_count, stream),
         "cost kernel");
    }
    last_path = 2;
    if (!capturing) {
      CK(cudaEventRecord(ev[4], stream), "event");
      timed = true;
    }
    return PERCH_OK;
  }
  // group by mesh; one persistent launch per mesh with its own tile and CTA width
  CK(g_hist.ensure(sizeof(int) * (size_t)n_mesh), "alloc");
  CK(g_off.ensure(sizeof(int) * ((size_t)n_mesh + 1)), "alloc");
  CK(g_cursor.ensure(sizeof(int) * (2 * (size_t)n_mesh + 1)), "alloc");
  CK(g_next.ensure(sizeof(int) * (size_t)n_mesh), "alloc");
  CK(g_order.ensure(sizeof(int) * (size_t)std::max(n_hyp, 1LL)), "alloc");
  CK(scan_tmp.ensure(sizeof(int) * ((size_t)n_mesh / 1024 + 2)), "alloc");
  CK(launch_group_by_mesh(d_hyp, n_hyp, n_mesh, g_hist.as<int>(), g_off.as<int>(), g_cursor.as<int>(),
                          g_order.as<int>(), scan_tmp.as<int>(), stream, use_short ? skip.as<uint8_t>() : nullptr),
     "group by mesh");
  CK(cudaMemsetAsync(g_next.p, 0, sizeof(int) * (size_t)n_mesh, stream), "memset");
  if (!capturing) CK(cudaEventRecord(ev[2], stream), "event");
  for (int m = 0; m < n_mesh; ++m) {
    Batch bm = b;
    bm.tile_w = mesh_tile_w[m];
    bm.tile_h = mesh_tile_h[m];
    bm.queue_cap = mesh_queue[m];
    CK(launch_eval_group(cam, g, obs, bm, g_order.as<int>(), g_off.as<int>() + m, g_hist.as<int>() + m,
                         g_next.as<int>() + m, n_hyp, mesh_threads[m], sm_count, stream),
       "eval kernel");
  }
  last_path = 1;
  if (!capturing) {
    CK(cudaEventRecord(ev[3], stream), "event");
    CK(cudaEventRecord(ev[4], stream), "event");
    timed = true;
  }
  return PERCH_OK;
}

static int check_obj(perch_ctx* ctx, const perch_obj& o, const char* what, long long i) {
  if (o.mesh >= ctx->n_mesh || o.ix < 0 || o.ix >= ctx->nx || o.iy < 0 || o.iy >= ctx->ny || o.iyaw >= ctx->n_yaw)
    return ctx->fail(PERCH_E_ARG, "%s %lld: object (%d, %d, %d, %d) outside meshes / pose grid", what, i, o.mesh,
                     o.ix, o.iy, o.iyaw);
  return PERCH_OK;
}

extern "C" {

int perch_eval_successors(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride, const int32_t* parent_len,
                          int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp, int64_t n_hyp,
                          int32_t K_total, perch_cost* out) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  if (n_hyp < 0 || n_hyp > 0x7fffffffLL) return ctx->fail(PERCH_E_ARG, "n_hyp out of range");
  if (n_hyp == 0) return PERCH_OK;
  if (!parent_len || !hyp_parent || !hyp || !out || n_par < 1 || parent_stride < 0 || K_total < 1 ||
      (parent_stride > 0 && !parents))
    return ctx->fail(PERCH_E_ARG, "null pointer or bad sizes");
  if (n_par > 65535 || (long long)n_par * std::max(parent_stride, 1) > 65535)
    return ctx->fail(PERCH_E_ARG, "too many parents in one batch (n_par x stride <= 65535)");
  for (int i = 0; i < n_par; ++i) {
    if (parent_len[i] < 0 || parent_len[i] > parent_stride || parent_len[i] >= K_total)
      return ctx->fail(PERCH_E_ARG, "parent %d: length %d outside [0, min(stride, K_total - 1)]", i, parent_len[i]);
    for (int k = 0; k < parent_len[i]; ++k) {
      int rc = check_obj(ctx, parents[(long long)i * parent_stride + k], "parent object", i);
      if (rc) return rc;
    }
  }
  for (long long h = 0; h < n_hyp; ++h) {
    if (hyp_parent[h] < 0 || hyp_parent[h] >= n_par)
      return ctx->fail(PERCH_E_ARG, "hypothesis %lld: parent %d out of range", h, hyp_parent[h]);
    int rc = check_obj(ctx, hyp[h], "hypothesis", h);
    if (rc) return rc;
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t pbytes = sizeof(perch_obj) * std::max<size_t>((size_t)n_par * parent_stride, 1);
  CK(ctx->b_parents.ensure(pbytes), "alloc");
  CK(ctx->b_plen.ensure(4 * (size_t)n_par), "alloc");
  CK(ctx->b_hp.ensure(4 * (size_t)n_hyp), "alloc");
  CK(ctx->b_hyp.ensure(sizeof(perch_obj) * (size_t)n_hyp), "alloc");
  CK(ctx->b_out.ensure(sizeof(perch_cost) * (size_t)n_hyp), "alloc");
  if (parent_stride > 0)
    CK(cudaMemcpyAsync(ctx->b_parents.p, parents, sizeof(perch_obj) * (size_t)n_par * parent_stride,
                       cudaMemcpyHostToDevice, ctx->stream), "copy parents");
  CK(cudaMemcpyAsync(ctx->b_plen.p, parent_len, 4 * (size_t)n_par, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->b_hp.p, hyp_parent, 4 * (size_t)n_hyp, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->b_hyp.p, hyp, sizeof(perch_obj) * (size_t)n_hyp, cudaMemcpyHostToDevice, ctx->stream),
     "copy");
  int rc = ctx->enqueue_eval(ctx->b_parents.as<perch_obj>(), parent_stride, ctx->b_plen.as<int32_t>(), n_par,
                             ctx->b_hp.as<int32_t>(), ctx->b_hyp.as<perch_obj>(), n_hyp, K_total,
                             ctx->b_out.as<perch_cost>());
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, ctx->b_out.p, sizeof(perch_cost) * (size_t)n_hyp, cudaMemcpyDeviceToHost, ctx->stream),
     "copy results");
  CK(cudaStreamSynchronize(ctx->stream), "eval");
  return ctx->check_records(out, n_hyp);
}

int perch_eval_successors_dev(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                              const int32_t* parent_len, int32_t n_par, const int32_t* hyp_parent,
                              const perch_obj* hyp, int64_t n_hyp, int32_t K_total, perch_cost* out) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  if (n_hyp < 0 || n_hyp > 0x7fffffffLL) return ctx->fail(PERCH_E_ARG, "n_hyp out of range");
  if (n_hyp == 0) return PERCH_OK;
  if (!parent_len || !hyp_parent || !hyp || !out || n_par < 1 || parent_stride < 0 || K_total < 1 ||
      (parent_stride > 0 && !parents))
    return ctx->fail(PERCH_E_ARG, "null pointer or bad sizes");
  if (n_par > 65535 || (long long)n_par * std::max(parent_stride, 1) > 65535)
    return ctx->fail(PERCH_E_ARG, "too many parents in one batch (n_par x stride <= 65535)");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  return ctx->enqueue_eval(parents, parent_stride, parent_len, n_par, hyp_parent, hyp, n_hyp, K_total, out);
}

int perch_last_timing(perch_ctx* ctx, float* prep_ms, float* eval_ms) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->timed) return ctx->fail(PERCH_E_STATE, "no evaluation issued yet");
  CK(cudaEventSynchronize(ctx->ev[4]), "event sync");
  float a = 0.0f, b = 0.0f;
  CK(cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]), "event time");
  CK(cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[4]), "event time");
  if (prep_ms) *prep_ms = a;
  if (eval_ms) *eval_ms = b;
  return PERCH_OK;
}

int perch_last_phase_times(perch_ctx* ctx, float* ms, int32_t* shared) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->timed) return ctx->fail(PERCH_E_STATE, "no evaluation issued yet");
  CK(cudaEventSynchronize(ctx->ev[4]), "event sync");
  for (int k = 0; k < 4; ++k)
    if (ms) CK(cudaEventElapsedTime(&ms[k], ctx->ev[k], ctx->ev[k + 1]), "event time");
  if (shared) *shared = ctx->last_path == 2 ? 1 : 0;
  return PERCH_OK;
}

int perch_set_render_cache(perch_ctx* ctx, int32_t on) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  ctx->render_cache = on != 0;
  ++ctx->render_epoch;    // what the store held before is not trusted
  ctx->tables_version++;  // a captured graph holds the old path
  return PERCH_OK;
}

int perch_set_share_renders(perch_ctx* ctx, int32_t on) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  ctx->share_renders = on != 0;
  ctx->tables_version++;  // a captured graph holds the old path
  return PERCH_OK;
}

int perch_render(perch_ctx* ctx, const perch_obj* objs, int32_t n, float* depth_out, int64_t* n_culled) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_cam) return ctx->fail(PERCH_E_STATE, "set an observation (camera) first");
  if (!depth_out || n < 0 || n > 65535 || (n > 0 && !objs)) return ctx->fail(PERCH_E_ARG, "bad arguments");
  for (int i = 0; i < n; ++i) {
    int rc = check_obj(ctx, objs[i], "object", i);
    if (rc) return rc;
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t npx = (size_t)ctx->cam.W * ctx->cam.H;
  CK(ctx->parent_z.ensure(4 * npx), "alloc");
  CK(ctx->b_parents.ensure(sizeof(perch_obj) * std::max(n, 1)), "alloc");
  CK(ctx->b_plen.ensure(4), "alloc");
  CK(ctx->scratch_small.ensure(64), "alloc");
  if (n > 0)
    CK(cudaMemcpyAsync(ctx->b_parents.p, objs, sizeof(perch_obj) * n, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->b_plen.p, &n, 4, cudaMemcpyHostToDevice, ctx->stream), "copy");
  unsigned long long* culled = reinterpret_cast<unsigned long long*>(ctx->scratch_small.as<int>() + 8);
  CK(cudaMemsetAsync(culled, 0, 8, ctx->stream), "memset");
  CK(launch_fill_u32(ctx->parent_z.as<uint32_t>(), kInfBits, (long long)npx, ctx->stream), "clear");
  Batch b;
  std::memset(&b, 0, sizeof b);
  b.parents = ctx->b_parents.as<perch_obj>();
  b.parent_stride = std::max(n, 1);
  b.parent_len = ctx->b_plen.as<int32_t>();
  b.n_par = 1;
  b.parent_z = ctx->parent_z.as<float>();
  CK(launch_render_parents(ctx->cam, ctx->geometry(), b, ctx->max_chunks, culled, ctx->stream), "render");
  unsigned long long hc = 0;
  CK(cudaMemcpyAsync(depth_out, ctx->parent_z.p, 4 * npx, cudaMemcpyDeviceToHost, ctx->stream), "copy depth");
  CK(cudaMemcpyAsync(&hc, culled, 8, cudaMemcpyDeviceToHost, ctx->stream), "copy");
  CK(cudaStreamSynchronize(ctx->stream), "render");
  if (n_culled) *n_culled = (int64_t)hc;
  return PERCH_OK;
}


int perch_set_wait_limit(perch_ctx* ctx, int32_t polls) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  ctx->wait_polls = polls < 0 ? kWaitSpins : polls;
  ctx->tables_version++;  // a captured graph holds the old limit
  return PERCH_OK;
}

int perch_set_shortcut(perch_ctx* ctx, int32_t on) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  ctx->shortcut = on != 0;
  ctx->tables_version++;  // a captured graph holds the old choice
  return PERCH_OK;
}

int perch_shortcut_stats(perch_ctx* ctx, int64_t* n_short, int64_t* n_total) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  int64_t a = 0;
  if (ctx->short_counted) {
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, ctx->n_short.p, 8, cudaMemcpyDeviceToHost, ctx->stream), "copy");
    CK(cudaStreamSynchronize(ctx->stream), "shortcut stats");
    a = (int64_t)v;
  }
  if (n_short) *n_short = a;
  if (n_total) *n_total = ctx->last_total;
  return PERCH_OK;
}

int perch_set_scene(perch_ctx* ctx, int32_t scene, const float* depth) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "call perch_set_observation first (camera and delta)");
  if (!depth || scene < 0 || scene > 65535) return ctx->fail(PERCH_E_ARG, "bad scene index or null depth");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (scene == 0) {
    int rc = ctx->build_scene(0, depth);
    ctx->tables_version++;
    return rc;
  }
  for (int s = (int)ctx->scenes.size(); s < scene; ++s) {  // gaps: empty scenes
    std::vector<float> empty((size_t)ctx->cam.W * ctx->cam.H, 0.0f);
    int rc = ctx->build_scene(s, empty.data());
    if (rc != PERCH_OK) return rc;
  }
  int rc = ctx->build_scene(scene, depth);
  ctx->tables_version++;
  return rc;
}

int perch_eval_successors_multi(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                                const int32_t* parent_len, const int32_t* parent_scene, const int32_t* parent_K,
                                int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp, int64_t n_hyp,
                                perch_cost* out) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  if (n_hyp < 0 || n_hyp > 0x7fffffffLL) return ctx->fail(PERCH_E_ARG, "n_hyp out of range");
  if (n_hyp == 0) return PERCH_OK;
  if (!parent_len || !parent_scene || !parent_K || !hyp_parent || !hyp || !out || n_par < 1 || parent_stride < 0 ||
      (parent_stride > 0 && !parents))
    return ctx->fail(PERCH_E_ARG, "null pointer or bad sizes");
  if (n_par > 65535 || (long long)n_par * std::max(parent_stride, 1) > 65535)
    return ctx->fail(PERCH_E_ARG, "too many parents in one batch (n_par x stride <= 65535)");
  for (int i = 0; i < n_par; ++i) {
    if (parent_scene[i] < 0 || parent_scene[i] >= (int)ctx->scenes.size())
      return ctx->fail(PERCH_E_ARG, "parent %d: scene %d not set", i, parent_scene[i]);
    if (parent_K[i] < 1 || parent_len[i] < 0 || parent_len[i] > parent_stride || parent_len[i] >= parent_K[i])
      return ctx->fail(PERCH_E_ARG, "parent %d: length %d / K %d inconsistent", i, parent_len[i], parent_K[i]);
    for (int k = 0; k < parent_len[i]; ++k) {
      int rc = check_obj(ctx, parents[(long long)i * parent_stride + k], "parent object", i);
      if (rc) return rc;
    }
  }
  for (long long h = 0; h < n_hyp; ++h) {
    if (hyp_parent[h] < 0 || hyp_parent[h] >= n_par)
      return ctx->fail(PERCH_E_ARG, "hypothesis %lld: parent %d out of range", h, hyp_parent[h]);
    int rc = check_obj(ctx, hyp[h], "hypothesis", h);
    if (rc) return rc;
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const size_t pbytes = sizeof(perch_obj) * std::max<size_t>((size_t)n_par * parent_stride, 1);
  CK(ctx->b_parents.ensure(pbytes), "alloc");
  CK(ctx->b_plen.ensure(12 * (size_t)n_par), "alloc");  // lengths, scenes, K
  CK(ctx->b_hp.ensure(4 * (size_t)n_hyp), "alloc");
  CK(ctx->b_hyp.ensure(sizeof(perch_obj) * (size_t)n_hyp), "alloc");
  CK(ctx->b_out.ensure(sizeof(perch_cost) * (size_t)n_hyp), "alloc");
  int32_t* d_plen = ctx->b_plen.as<int32_t>();
  if (parent_stride > 0)
    CK(cudaMemcpyAsync(ctx->b_parents.p, parents, sizeof(perch_obj) * (size_t)n_par * parent_stride,
                       cudaMemcpyHostToDevice, ctx->stream), "copy parents");
  CK(cudaMemcpyAsync(d_plen, parent_len, 4 * (size_t)n_par, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(d_plen + n_par, parent_scene, 4 * (size_t)n_par, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(d_plen + 2 * n_par, parent_K, 4 * (size_t)n_par, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->b_hp.p, hyp_parent, 4 * (size_t)n_hyp, cudaMemcpyHostToDevice, ctx->stream), "copy");
  CK(cudaMemcpyAsync(ctx->b_hyp.p, hyp, sizeof(perch_obj) * (size_t)n_hyp, cudaMemcpyHostToDevice, ctx->stream),
     "copy");
  int rc = ctx->enqueue_eval(ctx->b_parents.as<perch_obj>(), parent_stride, d_plen, n_par, ctx->b_hp.as<int32_t>(),
                             ctx->b_hyp.as<perch_obj>(), n_hyp, 1, ctx->b_out.as<perch_cost>(), d_plen + n_par,
                             d_plen + 2 * n_par);
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, ctx->b_out.p, sizeof(perch_cost) * (size_t)n_hyp, cudaMemcpyDeviceToHost, ctx->stream),
     "copy results");
  CK(cudaStreamSynchronize(ctx->stream), "eval");
  return ctx->check_records(out, n_hyp);
}

}  // extern "C"
