// Internal declarations of the PERCH CUDA library (shared by its own
// translation units only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "perch.h"

namespace perch {

constexpr uint32_t kInfBits = 0x7f800000u;  // +inf: empty z-buffer pixel
constexpr uint32_t kFlagBadIndex = 0x80000000u;
constexpr uint32_t kFlagTimeout = 0x40000000u;  // a bounded wait in the kernel gave up
constexpr int kChunkMaxVerts = 512;   // vertices of one mesh chunk (10-bit local indices)
constexpr int kChunkMaxTris = 1024;   // triangles of one mesh chunk (list padded to 4 entries)
constexpr int kEvalThreads = 256;
constexpr int kEvalWarps = kEvalThreads / 32;
constexpr int kInlinePixels = 16;  // a lane tests at most this many pixel centres per triangle (k_eval;
                                   // k_render takes 8, 16 or 32 per mesh from the autotuner)
constexpr int kBigQueue = 128;     // per-chunk queue of larger triangles, shared by the CTA
constexpr int kWaitSpins = 1 << 20;  // bound on mbarrier polls before a kernel gives up
constexpr int kMaxObjectPixels = 1000;  // screen box limit that keeps edge arithmetic in int32
constexpr float kNearZ = 0.05f;    // cull: vertex depth at or below this
constexpr float kGuard = 2048.0f;  // cull: |u| or |v| beyond this (pixels)
constexpr int kMaxExtent = 16384;  // cull: snapped extent (1/16 px) at or above

// Camera constants, derived on the host from the caller's intrinsics and
// camera-to-world pose (double arithmetic, rounded once to binary32).
struct Camera {
  int W, H;
  float fx, fy, cx, cy;
  float Rcw[9], tcw[3];  // world -> camera
  float Rwc[9], twc[3];  // camera -> world
  float delta, delta2;
};

// One object type, split into chunks of <= 512 vertices / <= 1024 triangles.
struct DevMesh {
  int chunk_begin, chunk_count;
  int n_tris, n_verts;
  float vol_r2, vol_zlo, vol_zhi;  // the inscribed cylinder (also the crops' reference height)
  float lo[3], hi[3];  // object-frame bounding box
  float fp_r;          // max(largest horizontal vertex radius, V(O) radius), rounded up
  // V(O) (in_volume): kind 0 the inscribed cylinder; 1 box, p = (half x,
  // half y); 2 regular prism of vol_n <= 256 sides, p = (apothem, quick
  // accept r^2, quick reject r^2), normals at vol_normals[vol_nrm ..];
  // 3 superquadric, p = (1/a1, 1/a2, 1/a3, centre height), vol_n = exponent
  // pair (1: ellipsoid, 2: eps1 = 0.5, eps2 = 1)
  int vol_kind, vol_n, vol_nrm;
  float vol_p[4];
  float vol_z0, vol_z1;  // kinds 1 and 2: height range
  float vol_rmax;  // radius of a vertical cylinder about the origin that holds V(O)
};
constexpr int kMaxPrismSides = 256;

// Observed cloud with its two spatial indices.
struct ObsIndex {
  int n;
  // camera-frame points bucketed by a 3D grid of cell >= delta (Eq. (1) query)
  const float4* cam3;  // x, y, z, pixel index (int bits)
  const int* start3;   // n_cells3 + 1
  const uint32_t* dil3;  // bit per cell: some point in its 3x3x3 neighbourhood
  float g3x, g3y, g3z, inv3;
  int n3x, n3y, n3z;
  // the same points bucketed by a 2D world (x, y) grid (V(O) candidates)
  const float4* world2;  // x_w, y_w, z_w, -
  const float4* cam2;    // x_c, y_c, z_c, pixel index (int bits)
  const int* start2;     // n_cells2 + 1
  float g2x, g2y, inv2;
  int n2x, n2y;
  const int* sat2;       // summed-area table of points per 2D cell, (n2y + 1) x (n2x + 1)
};

struct Geometry {
  const DevMesh* meshes;
  int n_mesh;
  const int4* chunk_info;     // vertex offset, n_vtx, triangle offset, n_tri
  const uint32_t* chunk_tris; // 3 x 10-bit chunk-local vertex indices
  const float4* chunk_verts;  // object-frame positions, chunk order (all meshes)
  int n_cverts;               // length of chunk_verts
  const float4* vtab;         // per yaw: M_yaw * v for every chunk vertex (n_yaw x n_cverts)
  const float4* pose_off;     // per (ix, iy): b = R_cw (x, y, 0) + t_cw
  const float* xs;
  const float* ys;
  const float2* cs;
  int nx, ny, n_yaw;
  const int4* pose_bbox;  // per (mesh, ix, iy, iyaw): x0, y0, w, h in pixels
  const float* rx;        // ray slope per column
  const float* ry;        // ray slope per row
  const float2* vol_normals;  // face normals of the prism volumes
};

struct Batch {
  const perch_obj* parents;
  int parent_stride;
  const int32_t* parent_len;
  int n_par;
  float* parent_z;      // n_par x H x W
  int* uset;            // n_par x uset_stride indices into the 2D-sorted cloud
  int* uset_count;      // n_par
  int uset_stride;
  const int32_t* hyp_parent;
  const perch_obj* hyp;
  long long n_hyp;
  int K_total;
  perch_cost* out;
  int tile_w, tile_h;
  // several scenes in one batch (nullable: every parent in scene 0 with K_total)
  const ObsIndex* scenes;       // device array, one observation index per scene
  int n_scenes;
  const int32_t* parent_scene;  // scene of each parent
  const int32_t* parent_K;      // objects in a complete scene, per parent
  // exact shortcut (nullable): per (mesh, pose) solo pixel count and flags,
  // per parent a summed-area table of occupied 8x8-pixel tiles, per
  // hypothesis the shortcut decision, and a counter of shortcut records
  const int2* solo;
  const int* parent_sat;
  int tiles_w, tiles_h;
  uint8_t* skip;
  unsigned long long* n_short;
  // bound on the polls of the first wait for each bulk copy (kWaitSpins by
  // default); the wait that drains a copy after one gave up always uses
  // kWaitSpins
  int wait_polls;
  // depth of the render's shared bin (queue) of larger triangles, per mesh
  // (autotuned; <= 0 or above kBigQueue: kBigQueue); a triangle that finds
  // the bin full is rasterised by its own thread
  int queue_cap = 0;
};

// Shared renders (k_render, then k_cost): per-pose flags of the tile store
constexpr uint8_t kPoseCulled = 1;  // a triangle of the render was culled
constexpr uint8_t kPoseFailed = 2;  // the render's bounded wait gave up: no tile

// k_render's work: the distinct poses of a batch (pose index = ((mesh * nx +
// ix) * ny + iy) * n_yaw + iyaw), one mesh's range per launch
struct RenderWork {
  const int* gpose;     // distinct poses, in pose order
  const int* offset;    // device scalar: this launch's first entry of gpose
  const int* count;     // device scalar: its entries
  int* next;            // device counter, zero before the launch
  uint32_t* store;      // tile store: z of each pose's screen box (+inf = empty), rows of its width; for a
                        // single-scene batch the sign bit says the point is explained by I (Eq. (1))
  const int* tile_off;  // per pose: offset of its tile in the store, in 16-byte units
  uint8_t* pose_flags;  // per pose: kPoseCulled, kPoseFailed
  uint32_t* valid;      // render cache (or nullptr): per pose, the tag of its stored render
  uint32_t tag;         // this batch's tag, written for every pose rendered in full
  int4* tile_box;       // per pose: the stored box (x0, y0, width, height; the covered pixels' box)
};

// k_cost's work: hypotheses sorted by pose, one mesh's range per launch
struct CostWork {
  const int* order;
  const int* offset;  // device scalar
  const int* count;   // device scalar
  int* next;          // device counter, zero before the launch
  const uint32_t* store;
  const int* tile_off;
  const uint8_t* pose_flags;
  const int4* tile_box;  // per pose: the stored box (k_render)
};

// Hypotheses grouped by pose; P = n_mesh x nx x ny x n_yaw. All device arrays.
struct PoseGroups {
  int* cnt;     // P: hypotheses per pose (zero again after the grouping)
  int* start;   // P + 1: exclusive scan of cnt
  int* flag;    // P: cnt > 0
  int* gix;     // P + 1: exclusive scan of flag
  int* gpose;   // P: the distinct poses, in pose order
  int* tmp;     // P / 1024 + 2: scan scratch
  int* ranges;  // 4 per mesh: first hypothesis in order, hypotheses, first entry of gpose, entries
  int* order;   // n_hyp: hypotheses sorted by pose
};

// ICP refinement (k_icp): the observed cloud's world points bucketed by a
// 3D grid; cell (ix, iy, iz) is key (iz ny + iy) nx + ix, so the cells of a
// row in x are one contiguous range of pts
struct IcpGrid {
  const float4* pts;  // world x, y, z; w = the point's index in I (pixel order, int bits)
  const int* start;   // cells + 1
  float gx, gy, gz, inv;
  int nx, ny, nz;
};

struct IcpWork {
  float r2;      // (float)(radius^2)
  float rwin;    // 1.01 radius + 1e-6 m: the search window before a pair is known
  int max_iter;
  perch_icp* out;
  int* prev;     // per CTA, 2 tile_w x tile_h entries: the model pixels, then each one's last paired point
};

// kernels.cu launchers (all asynchronous on `s`)
cudaError_t launch_fill_u32(uint32_t* p, uint32_t v, long long n, cudaStream_t s);
cudaError_t launch_obs_count(const float* depth, int W, int H, int* block_counts, cudaStream_t s);
cudaError_t launch_exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s);
cudaError_t launch_obs_write(const float* depth, const Camera& cam, const float* rx, const float* ry,
                             const int* block_offsets, float4* cam_pts, float4* world_pts,
                             int* bounds, cudaStream_t s);
cudaError_t launch_grid3_keys(const float4* cam_pts, int n, float g3x, float g3y, float g3z, float inv3,
                              int n3x, int n3y, int n3z, int* keys, int* counts, cudaStream_t s);
cudaError_t launch_grid2_keys(const float4* world_pts, int n, float g2x, float g2y, float inv2,
                              int n2x, int n2y, int* keys, int* counts, cudaStream_t s);
cudaError_t launch_scatter(const int* keys, int n, int* cursor, const float4* a_in, float4* a_out,
                           const float4* b_in, float4* b_out, cudaStream_t s);
cudaError_t launch_rays(const Camera& cam, float* rx, float* ry, cudaStream_t s);
cudaError_t launch_dilate3(const int* start3, int n3x, int n3y, int n3z, uint32_t* dil3, cudaStream_t s);
cudaError_t launch_pose_tables(const Camera& cam, const Geometry& g, float* yaw_mats, float4* pose_off,
                               float4* vtab, cudaStream_t s);
cudaError_t launch_pose_bbox(const Camera& cam, const Geometry& g, const float* yaw_mats, int4* bbox,
                             int* max_wh, int* bad, cudaStream_t s);
cudaError_t launch_render_parents(const Camera& cam, const Geometry& g, const Batch& b, int max_chunks,
                                  unsigned long long* culled, cudaStream_t s);
cudaError_t launch_uset(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                        cudaStream_t s);
cudaError_t launch_group_by_mesh(const perch_obj* hyp, long long n, int n_mesh, int* hist, int* offsets,
                                 int* cursor, int* order, int* scan_tmp, cudaStream_t s,
                                 const uint8_t* skip = nullptr);
// exact shortcut (see k_shortcut)
cudaError_t launch_grid2_sat(const int* start2, int n2x, int n2y, int* counts, int* sat, cudaStream_t s);
cudaError_t launch_parent_tiles(const Camera& cam, const Batch& b, int* counts, int* sat, cudaStream_t s);
cudaError_t launch_shortcut(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                            cudaStream_t s);
cudaError_t launch_solo_pack(const perch_cost* rec, long long n, int2* solo, cudaStream_t s);
cudaError_t launch_eval_group(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                              const int* order, const int* offset, const int* count, int* next, long long max_items,
                              int threads, int sm_count, cudaStream_t s);
size_t eval_smem_bytes(int tile_w, int tile_h);
size_t render_smem_bytes(int tile_w, int tile_h);
size_t cost_smem_bytes(int tile_w, int tile_h, int stages);
// per pose: its tile's size in 16-byte units (screen box area rounded up to 4
// pixels), exclusive scan into tile_off[P + 1]
cudaError_t launch_tile_offsets(const Geometry& g, int* sizes, int* tile_off, int* tmp, cudaStream_t s);
// hypotheses of the batch grouped by pose; writes the bad-index record of a
// hypothesis with an out-of-range parent or pose (it joins no group) and
// leaves out those the shortcut answered (b.skip)
cudaError_t launch_group_by_pose(const Geometry& g, const Batch& b, const PoseGroups& pg, const uint32_t* valid,
                                 uint32_t tag, cudaStream_t s);
cudaError_t launch_render_group(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                                const RenderWork& w, long long max_items, int threads, int inline_px,
                                int sm_count, cudaStream_t s);
cudaError_t launch_cost_group(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                              const CostWork& w, long long max_items, int threads, int stages, int sm_count,
                              cudaStream_t s);
bool cost_stages_fit(int device, int tile_w, int tile_h, int stages);
// loads the kernels the allocation-free evaluation launches (a lazily loaded
// module or function would otherwise be loaded, and may allocate, at its
// first launch)
cudaError_t preload_eval_kernels();
bool eval_tile_fits(int device, int tile_w, int tile_h);
// ICP: the observed world points with their pixel index, and their bounds
// (ordered ints: x, y, z min, then x, y, z max)
cudaError_t launch_icp_points(const float4* world2, const float4* cam2, int n, float4* pts, int* bounds,
                              cudaStream_t s);
// ICP of each hypothesis of the batch (one CTA per hypothesis at a time,
// claimed from the device counter `next`, zero before the launch; the
// parents' renders must be in b.parent_z). The grid is capped so that every
// CTA has its 2 tile_w x tile_h slice of w.prev (prev_elems entries in all).
cudaError_t launch_icp(const Camera& cam, const Geometry& g, const Batch& b, const IcpGrid& q, const IcpWork& w,
                       long long prev_elems, int* next, int sm_count, cudaStream_t s);

}  // namespace perch
