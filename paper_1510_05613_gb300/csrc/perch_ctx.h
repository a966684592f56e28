// Context object behind the opaque perch_ctx handle (library-internal).
#pragma once

#include <string>
#include <vector>

#include "perch_internal.h"

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes);  // grow-only; contents are not preserved
  // reallocations so far (every buffer of every context): a captured graph
  // is replayed only while this is unchanged, since it holds the old addresses
  static long long reallocs;
  void release();
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Arguments a captured evaluation graph was made for (all 8-byte fields: no
// padding, so keys compare with memcmp).
struct GraphKey {
  const void* parents;
  long long stride;
  const void* plen;
  long long n_par;
  const void* hp;
  const void* hyp;
  long long n_hyp;
  long long K;
  const void* out;
  const void* out_host;
  long long version;
  long long reallocs;  // DevBuf::reallocs when the graph was captured
};

// One scene's observed cloud and its indices (device buffers).
struct SceneBufs {
  DevBuf start3, start2, obs3, world2, cam2, dil3;
  DevBuf img;  // the scene's depth image (H x W, metres, 0 = no return)
  DevBuf sat2;  // summed-area table of observed points per 2D world cell
  perch::ObsIndex idx{};
  void release() {
    for (DevBuf* b : {&start3, &start2, &obs3, &world2, &cam2, &dil3, &img, &sat2}) b->release();
  }
};

struct perch_cnn;

struct perch_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;

  // object meshes, split into chunks
  int n_mesh = 0, max_chunks = 0, max_tris = 0, n_cverts = 0;
  std::vector<perch::DevMesh> h_meshes;   // as on the device (with the current V(O))
  std::vector<perch::DevMesh> base_meshes;  // as loaded (V(O) = the inscribed cylinders)
  std::vector<double> vert_r;             // largest horizontal vertex radius per mesh
  DevBuf meshes, chunk_verts, chunk_info, chunk_tris, vol_normals;

  // pose grid
  int nx = 0, ny = 0, n_yaw = 0;
  DevBuf xs, ys, cs;
  std::vector<float> h_cos_sin;  // host copy of the yaw table
  // the search's yaws per mesh: all of them, or with a rotational symmetry
  // (perch_set_symmetry) the smallest index of each class of equivalent yaws
  std::vector<int> mesh_sym;
  std::vector<std::vector<int>> search_yaws;
  void update_search_yaws();

  // camera, observation and its indices
  bool has_cam = false, has_obs = false;
  perch::Camera cam{};
  perch::ObsIndex obs{};
  DevBuf depth, rx, ry, blockcnt, blockoff, scan_tmp, cam_pts, world_pts, keys, counts, cursor;
  DevBuf scratch_small;
  std::vector<SceneBufs> scenes;  // scene 0: perch_set_observation; others: perch_set_scene
  DevBuf d_scenes;                // ObsIndex per scene
  DevBuf d_scene_img;             // const float* per scene: its depth image
  int max_obs = 0;                // largest cloud over the scenes

  // camera-frame pose tables and the screen box of every (mesh, pose)
  DevBuf yaw_mats, pose_off, vtab, pose_bbox;
  bool tables_valid = false;
  int tile_w = 0, tile_h = 0;             // largest over all meshes
  std::vector<int> mesh_tile_w, mesh_tile_h;  // per mesh
  std::vector<int> mesh_threads;          // CTA width per mesh (autotuned; 256 by default)
  int sm_count = 0;

  // per-batch buffers
  DevBuf parent_z, uset, uset_count;
  DevBuf g_hist, g_off, g_cursor, g_order, g_next;  // hypotheses grouped by mesh

  // shared renders (perch_set_share_renders, on by default): the tile store
  // holds one render per pose, indexed by pose; it is sized once per
  // geometry and camera (tile_off, built with the pose boxes). Without room
  // for it, or with sharing off, every hypothesis is rendered by k_eval.
  bool share_renders = true;
  bool store_ok = false;
  DevBuf tile_store, tile_off, tile_sizes, pose_flags, tile_box;
  DevBuf pg_cnt, pg_start, pg_flag, pg_gix, pg_gpose, pg_tmp, pg_ranges;  // hypotheses grouped by pose
  std::vector<int> mesh_cost_threads;  // CTA width of k_cost per mesh (autotuned; 128 by default)
  std::vector<int> mesh_cost_stages;   // stage buffers of k_cost per mesh (1 or 2; autotuned; 1 by default)
  std::vector<int> mesh_inline;        // k_render's inline limit per mesh (autotuned; 16 by default)
  std::vector<int> mesh_queue;         // depth of the render's bin of larger triangles per mesh (autotuned)
  int last_path = 0;       // last evaluation: 1 = one render per hypothesis, 2 = shared renders
  // render cache (perch_set_render_cache, off by default): a pose's tile in
  // the store stays valid, with its pose flags, until the observation, the
  // scenes or the pose tables change. pose_valid[p] holds the tag it was
  // rendered under (2 render_epoch + 1 for the single-scene form with the
  // explained bit, 2 render_epoch for plain z); the grouping leaves such
  // poses out of a batch's render list
  bool render_cache = false;
  uint32_t render_epoch = 1;
  DevBuf pose_valid;
  DevBuf b_parents, b_plen, b_hp, b_hyp, b_out;

  // captured evaluation graph (perch_eval_graph); `version` changes whenever
  // the meshes, the pose grid or the observation change
  cudaGraphExec_t graph_exec = nullptr;
  GraphKey graph_key{};
  bool capturing = false;
  long long tables_version = 0;

  // exact shortcut: per (mesh, pose) solo render (pixels, cull flag), valid
  // for the geometry version and camera it was built for
  bool shortcut = true;
  bool building_solo = false;
  DevBuf solo, solo_rec, solo_hyp, solo_hp, solo_parent, ptile_counts, ptile_sat, skip, n_short;
  long long geom_version = 0, solo_version = -1;
  perch::Camera solo_cam{};
  long long last_short = 0, last_total = 0;
  bool short_counted = false;

  // learned heuristic used by the search (heuristics bit 2); not owned
  perch_cnn* net = nullptr;
  int net_candidates = 16;
  DevBuf net_crops, net_onehot, net_pred;
  double net_seconds = 0.0;            // last search: host time spent scoring the learned queue
  long long net_states = 0, net_crops_scored = 0;
  // last search: wall seconds in device evaluation calls, in absorbing their
  // records, and in selecting states and building batches (learned scoring included)
  double search_eval_seconds = 0.0, search_absorb_seconds = 0.0, search_host_seconds = 0.0;

  // ICP refinement (perch_icp_refine): scene 0's observed world points
  // bucketed by a grid of cells >= 1.05 x the radius it was built for,
  // rebuilt when the observation (obs_serial) or the radius changes
  long long obs_serial = 0, icp_serial = -1;
  float icp_radius = -1.0f;
  perch::IcpGrid icp_grid{};
  DevBuf icp_src, icp_pts, icp_start, icp_next, icp_out, icp_prev;

  // poll bound of the evaluation kernel's first wait for each bulk copy
  // (perch_set_wait_limit); the solo table always uses the default
  int wait_polls = perch::kWaitSpins;

  // events around the phases of the last evaluation: start, after parent
  // prep (and shortcut), after grouping, after the render launches (or the
  // per-hypothesis evaluation), after the cost launches
  static constexpr int kEvents = 5;
  cudaEvent_t ev[kEvents] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool timed = false;

  std::vector<DevBuf*> all_buffers() {
    return {&meshes, &chunk_verts, &chunk_info, &chunk_tris, &vol_normals, &yaw_mats, &pose_off, &vtab, &xs, &ys, &cs, &depth, &rx, &ry, &blockcnt, &blockoff,
            &scan_tmp, &cam_pts, &world_pts, &keys, &counts, &cursor, &d_scenes, &d_scene_img,
            &scratch_small, &pose_bbox, &parent_z, &uset, &uset_count, &b_parents, &b_plen, &b_hp, &b_hyp,
            &b_out, &g_hist, &g_off, &g_cursor, &g_order, &g_next, &net_crops, &net_onehot, &net_pred,
            &solo, &solo_rec, &solo_hyp, &solo_hp, &solo_parent, &ptile_counts, &ptile_sat, &skip, &n_short,
            &tile_store, &tile_off, &tile_sizes, &pose_flags, &pg_cnt, &pg_start, &pg_flag, &pg_gix, &pg_gpose,
            &pg_tmp, &pg_ranges, &pose_valid, &tile_box, &icp_src, &icp_pts, &icp_start, &icp_next,
            &icp_out, &icp_prev};
  }

  int fail(int code, const char* fmt, ...);
  // PERCH_E_DEVICE if some record of a finished host-side evaluation carries
  // kFlagTimeout or kFlagBadIndex (no cost was computed for it)
  int check_records(const perch_cost* out, long long n);
  int cuda(cudaError_t e, const char* what);
  perch::Geometry geometry() const;
  int ensure_tables();
  int ensure_tile_store();
  int create_events();
  int build_scene(int s, const float* depth_host);
  int ensure_solo();
  int ensure_icp_grid(float radius);
  int enqueue_icp(const perch_obj* d_parents, int parent_stride, const int32_t* d_plen, int n_par,
                  const int32_t* d_hp, const perch_obj* d_hyp, long long n_hyp, float radius, int max_iter,
                  perch_icp* d_out);
  int enqueue_eval(const perch_obj* d_parents, int parent_stride, const int32_t* d_plen, int n_par,
                   const int32_t* d_hp, const perch_obj* d_hyp, long long n_hyp, int K_total, perch_cost* d_out,
                   const int32_t* d_parent_scene = nullptr, const int32_t* d_parent_K = nullptr);
};

// Set-up of perch_eval_successors_noalloc on the context's device (scratch
// address, kernels, events); called by perch_set_observation.
int noalloc_prepare(perch_ctx* ctx);

// Learned heuristic: network predictions (host) for hypotheses over parents
// (host arrays as perch_cnn_crops); crops and forward pass on the device.
int net_predict(perch_ctx* ctx, perch_cnn* net, const perch_obj* parents, int parent_stride, const int32_t* plen,
                const int32_t* pscene, int n_par, const int32_t* hyp_parent, const perch_obj* hyp, long long n_hyp,
                float* pred_host);
