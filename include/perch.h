/*
 * perch.h -- C ABI of the GB300 PERCH successor-evaluation library.
 *
 * PERCH (Narayanan & Likhachev, "PERCH: Perception via Search for
 * Multi-Object Recognition and Localization") localises K known objects on a
 * table by searching the Monotone Scene Generation Tree (MSGT, Sec. IV-A).
 * This library evaluates MSGT successors in bulk on one GPU: it z-buffer
 * renders each (object, x, y, yaw) hypothesis over its parent scene and counts
 * the explanation edge cost of Eq. (4). It also runs the tree search of
 * Sec. IV-B over those evaluations.
 *
 * Conventions for every entry point:
 *   - returns a perch_status (0 = PERCH_OK); never aborts or exits; the
 *     message of the last failure is available from perch_last_error();
 *   - host input buffers are owned by the caller and are copied (or fully
 *     consumed) before the call returns; nothing keeps a caller pointer;
 *   - all device memory the library allocates is owned by the context and
 *     released by perch_destroy();
 *   - a context is not thread-safe; use one context per host thread;
 *   - world frame: z up, table plane z = 0; camera frame: x right, y down,
 *     z forward (pinhole, pixel centres at integer (u, v), depth = camera Z);
 *   - all floating-point arithmetic on the evaluation path is IEEE binary32
 *     with round-to-nearest-even, in the operation order the oracle in
 *     oracle/ states; a fused multiply-add (one rounding) appears exactly
 *     where that order writes one and nowhere else, so results are bit-exact
 *     with it:
 *       vertex   c_r = fma(M_r2, v_z, fma(M_r1, v_y, M_r0 v_x)) + b_r with
 *                M = R_cw Rz(yaw) and b = R_cw (x, y, 0) + t_cw (double,
 *                rounded once); 1/z = 1 / c_z; u = fma(f_x, c_x (1/z), c_x0);
 *                snapped X = rint(16 u);
 *       depth    1/z = fma(b2, 1/z2, fma(b1, 1/z1, b0 (1/z0))), z = 1 / (1/z),
 *                b_i = (float)E_i * (1 / (float)A) from exact integer edge
 *                functions E_i and twice the area A;
 *       Eq. (1)  d^2 = fma(dz, dz, fma(dy, dy, dx dx)) <= (float)(delta^2);
 *       V(O)     fma(dy, dy, dx dx) <= (float)(r^2), z_lo <= z <= z_hi.
 */
#ifndef PERCH_H_
#define PERCH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PERCH_OK = 0,
  PERCH_E_ARG = -1,     /* invalid argument (null pointer, bad size, bad index) */
  PERCH_E_CUDA = -2,    /* a CUDA call failed; the message names it */
  PERCH_E_OOM = -3,     /* device or host allocation failed */
  PERCH_E_STATE = -4,   /* call order: meshes / pose grid / observation missing */
  PERCH_E_TIMEOUT = -5, /* search limit reached; best solution so far returned */
  PERCH_E_RANGE = -6,   /* a hypothesis does not fit the renderer's tile limit */
  PERCH_E_DEVICE = -7   /* a bounded wait in a kernel gave up (flags bit 30) or a
                           device-side index check failed (bit 31): the affected
                           records hold no cost; the context stays usable */
} perch_status;

typedef struct perch_ctx perch_ctx;

/* Triangle mesh of one object type (Sec. III: "3D models of N unique
 * objects"). Object frame: z up, base on z = 0, origin on the vertical axis the
 * yaw turns about. Triangles are counter-clockwise seen from outside. V(O),
 * the conservative object volume of Sec. III-A, is the inscribed vertical
 * cylinder of radius vol_r about the origin between heights vol_zlo..vol_zhi. */
typedef struct {
  const float* verts;   /* n_verts x 3 */
  int32_t n_verts;
  const int32_t* tris;  /* n_tris x 3 vertex indices */
  int32_t n_tris;
  float vol_r, vol_zlo, vol_zhi;
} perch_mesh;

/* V(O) of one mesh in closed form (Sec. III-A: the set of points in the
 * volume the object occupies; the inscribed cylinder of perch_mesh stands in
 * where there is no closed form), in the object frame (z up, base on z = 0,
 * yaw about the z axis):
 *   kind 0: the inscribed cylinder of perch_mesh (the default);
 *   kind 1: box |x| <= p[0], |y| <= p[1], zlo <= z <= zhi;
 *   kind 2: regular prism of n sides (3..256): normals[k] . (x, y) <= p[1]
 *           (the apothem) for every face k, zlo <= z <= zhi; normals = n
 *           (cos, sin) pairs, the unit outward face normals in order of
 *           angle, 2 pi / n apart (checked to 2e-7 rad); p[0] unused;
 *   kind 3: superquadric with semi-axes p[0..2] and centre height p[3]:
 *           n = 1: X^2 + Y^2 + Z^2 <= 1 (ellipsoid); n = 2:
 *           (X^2 + Y^2)^2 + Z^4 <= 1 (eps1 = 0.5, eps2 = 1), where
 *           X = x (1/p[0]), Y = y (1/p[1]), Z = (z - p[3]) (1/p[2]) with the
 *           reciprocals computed in double and rounded to binary32;
 *           t = fma(Y, Y, X X), F = fma(t, t, Z^2 Z^2) (n = 2) or t + Z^2.
 * A world point enters the object frame through the pose table's (c, s):
 * x = fma(s, dy, c dx), y = fma(c, dy, -(s dx)) with (dx, dy) its offset
 * from the pose's (x, y); z is its world height. */
typedef struct {
  int32_t kind;
  int32_t n;
  float p[4];
  float zlo, zhi;
  const float* normals; /* kind 2: n x 2 */
} perch_volume;

/* One object state O = (ID, x, y, theta) of Sec. III-A, as indices into the
 * pose grid: x = xs[ix], y = ys[iy], (cos, sin) = cos_sin[iyaw]. 8 bytes. */
typedef struct {
  uint16_t mesh;
  uint16_t iyaw;
  int16_t ix, iy;
} perch_obj;

/* Result for one successor (28 bytes). For a valid child (viol == 0) the edge
 * cost of Eq. (4) is djr + djo + resid:
 *   djr   = #{p in dR unexplained by I}             (Sec. IV-A, dJ_r)
 *   djo   = #{q in I n V(O) unexplained by dR}       (Sec. IV-A, dJ_o)
 *   resid = #{q in I - V_K unexplained by R_K} on edges into level K, else 0
 *   viol  = #{pixels where the child lies strictly in front of the parent};
 *           viol > 0 means the child breaks R_{j} subset R_{j+1} (Eq. (3)) and
 *           is not a successor: its cost fields are then 0
 *   n_new = |dR|, the child's pixels where the parent render is empty
 *   flags = bit 0: a triangle of the child was culled (near plane / guard
 *           band); bit 1: invalid (viol > 0); bit 30: a bounded wait of the
 *           evaluation kernel for one of its bulk copies gave up, so no cost
 *           was computed (every other field is 0); bit 31: a parent or pose
 *           index was out of range (device-pointer calls only; other fields 0).
 *           The host-pointer calls and the search return PERCH_E_DEVICE when
 *           any record carries bit 30 or 31
 *   n_vol = #{q in I n V(O) outside every parent object's volume}: how much
 *           the overlap heuristic h_overlap of Sec. IV-C (observed points
 *           outside the assigned volumes) drops from parent to child; 0 when
 *           viol > 0. */
typedef struct {
  int32_t djr, djo, resid, viol, n_new;
  uint32_t flags;
  int32_t n_vol;
} perch_cost;

#define PERCH_FLAG_CULLED 1u
#define PERCH_FLAG_INVALID 2u

/* Create a context on CUDA device `device`. `cuda_stream` (a cudaStream_t,
 * may be NULL) is the stream all work is issued on; with NULL the context
 * creates and owns a non-blocking stream. */
int perch_create(perch_ctx** out, int device, void* cuda_stream);

/* Release every device buffer and the owned stream. NULL is accepted. */
int perch_destroy(perch_ctx* ctx);

/* Message of the last failing call on this context ("" if none). The string
 * stays valid until the next call on the context. */
const char* perch_last_error(const perch_ctx* ctx);

/* Upload n object meshes (Sec. III: the known 3D models). Replaces any
 * previous meshes. Meshes are split into chunks on the host (at most 512
 * vertices and 1024 triangles each). Errors: PERCH_E_ARG for empty meshes,
 * out-of-range indices or n < 1. */
int perch_load_meshes(perch_ctx* ctx, const perch_mesh* meshes, int32_t n);

/* V(O) of every mesh (volumes[n], n = the number of meshes loaded), used by
 * dJ_o, the residual and n_vol from the next evaluation on; volumes = NULL
 * restores the inscribed cylinders. Copied. perch_load_meshes resets to the
 * cylinders. PERCH_E_ARG for a bad kind, side count, normal table or
 * parameter; PERCH_E_STATE before perch_load_meshes. */
int perch_set_volumes(perch_ctx* ctx, const perch_volume* volumes, int32_t n);

/* Rotational symmetry of the meshes for the search (Sec. IV-E: for a
 * rotationally symmetric object only (x, y) matters): sym[m] = s means mesh m
 * is the same vertex set after a turn of 2 pi / s about its vertical axis
 * (1 = no symmetry). The search then places mesh m only at the yaws of the
 * pose grid that no smaller yaw index equals modulo 2 pi / s (compared in
 * double from the yaw table), which removes the other yaws of each
 * equivalence class from the tree: the returned scene is the optimum of that
 * smaller tree (a rotated mesh's binary32 vertices, hence its render, can
 * differ in the last bit). sym = NULL: no symmetry (the default, also after
 * perch_load_meshes). Evaluation calls are unaffected. */
int perch_set_symmetry(perch_ctx* ctx, const int32_t* sym, int32_t n);

/* Discretised 3-DoF poses (Sec. III; Sec. V-B discretises x, y and yaw):
 * xs[nx], ys[ny] in metres, cos_sin[2 * n_yaw] = (cos, sin) per yaw. The
 * tables are used as given (no trigonometry on the device). */
int perch_set_pose_grid(perch_ctx* ctx, const float* xs, int32_t nx, const float* ys,
                        int32_t ny, const float* cos_sin, int32_t n_yaw);

/* Set the observation (Sec. III: the input cloud I and the sensor pose):
 * depth[H * W] in metres, row-major, 0 (or non-finite) = missing;
 * fxfycxcy = pinhole intrinsics; T_world_cam = row-major 3x4 camera-to-world
 * transform; delta = the sensor-noise threshold of Eq. (1), in metres.
 * Builds the observed cloud and its delta-grid index on the device. Requires
 * meshes and the pose grid (PERCH_E_STATE otherwise). */
int perch_set_observation(perch_ctx* ctx, const float* depth, int32_t W, int32_t H,
                          const float fxfycxcy[4], const float T_world_cam[12], float delta);

/* Evaluate n_hyp MSGT successors (Eq. (3), Eq. (4)).
 * parents: n_par partial assignments, parent i = parents[i * parent_stride ..
 *          + parent_len[i]) (parent_len may be 0: the root);
 * hyp_parent[h] in [0, n_par): the parent hypothesis h extends;
 * hyp[h]: the object added; K_total: objects in a complete scene (the
 *          residual term is added when parent_len + 1 == K_total);
 * out[n_hyp]: results.
 * All pointers are host pointers; the call returns when out is written.
 * Errors: PERCH_E_ARG (bad index / length), PERCH_E_STATE (no observation),
 * PERCH_E_RANGE (a hypothesis larger than the tile limit). */
int perch_eval_successors(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                          const int32_t* parent_len, int32_t n_par, const int32_t* hyp_parent,
                          const perch_obj* hyp, int64_t n_hyp, int32_t K_total, perch_cost* out);

/* Same as perch_eval_successors, but parents, parent_len, hyp_parent, hyp and
 * out are DEVICE pointers (e.g. torch tensors on the context's device) and
 * the work is only enqueued on the context's stream; out is valid once that
 * stream reaches this point. Indices are not validated on the host (an
 * out-of-range parent or pose index sets bit 31 in that record's flags and
 * zeroes the rest); a record whose bounded wait gave up carries bit 30. */
int perch_eval_successors_dev(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                              const int32_t* parent_len, int32_t n_par, const int32_t* hyp_parent,
                              const perch_obj* hyp, int64_t n_hyp, int32_t K_total, perch_cost* out);

/* Same work and arguments as perch_eval_successors_dev (device pointers,
 * enqueued on the context's stream), but the call allocates no memory: its
 * scratch (parent z-buffers, residual sets) is a fixed 8 MiB device array
 * compiled into the library. The paper has no counterpart; this serves
 * callers that cannot allocate device memory when they evaluate (a real-time
 * loop that must not stall on cudaMalloc/cudaFree, or a process whose GPU
 * memory is fixed by its own pool after start-up). They set the context up
 * first; the set-up calls do allocate.
 * Limit: 4*n_par*W*H + 4*n_par*max(|I|,1) + 4*n_par + 8 bytes (each of the
 * three parts rounded up to 256) must not exceed 8 MiB, else PERCH_E_RANGE
 * and nothing is enqueued.
 * perch_set_observation does this entry point's own set-up, once per device:
 * it looks up the array's device address and loads the kernels the call
 * launches (either could otherwise allocate on first use); the call itself
 * then only enqueues work. Every call shares the array and re-initialises
 * it, so calls whose work overlaps on the GPU (other streams, or other
 * contexts on the same device) race; serialise them. The array is held by
 * every GPU that loads the library until the process exits. */
int perch_eval_successors_noalloc(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                                  const int32_t* parent_len, int32_t n_par, const int32_t* hyp_parent,
                                  const perch_obj* hyp, int64_t n_hyp, int32_t K_total, perch_cost* out);

/* Several scenes in one context (many independent searches at once). Every
 * scene shares the meshes, the pose grid, the camera and delta of
 * perch_set_observation, which is scene 0; this call sets (or replaces) the
 * observed depth of scene `scene` (0..65535; unset scenes in between are
 * empty). depth[H * W] as in perch_set_observation. */
int perch_set_scene(perch_ctx* ctx, int32_t scene, const float* depth);

/* perch_eval_successors for a batch that mixes scenes: parent i belongs to
 * scene parent_scene[i] and to a problem of parent_K[i] objects (the residual
 * is added on its children when parent_len[i] + 1 == parent_K[i]). Host
 * pointers; returns when out is written. */
int perch_eval_successors_multi(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                                const int32_t* parent_len, const int32_t* parent_scene, const int32_t* parent_K,
                                int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp, int64_t n_hyp,
                                perch_cost* out);

/* z-buffer render (min depth, +inf where empty) of n objects into
 * depth_out[H * W] (host pointer), the R_j of Sec. III-A. Returns the number
 * of culled triangles in *n_culled (may be NULL). */
int perch_render(perch_ctx* ctx, const perch_obj* objs, int32_t n, float* depth_out,
                 int64_t* n_culled);

/* ICP refinement of successors (Sec. IV-E-1, compensating for
 * discretization: each time a state is rendered with a new object, the
 * object's non-occluded portion is aligned with the observed cloud by ICP in
 * its local vicinity; Sec. V-B: correspondences only within 2 cm, half the
 * grid step). The paper leaves the variant open; this one is fixed step by
 * step, in exact arithmetic where order could matter, so that every record
 * is bit-exact with the oracle:
 *   model set M: the pixels where the new object's own render z_O is finite
 *     and lies strictly in front of the parent's render z_P (+inf where
 *     empty) -- for a valid child, dR of Eq. (3) -- back-projected to the
 *     world frame as the observed cloud is;
 *   motion T = (c, s, tx, ty): a turn about the world's vertical axis and a
 *     shift in the table plane, applied in binary32 from T rounded to
 *     binary32: x' = (c x - s y) + tx, y' = (s x + c y) + ty, z' = z;
 *   correspondence of m: the observed point q of smallest
 *     d^2 = fma(dz, dz, fma(dy, dy, dx dx)) (d = T m - q, world frame) with
 *     d^2 <= (float)(radius^2); ties to the smaller index of q in I (pixel
 *     order); none: m is unmatched;
 *   sums over the pairs in fixed point (coordinates times 2^16, rounded to
 *     the nearest integer, ties to even; a pair with |x| or |y| >= 32 m is
 *     left out): n, sum X_m, sum Y_m, sum X_q, sum Y_q, sum X_m X_q,
 *     sum Y_m Y_q, sum X_m Y_q, sum Y_m X_q -- exact, in any order;
 *   fit (planar Procrustes, in closed form): with the exact integers
 *     C = n sum(m . q) - sum m . sum q and S = n sum(m x q) - sum m x sum q,
 *     each rounded to double as hi 2^64 + lo (hi, lo rounded, one rounded
 *     sum), h = sqrt(C^2 + S^2), c = C / h, s = S / h,
 *     tx = ((sum X_q - (c sum X_m - s sum Y_m)) / n) 2^-16, ty likewise with
 *     (s sum X_m + c sum Y_m) (double, each operation rounded once);
 *   iteration k = 1 .. max_iter from T = identity: match under T; fewer than
 *     3 pairs: stop (PERCH_ICP_FEW); the same sums as at k - 1: stop
 *     (PERCH_ICP_CONVERGED); C = S = 0: stop (PERCH_ICP_DEGENERATE); else T =
 *     the fit. After max_iter fits: PERCH_ICP_CAP.
 * The refined pose of the object at grid pose (x, y, yaw) is
 * (c x - s y + tx, s x + c y + ty, yaw + atan2(s, c)). The search itself
 * keeps the grid poses (its costs, renders and parity stay those of the
 * grid MSGT); this call refines any batch of successors, such as the
 * objects of a returned scene, each against the state it was added to. */
typedef struct {
  double c, s, tx, ty;  /* the motion T */
  int32_t n_model;      /* |M| */
  int32_t n_corr;       /* pairs of the last matching */
  int32_t iters;        /* fits made */
  int32_t status;       /* PERCH_ICP_*, or flags bit 30 / bit 31 as in perch_cost */
} perch_icp;            /* 48 bytes */

enum { PERCH_ICP_CONVERGED = 0, PERCH_ICP_CAP = 1, PERCH_ICP_FEW = 2, PERCH_ICP_DEGENERATE = 3 };

/* Refine n_hyp successors against the observation of perch_set_observation
 * (scene 0). parents, parent_stride, parent_len, n_par, hyp_parent, hyp as
 * in perch_eval_successors (parent_len[i] <= parent_stride; no K_total);
 * radius: the correspondence distance in metres (>= 0, finite); max_iter:
 * the most fits per successor (0 .. 1000); out[n_hyp]. Host pointers; the
 * call returns when out is written. Errors: PERCH_E_ARG (bad index, length,
 * radius or max_iter), PERCH_E_STATE (no observation), PERCH_E_DEVICE (a
 * record with bit 30 or 31). The first call after an observation builds
 * the cloud's world-frame grid of cells >= 1.05 radius (one more set of
 * device buffers, held by the context). */
int perch_icp_refine(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride, const int32_t* parent_len,
                     int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp, int64_t n_hyp, float radius,
                     int32_t max_iter, perch_icp* out);

/* Same, with parents, parent_len, hyp_parent, hyp and out as DEVICE pointers;
 * the work is only enqueued on the context's stream (the grid, if it must
 * be built, is built first, synchronously). Indices are checked on the
 * device: a bad one gives a record with status bit 31 and the rest zero. */
int perch_icp_refine_dev(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride,
                         const int32_t* parent_len, int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp,
                         int64_t n_hyp, float radius, int32_t max_iter, perch_icp* out);

/* Tree search (Sec. IV-B, Alg. 1). With w = 1 and no heuristics:
 * uniform-cost search (A* with the admissible h0 = 0), which returns an
 * optimal scene. Otherwise Focal-MHA*: the anchor queue is keyed by g + h0,
 * states with g <= w * (smallest anchor key) are also expanded greedily by
 * each inadmissible heuristic in `heuristics` (bit 0: h_depth = K - |s|;
 * bit 1: h_overlap = observed points outside the assigned volumes,
 * Sec. IV-C; bits 2 and 3, exclusive: the learned heuristic of
 * perch_set_heuristic_net, PERCH_E_STATE without a network. Each expansion
 * keeps the n_candidates cheapest valid placements of every remaining type.
 * A child s' gets h_free = the sum over its remaining objects of their
 * cheapest exact costs at the parent, and h_cnn = the sum over its remaining
 * objects of the smallest predicted edge cost exp(y) - 1 among the parent's
 * candidates of that type, predicted with s' as parent. Each round the
 * learned queue takes a pool of its front states (max(16, 2 batch_states)),
 * scores them, expands the best batch_states and returns the rest. Bit 2:
 * the queue is ordered by g + h_free across depths (ties: deeper first) and
 * the pool expanded in order of g + h_cnn. Bit 3: the queue is ordered
 * deepest first, then by g + h_free, and the pool re-ranked by g + h_cnn
 * within each depth), and the search returns a scene of cost <= w * OPT
 * (Theorem 2). Bit 4 (with any of the above or none; not in the paper): an
 * incumbent first. A greedy completion from the root expands, one state per
 * round, the cheapest valid child of the state it expanded last, down to a
 * goal; that goal is the first best goal, so every later successor dearer
 * than it is dropped as its record arrives instead of entering the open
 * set. With w = 1 the returned scene is the same as without bit 4 (the
 * optimum, ties broken by the smallest sorted key); with w > 1 it stays
 * within w * OPT. The open set, host memory and time shrink. mesh_multiset[K]: the types of the K objects (Sec. III: known
 * number and types). batch_states: states taken from each queue per device
 * launch (>= 1). Stops at the optimum / the bound, or at time_limit_s /
 * max_expansions (0 = none) and then returns PERCH_E_TIMEOUT with the best
 * goal found so far (or cost -1 if none). */
typedef struct {
  int32_t K;
  const uint16_t* mesh_multiset;
  float w;
  int32_t batch_states;
  double time_limit_s;
  int64_t max_expansions;
  int32_t heuristics;
} perch_search_params;

typedef struct {
  perch_obj objs[16];   /* the goal state, sorted by (mesh, ix, iy, iyaw) */
  int32_t n_objs;
  int64_t cost;         /* sum of edge costs along the returned path */
  int64_t expansions;   /* states expanded */
  int64_t successors;   /* hypotheses evaluated */
  double seconds;
  int32_t proven_optimal;
  double found_seconds;     /* when the returned scene was first found (its records absorbed) */
  int64_t found_expansions; /* states expanded by then */
} perch_result;

int perch_search(perch_ctx* ctx, const perch_search_params* params, perch_result* result);

/* One search per scene (scenes[i] with params[i]), run together: the
 * expansions of every unfinished search are packed into shared evaluation
 * launches of at most max_hyps_per_launch hypotheses (at least one state's
 * children). results[i].seconds is the time from the start until search i
 * finished (its time to the optimum). Limits as perch_search, taken as the
 * largest over params. */
int perch_search_multi(perch_ctx* ctx, int32_t n_scenes, const int32_t* scenes, const perch_search_params* params,
                       int64_t max_hyps_per_launch, perch_result* results);

/* Cost of the learned queue in the most recent perch_search or
 * perch_search_multi: wall seconds spent scoring states (parent renders,
 * crops, forward pass, host work), states scored and crops evaluated. Any
 * pointer may be NULL. */
int perch_search_stats(perch_ctx* ctx, double* learned_seconds, int64_t* learned_states, int64_t* learned_crops);

/* Where the wall time of the most recent search went: device evaluation
 * calls (uploads, kernels, record downloads), absorbing the records into the
 * search (duplicate detection, queues), and selecting the next states and
 * building their batch (including the learned queue's scoring). Any pointer
 * may be NULL. */
int perch_search_times(perch_ctx* ctx, double* eval_seconds, double* absorb_seconds, double* select_seconds);

/* Launch tuning (not in the paper). The evaluation runs persistent launches
 * per mesh with a shared-memory tile sized for that mesh; this call times the
 * launch parameters (see perch_launch_config: CTA widths 128, 256, 512 and
 * the render's inline limit; the cost launch's width) on
 * max(n_sample, 32 x SM count) hypotheses of each mesh (a fixed spread of its poses, children of
 * the empty scene), keeps the fastest per mesh for all later evaluations on
 * this context, and writes them to threads_out[n_mesh] (may be NULL). Results
 * are cached in the process per (device, triangle count, vertex count, tile
 * size). Without this call every mesh uses 256 threads. Requires an
 * observation (PERCH_E_STATE). */
int perch_autotune(perch_ctx* ctx, int32_t n_sample, int32_t* threads_out);

/* Set the CTA width (128, 256 or 512) used for one mesh (mesh = -1: all
 * meshes), overriding the default 256 or an autotuned choice. */
int perch_set_threads(perch_ctx* ctx, int32_t mesh, int32_t threads);

/* The launch configuration evaluations use now, per mesh (arrays of the
 * number of meshes, any may be NULL): the CTA width of the render (or
 * per-hypothesis evaluation) launch, the render's inline limit (a front-facing
 * triangle with at most that many candidate pixel centres is rasterised by
 * its own thread, a larger one by a warp through the CTA's queue) and the CTA
 * width of the cost launch. With shared renders on, perch_autotune times
 * every render width with every inline limit (8, 16, 32), then the cost
 * widths 128 and 256. */
int perch_launch_config(perch_ctx* ctx, int32_t* render_threads, int32_t* inline_pixels, int32_t* cost_threads);

/* Set the render's inline limit (8, 16 or 32) for one mesh (mesh = -1: all),
 * overriding the default 16 or an autotuned choice. Records do not depend on
 * it (coverage resolves by an order-independent max). */
int perch_set_inline_pixels(perch_ctx* ctx, int32_t mesh, int32_t inline_pixels);

/* The render's bin of larger triangles (the shared-memory queue each CTA
 * fills with front faces whose box holds more than the inline limit's
 * candidate centres, one warp per queued triangle): set its depth (32, 64 or
 * 128 entries) for one mesh (mesh = -1: all), overriding the default 128 or
 * an autotuned choice; a triangle that finds the bin full is rasterised by
 * its own thread, so records do not depend on it. perch_autotune times the
 * three depths per mesh after the CTA width and inline limit.
 * perch_launch_bin_depths writes the depths in use to depths[n_mesh]
 * (PERCH_E_STATE before meshes and pose grid are set). */
int perch_set_bin_depth(perch_ctx* ctx, int32_t mesh, int32_t depth);
int perch_launch_bin_depths(perch_ctx* ctx, int32_t* depths);

/* The cost launch's stage buffers for the stored tiles: 1 (default; the next
 * tile is copied once the current hypothesis is done, and more CTAs fit per
 * SM) or 2 (the next tile is copied while the current one is costed), for
 * one mesh (mesh = -1: all). Two are used only where they fit in shared
 * memory; records do not depend on it. perch_autotune times both with each
 * cost CTA width. perch_launch_cost_stages writes the stages in use to
 * stages[n_mesh] (PERCH_E_STATE before meshes and pose grid are set). */
int perch_set_cost_stages(perch_ctx* ctx, int32_t mesh, int32_t stages);
int perch_launch_cost_stages(perch_ctx* ctx, int32_t* stages);

/* Same work and arguments as perch_eval_successors_dev (device pointers), run
 * as a CUDA graph: the first call for a given argument set (and after any
 * change of meshes, pose grid or observation) runs the evaluation once and
 * captures it; later calls only launch the graph on the context's stream.
 * out_host (may be NULL) must be page-locked host memory; when given, the
 * graph also copies the n_hyp records there. The caller may rewrite the
 * contents of the device buffers between calls. perch_last_timing does not
 * cover graph launches. */
int perch_eval_graph(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride, const int32_t* parent_len,
                     int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp, int64_t n_hyp,
                     int32_t K_total, perch_cost* out, perch_cost* out_host);

/* Exact shortcut (on by default; not in the paper). A hypothesis whose
 * parent render is empty over its screen box and which has no observed point
 * within (its largest horizontal vertex radius + delta + 2 cm) of its (x, y)
 * gets its record without being rasterised again: all its pixels are new
 * (dR = its solo render, viol = 0), none is explained (djr = n_new = the
 * solo pixel count), no observed point lies in V(O) (djo = n_vol = 0) and on a
 * last-level edge every point of U stays unexplained (resid = |U|). The solo
 * pixel counts and cull flags come from the same rasteriser, run once per
 * (mesh, pose) against an empty parent and observation; the table is rebuilt
 * when the meshes, the pose grid or the camera change. Records are identical
 * with the shortcut on or off. on = 0 renders every hypothesis. */
int perch_set_shortcut(perch_ctx* ctx, int32_t on);

/* Shared renders (on by default; not in the paper). A successor's new-object
 * render depends only on its mesh and pose, not on its parent, so a batch is
 * grouped by pose: each distinct (mesh, x, y, yaw) is rasterised once into a
 * tile store in device memory (one tile per pose of the grid, sized by the
 * pose's screen box and allocated with the pose tables), and every
 * hypothesis is then compared with its own parent render and costed from
 * that tile. Records are identical with sharing on or off; on = 0 renders
 * every hypothesis separately (one kernel per hypothesis, no tile store).
 * Sharing applies to batches of two or more parents (one parent repeats no
 * pose), and stays off when the tile store would take more than a quarter of
 * the free device memory. */
int perch_set_share_renders(perch_ctx* ctx, int32_t on);

/* Render cache (not in the paper; off by default). With on != 0 and shared
 * renders in use, a pose's tile in the tile store stays valid after the
 * batch that rendered it: later evaluations on this context cost their
 * hypotheses of that pose from it and render only the poses they have not
 * seen (any number of parents then takes the shared path). An object's
 * render depends on its mesh and pose alone (and, for a single-scene batch,
 * the explained flag of each rendered point on the observation), so records
 * are identical with the cache on or off. Every change of the observation,
 * of the scenes or of the pose tables empties the cache, and so does this
 * call. perch_autotune turns it off while it times launches; a captured
 * evaluation (perch_eval_graph) never uses it. */
int perch_set_render_cache(perch_ctx* ctx, int32_t on);

/* Device time of the four phases of the most recent evaluation (CUDA
 * events on the context's stream): ms[0] parent z-buffers, residual sets and
 * the exact shortcut; ms[1] grouping the hypotheses; ms[2] the render
 * launches (with shared renders) or the per-hypothesis evaluation launches;
 * ms[3] the cost launches (0 without shared renders). *shared (may be NULL)
 * = 1 if the evaluation used shared renders. Waits for the events.
 * PERCH_E_STATE if no evaluation has been issued yet. */
int perch_last_phase_times(perch_ctx* ctx, float ms[4], int32_t* shared);

/* Bound on the polls of the evaluation kernel's first wait for each of its
 * bulk copies into shared memory (default, and for polls < 0: 2^20 polls or
 * 2 s, whichever comes first). A wait that gives up marks its record with
 * flags bit 30 and no cost; the kernel then waits for every copy still in
 * flight with the default bound before it takes further work, so a small
 * limit (0 = give up at once) exercises the failure path without leaving a
 * copy outstanding. Not in the paper; for failure-path tests. */
int perch_set_wait_limit(perch_ctx* ctx, int32_t polls);

/* Of the hypotheses of the most recent evaluation, how many took the
 * shortcut (0 if it was off) and how many there were. Waits for the stream. */
int perch_shortcut_stats(perch_ctx* ctx, int64_t* n_short, int64_t* n_total);

/* Device time of the most recent evaluation (perch_eval_successors or
 * perch_eval_successors_dev), measured with CUDA events recorded on the
 * context's stream around its two phases: prep_ms = parent z-buffers and
 * residual sets, eval_ms = the per-hypothesis evaluation kernel. Waits for
 * those events. Either pointer may be NULL. PERCH_E_STATE if no evaluation
 * has been issued yet. */
int perch_last_timing(perch_ctx* ctx, float* prep_ms, float* eval_ms);


/* ------------------------------------------------------------------------
 * Learned heuristic (the inadmissible heuristics of Sec. IV-C admit any
 * estimate of cost-to-go; Sec. VI proposes learning them; no network is
 * given in the paper). A small convolutional network predicts
 * y = log(1 + dJr + dJo + residual) of one successor from two 64 x 64 crops
 * centred on the projected hypothesis and a one-hot of (mesh, yaw):
 *   conv 3x3 2->32 stride 1, 32->64 s2, 64->128 s2, 128->128 s2 (pad 1,
 *   ReLU) -> flatten (row, column, channel) ++ one-hot -> FC 96 (ReLU) -> FC 1.
 * Activations and weights are bfloat16 with FP32 accumulation on the tensor
 * cores; Adam (beta 0.9 / 0.999, eps 1e-8) keeps FP32 master weights.
 * ------------------------------------------------------------------------ */
typedef struct perch_cnn perch_cnn;

/* Create a network with all parameters zero on `device` (stream as in
 * perch_create). n_onehot >= 1 one-hot inputs (index mesh * n_yaw + iyaw);
 * max_batch in [32, 1024], a multiple of 32: the largest batch of one
 * training step (forward passes of more crops run in chunks of it). */
int perch_cnn_create(perch_cnn** out, int device, void* cuda_stream, int32_t n_onehot, int32_t max_batch);
int perch_cnn_destroy(perch_cnn* net);
const char* perch_cnn_last_error(const perch_cnn* net);

/* Parameters as one FP32 array in this order: for each convolution its
 * weights [Cout][3][3][Cin] then bias [Cout]; FC1 weights [96][8192 +
 * n_onehot] then bias [96]; FC2 weights [96]; FC2 bias [1]. */
int perch_cnn_param_count(const perch_cnn* net, int64_t* n);
/* Host array of param_count floats; resets Adam's moments and step. */
int perch_cnn_set_params(perch_cnn* net, const float* params, int64_t n);
int perch_cnn_get_params(perch_cnn* net, float* params, int64_t n);

/* Network inputs for n_hyp hypotheses (host arrays in, DEVICE arrays out):
 * parents / hyp_parent / hyp as perch_eval_successors; parent_scene (may be
 * NULL: scene 0) selects the observed depth image. crops: n_hyp x 64 x 64 x 2
 * bfloat16 (row, column, channel; channel 0 observed depth, channel 1 the
 * parent's z-buffer), centred on the projection of (x, y, middle of V(O)'s
 * height range) computed in double: pixel (floor(u + 0.5), floor(v + 0.5));
 * value clamp((z_ref - d) * 10 / m, -3, 3) rounded to float then bfloat16
 * where the depth d is finite and > 0, else -4. onehot: n_hyp indices
 * mesh * n_yaw + iyaw. Synchronous. */
int perch_cnn_crops(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride, const int32_t* parent_len,
                    const int32_t* parent_scene, int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp,
                    int64_t n_hyp, uint16_t* crops, int32_t* onehot);

/* Tensor-core path of the forward 3x3 convolutions of layers 2-4 (the
 * implicit-im2col GEMMs): 0 = warp-level mma.sync (the default), 1 = tcgen05
 * MMAs into a tensor-memory accumulator (one 128-row x C_out tile per CTA,
 * operands staged in shared memory by cp.async). Both accumulate BF16
 * products in FP32 and apply bias + ReLU before rounding to BF16; sums are
 * taken in a different order, so outputs may differ in the last BF16 bit.
 * The backward pass always uses mma.sync. PERCH_E_ARG for another value. */
int perch_cnn_set_tensor_path(perch_cnn* net, int32_t path);

/* The current tensor path and whether a bounded wait of the tcgen05 kernel
 * ever gave up (its tile then keeps stale outputs). Waits for the stream. */
int perch_cnn_tensor_status(perch_cnn* net, int32_t* path, int32_t* waits_gave_up);

/* Predictions for n crops (device arrays), asynchronous on the network's
 * stream. */
int perch_cnn_forward(perch_cnn* net, const uint16_t* crops, const int32_t* onehot, int64_t n, float* pred);

/* One Adam step on the batch (device arrays; n a multiple of 32 up to
 * max_batch; loss 0.5 mean (pred - target)^2 before the step written to the
 * device float `loss`, may be NULL). Asynchronous. */
int perch_cnn_train_step(perch_cnn* net, const uint16_t* crops, const int32_t* onehot, const float* target,
                         int32_t n, float lr, float* loss);

/* Forward and backward pass without an update: gradients of the loss in the
 * parameter order above (host array of param_count floats, may be NULL), the
 * loss and the n predictions (host, may be NULL). Device inputs as
 * perch_cnn_train_step. Synchronous. */
int perch_cnn_gradients(perch_cnn* net, const uint16_t* crops, const int32_t* onehot, const float* target, int32_t n,
                        float* grads, float* loss, float* pred);

/* Use `net` (not owned; NULL detaches) for the learned heuristic of the
 * search (heuristics bits 2 and 3). n_candidates: placements per remaining object
 * type scored for a state (see perch_search). PERCH_E_ARG if the network's
 * one-hot is narrower than meshes x yaws. */
int perch_set_heuristic_net(perch_ctx* ctx, perch_cnn* net, int32_t n_candidates);

#ifdef __cplusplus
}
#endif
#endif /* PERCH_H_ */
