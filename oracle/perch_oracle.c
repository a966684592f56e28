/*
 * PERCH CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct restatement of what the successor-evaluation
 * path computes (Narayanan & Likhachev, "PERCH: Perception via Search for
 * Multi-Object Recognition and Localization"). Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load this library; the product
 * path never does. It shares no code, header or table with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math [-fopenmp] -shared -fPIC.
 * Every float operation below is one IEEE binary32 operation rounded to
 * nearest-even; a fused multiply-add appears only where written as fmaf()
 * (one rounding, as IEEE 754 defines it) and the compiler contracts nothing
 * else, so the result is fixed by the arithmetic written out at each step.
 *
 * What is computed, per the paper:
 *   - observed cloud I (Sec. III-A notation): valid depth pixels back-projected
 *     through the pinhole model;
 *   - rendered clouds R_j (Sec. III-A): z-buffer render of objects
 *     O_1..O_j, each at a 3-DoF table pose (x, y, yaw) (Sec. III);
 *   - explanation indicator, Eq. (1): p is unexplained by C iff every point
 *     of C is farther than delta;
 *   - decomposed edge cost, Sec. IV-A / Eq. (2):
 *       dJr  = #{p in dR_i unexplained by I}
 *       dJo  = #{q in I n V(O_i) unexplained by dR_i}
 *       resid= #{q in I - V_K unexplained by R_K}   (only when i = K)
 *   - monotone constraint R_{i-1} subset R_i of Eq. (3): the child is invalid
 *     when any of its pixels lies strictly in front of the parent's render;
 *   - undecomposed J = J_o + J_r of Sec. III-B (used to pin the K = 1 case);
 *   - ICP refinement of a successor's new object (Sec. IV-E-1, Sec. V-B),
 *     each step fixed below (the section headed ICP).
 *
 * Readings where the paper is silent (it only says "render"):
 *   - pinhole with pixel centres at integer (u, v); depth = camera-frame Z;
 *   - vertices snapped to 1/16 pixel (round half to even);
 *   - exact integer edge functions, coverage of pixel centres with the
 *     top-left tie rule; front faces only (positive signed area);
 *   - 1/z interpolated with the screen-space barycentrics, z-buffer keeps
 *     the minimum z;
 *   - a triangle with a vertex at z_c <= 0.05 m, a vertex beyond 2048 px, or
 *     an extent of 1024 px or more is dropped and counted ("culled");
 *   - distances are measured in the camera frame; "explained" is d^2 <= delta^2
 *     (Eq. (1) calls a point unexplained only when the distance exceeds delta);
 *   - V(O) is an inscribed vertical cylinder about the object origin, the
 *     conservative volume the paper names in Sec. III-A, or, where the
 *     mesh describes a box, a regular prism or a superquadric with
 *     polynomial exponents, that solid in closed form (in_volume).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t n_verts, n_tris;
  const float* verts;   /* n_verts x 3, object frame, z up */
  const int32_t* tris;  /* n_tris x 3 */
  float vol_r, vol_zlo, vol_zhi; /* V(O): inscribed cylinder (kind 0) */
  /* V(O) in closed form (kind 1 box, 2 regular prism, 3 superquadric; 0 =
   * the inscribed cylinder above), in the object frame:
   *   box:          |x| <= p0, |y| <= p1, zlo <= z <= zhi
   *   prism:        zlo <= z <= zhi and normals[k] . (x, y) <= p1 for all k < n
   *   superquadric: X = x / p0, Y = y / p1, Z = (z - p3) / p2 (each as a
   *                 product with the binary32 reciprocal of the semi-axis);
   *                 n = 1: X^2 + Y^2 + Z^2 <= 1; n = 2: (X^2 + Y^2)^2 + Z^4 <= 1 */
  int32_t kind, n;
  float p[4];
  float zlo, zhi;
  const float* normals; /* prism: n x 2 */
} or_mesh;

typedef struct { uint16_t mesh, iyaw; int16_t ix, iy; } or_obj;

typedef struct {
  int32_t W, H;
  float fx, fy, cx, cy;
  float T_wc[12];       /* camera -> world, row-major 3x4 */
  const float* xs; int32_t nx;
  const float* ys; int32_t ny;
  const float* cos_sin; int32_t n_yaw; /* (cos, sin) per yaw */
  const or_mesh* meshes; int32_t n_mesh;
  float delta;
} or_world;

/* record: dJr, dJo, resid, viol, n_new, flags, n_vol
 * n_vol = #{q in I n V(O) : q outside every parent object's volume}, the
 * decrease of the overlap heuristic h_overlap of Sec. IV-C from parent to
 * child (h_overlap(s) = |I| - #{q in I n V_j}). */
enum { OR_DJR = 0, OR_DJO, OR_RESID, OR_VIOL, OR_NNEW, OR_FLAGS, OR_NVOL, OR_REC };
#define OR_FLAG_CULLED 1u
#define OR_FLAG_INVALID 2u

/* ------------------------------------------------------------------ camera */
typedef struct {
  float Rcw[9], tcw[3];  /* world -> camera */
  float Rwc[9], twc[3];  /* camera -> world */
  float* rx;             /* (u - cx) / fx, per column */
  float* ry;             /* (v - cy) / fy, per row */
  float delta2;
} or_cam;

static int cam_init(const or_world* w, or_cam* c) {
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) c->Rwc[r * 3 + k] = w->T_wc[r * 4 + k];
    c->twc[r] = w->T_wc[r * 4 + 3];
  }
  /* R_cw is the exact transpose; t_cw = -R_wc^T t_wc in double, then rounded */
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) c->Rcw[r * 3 + k] = c->Rwc[k * 3 + r];
    double acc = (double)c->Rwc[0 * 3 + r] * (double)c->twc[0];
    acc = acc + (double)c->Rwc[1 * 3 + r] * (double)c->twc[1];
    acc = acc + (double)c->Rwc[2 * 3 + r] * (double)c->twc[2];
    c->tcw[r] = (float)(-acc);
  }
  c->rx = (float*)malloc(sizeof(float) * (size_t)w->W);
  c->ry = (float*)malloc(sizeof(float) * (size_t)w->H);
  if (!c->rx || !c->ry) { free(c->rx); free(c->ry); return -1; }
  for (int u = 0; u < w->W; ++u) c->rx[u] = (float)(((double)u - (double)w->cx) / (double)w->fx);
  for (int v = 0; v < w->H; ++v) c->ry[v] = (float)(((double)v - (double)w->cy) / (double)w->fy);
  c->delta2 = (float)((double)w->delta * (double)w->delta);
  return 0;
}

static void cam_free(or_cam* c) { free(c->rx); free(c->ry); }

/* ------------------------------------------------------------ rasteriser */
typedef struct { int64_t X, Y; float iz; int bad; } or_vtx;

/* Camera-frame pose of a placed object: the yaw rotation and the
 * world->camera rotation composed into one matrix M = R_cw Rz(yaw), and the
 * table translation into one offset b = R_cw (x, y, 0) + t_cw. Both are
 * evaluated in double from the binary32 inputs (every product of two floats
 * is exact in double) and rounded once to binary32. */
typedef struct { float M[9]; float b[3]; } or_pose;

static or_pose placed_pose(const or_world* w, const or_cam* c, or_obj o) {
  or_pose p;
  double cs = w->cos_sin[2 * o.iyaw], sn = w->cos_sin[2 * o.iyaw + 1];
  double x = w->xs[o.ix], y = w->ys[o.iy];
  for (int r = 0; r < 3; ++r) {
    double r0 = c->Rcw[r * 3 + 0], r1 = c->Rcw[r * 3 + 1], r2 = c->Rcw[r * 3 + 2];
    p.M[r * 3 + 0] = (float)(r0 * cs + r1 * sn);
    p.M[r * 3 + 1] = (float)(r1 * cs - r0 * sn);
    p.M[r * 3 + 2] = (float)r2;
    p.b[r] = (float)((r0 * x + r1 * y) + (double)c->tcw[r]);
  }
  return p;
}

/* object-frame vertex -> camera -> pixel, snapped to 1/16 pixel:
 * c_r = fma(M_r2, vz, fma(M_r1, vy, M_r0 vx)) + b_r; 1/z = 1/c_z;
 * u = fma(fx, c_x (1/z), cx); X = rint(16 u) */
static or_vtx transform_vertex(const or_world* w, const or_pose* p, const float* v) {
  or_vtx o;
  float cam[3];
  for (int r = 0; r < 3; ++r) {
    float a = p->M[r * 3 + 0] * v[0];
    a = fmaf(p->M[r * 3 + 1], v[1], a);
    a = fmaf(p->M[r * 3 + 2], v[2], a);
    cam[r] = a + p->b[r];
  }
  o.bad = !(cam[2] > 0.05f);
  float iz = 1.0f / cam[2];
  float qx = cam[0] * iz, qy = cam[1] * iz;
  float u = fmaf(w->fx, qx, w->cx), vv = fmaf(w->fy, qy, w->cy);
  if (!(fabsf(u) <= 2048.0f) || !(fabsf(vv) <= 2048.0f)) o.bad = 1;
  if (o.bad) { o.X = o.Y = 0; o.iz = 0.0f; return o; }
  o.X = (int64_t)lrintf(16.0f * u);
  o.Y = (int64_t)lrintf(16.0f * vv);
  o.iz = iz;
  return o;
}

/* signed edge function of edge a->b at point P (exact integers); positive
 * on the inner side of a front-facing triangle */
static int64_t edge_fn(int64_t Xa, int64_t Ya, int64_t Xb, int64_t Yb, int64_t Px, int64_t Py) {
  return (Yb - Ya) * (Px - Xa) - (Xb - Xa) * (Py - Ya);
}

/* top-left tie rule for front faces in this orientation */
static int owns_edge(int64_t Xa, int64_t Ya, int64_t Xb, int64_t Yb) {
  int64_t dy = Yb - Ya, dx = Xb - Xa;
  return dy > 0 || (dy == 0 && dx < 0);
}

static int64_t floordiv16(int64_t a) { return a >= 0 ? a / 16 : -((-a + 15) / 16); }
static int64_t ceildiv16(int64_t a) { return -floordiv16(-a); }

/* render one object into zbuf (min), counting culled triangles */
static void render_object(const or_world* w, const or_cam* c, or_obj o, float* zbuf, int64_t* culled) {
  const or_mesh* m = &w->meshes[o.mesh];
  const or_pose pose = placed_pose(w, c, o);
  for (int t = 0; t < m->n_tris; ++t) {
    or_vtx v[3];
    int bad = 0;
    for (int k = 0; k < 3; ++k) {
      v[k] = transform_vertex(w, &pose, m->verts + 3 * (size_t)m->tris[3 * t + k]);
      bad |= v[k].bad;
    }
    if (bad) { (*culled)++; continue; }
    int64_t A = edge_fn(v[0].X, v[0].Y, v[1].X, v[1].Y, v[2].X, v[2].Y);
    if (A <= 0) continue; /* back-facing or degenerate */
    int64_t xmin = v[0].X, xmax = v[0].X, ymin = v[0].Y, ymax = v[0].Y;
    for (int k = 1; k < 3; ++k) {
      if (v[k].X < xmin) xmin = v[k].X;
      if (v[k].X > xmax) xmax = v[k].X;
      if (v[k].Y < ymin) ymin = v[k].Y;
      if (v[k].Y > ymax) ymax = v[k].Y;
    }
    if (xmax - xmin >= 16384 || ymax - ymin >= 16384) { (*culled)++; continue; }
    int64_t px0 = ceildiv16(xmin), px1 = floordiv16(xmax);
    int64_t py0 = ceildiv16(ymin), py1 = floordiv16(ymax);
    if (px0 < 0) px0 = 0;
    if (py0 < 0) py0 = 0;
    if (px1 > w->W - 1) px1 = w->W - 1;
    if (py1 > w->H - 1) py1 = w->H - 1;
    int own12 = owns_edge(v[1].X, v[1].Y, v[2].X, v[2].Y);
    int own20 = owns_edge(v[2].X, v[2].Y, v[0].X, v[0].Y);
    int own01 = owns_edge(v[0].X, v[0].Y, v[1].X, v[1].Y);
    float invA = 1.0f / (float)A;
    for (int64_t py = py0; py <= py1; ++py) {
      for (int64_t px = px0; px <= px1; ++px) {
        int64_t Px = 16 * px, Py = 16 * py;
        int64_t w0 = edge_fn(v[1].X, v[1].Y, v[2].X, v[2].Y, Px, Py);
        int64_t w1 = edge_fn(v[2].X, v[2].Y, v[0].X, v[0].Y, Px, Py);
        int64_t w2 = edge_fn(v[0].X, v[0].Y, v[1].X, v[1].Y, Px, Py);
        int in0 = w0 > 0 || (w0 == 0 && own12);
        int in1 = w1 > 0 || (w1 == 0 && own20);
        int in2 = w2 > 0 || (w2 == 0 && own01);
        if (!(in0 && in1 && in2)) continue;
        float b0 = (float)w0 * invA, b1 = (float)w1 * invA, b2 = (float)w2 * invA;
        float iz = b0 * v[0].iz;
        iz = fmaf(b1, v[1].iz, iz);
        iz = fmaf(b2, v[2].iz, iz);
        float z = 1.0f / iz;
        float* dst = &zbuf[py * w->W + px];
        if (z < *dst) *dst = z;
      }
    }
  }
}

static void render_scene(const or_world* w, const or_cam* c, const or_obj* objs, int n,
                         float* zbuf, int64_t* culled) {
  for (int64_t i = 0; i < (int64_t)w->W * w->H; ++i) zbuf[i] = INFINITY;
  for (int k = 0; k < n; ++k) render_object(w, c, objs[k], zbuf, culled);
}

/* ------------------------------------------------------------ point sets */
typedef struct { float x, y, z; } or_pt;

static or_pt pixel_point(const or_cam* c, int u, int v, float z) {
  or_pt p = {c->rx[u] * z, c->ry[v] * z, z};
  return p;
}

static or_pt cam_to_world(const or_cam* c, or_pt p) {
  float o[3];
  for (int r = 0; r < 3; ++r) {
    float a = c->Rwc[r * 3 + 0] * p.x;
    a = fmaf(c->Rwc[r * 3 + 1], p.y, a);
    a = fmaf(c->Rwc[r * 3 + 2], p.z, a);
    o[r] = a + c->twc[r];
  }
  or_pt q = {o[0], o[1], o[2]};
  return q;
}

static float dist2(or_pt a, or_pt b) {
  float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  float d = dx * dx;
  d = fmaf(dy, dy, d);
  return fmaf(dz, dz, d);
}

/* Eq. (1): p is explained by C iff some point of C lies within delta */
static int explained(or_pt p, const or_pt* C, int64_t n, float delta2) {
  for (int64_t i = 0; i < n; ++i)
    if (dist2(p, C[i]) <= delta2) return 1;
  return 0;
}

/* V(O) (Sec. III-A: the volume the object occupies) at the object's pose:
 * the inscribed vertical cylinder about its origin (kind 0), or the closed
 * form of its solid (kinds 1-3), tested in the object frame: the world
 * point's offset from (x, y) turned by -yaw with the pose table's binary32
 * (cos, sin): x' = fma(s, dy, c dx), y' = fma(c, dy, -(s dx)); z is the
 * world height (objects stand on the table plane z = 0). */
static int in_volume(const or_world* w, or_obj o, or_pt qw) {
  const or_mesh* m = &w->meshes[o.mesh];
  float dx = qw.x - w->xs[o.ix], dy = qw.y - w->ys[o.iy];
  if (m->kind == 0) {
    float r2 = (float)((double)m->vol_r * (double)m->vol_r);
    float d2 = fmaf(dy, dy, dx * dx);
    return d2 <= r2 && m->vol_zlo <= qw.z && qw.z <= m->vol_zhi;
  }
  float c = w->cos_sin[2 * o.iyaw], sn = w->cos_sin[2 * o.iyaw + 1];
  float xo = fmaf(sn, dy, c * dx);
  float yo = fmaf(c, dy, -(sn * dx));
  if (m->kind == 1) return fabsf(xo) <= m->p[0] && fabsf(yo) <= m->p[1] && m->zlo <= qw.z && qw.z <= m->zhi;
  if (m->kind == 2) {
    if (!(m->zlo <= qw.z && qw.z <= m->zhi)) return 0;
    for (int k = 0; k < m->n; ++k)
      if (fmaf(m->normals[2 * k + 1], yo, m->normals[2 * k] * xo) > m->p[1]) return 0;
    return 1;
  }
  /* superquadric */
  float X = xo * (float)(1.0 / (double)m->p[0]);
  float Y = yo * (float)(1.0 / (double)m->p[1]);
  float Z = (qw.z - m->p[3]) * (float)(1.0 / (double)m->p[2]);
  float t = fmaf(Y, Y, X * X);
  float z2 = Z * Z;
  float F = m->n == 2 ? fmaf(t, t, z2 * z2) : t + z2;
  return F <= 1.0f;
}

typedef struct { or_pt* cam; or_pt* world; int64_t n; } or_cloud;

/* observed cloud I: every pixel with a finite positive depth */
static int observed_cloud(const or_world* w, const or_cam* c, const float* depth, or_cloud* I) {
  int64_t n = 0, N = (int64_t)w->W * w->H;
  I->cam = (or_pt*)malloc(sizeof(or_pt) * (size_t)(N > 0 ? N : 1));
  I->world = (or_pt*)malloc(sizeof(or_pt) * (size_t)(N > 0 ? N : 1));
  if (!I->cam || !I->world) { free(I->cam); free(I->world); return -1; }
  for (int v = 0; v < w->H; ++v)
    for (int u = 0; u < w->W; ++u) {
      float d = depth[(int64_t)v * w->W + u];
      if (!(d > 0.0f) || !isfinite(d)) continue;
      I->cam[n] = pixel_point(c, u, v, d);
      I->world[n] = cam_to_world(c, I->cam[n]);
      n++;
    }
  I->n = n;
  return 0;
}

/* valid pixels of a z-buffer as camera-frame points */
static int64_t zbuf_points(const or_world* w, const or_cam* c, const float* z, or_pt* out) {
  int64_t n = 0;
  for (int v = 0; v < w->H; ++v)
    for (int u = 0; u < w->W; ++u) {
      float d = z[(int64_t)v * w->W + u];
      if (isfinite(d)) out[n++] = pixel_point(c, u, v, d);
    }
  return n;
}

/* ------------------------------------------------------------ edge cost */
/* One MSGT edge (Eq. (3), Eq. (4)): parent render zp, child object o. */
static void edge_cost(const or_world* w, const or_cam* c, const or_cloud* I,
                      const or_obj* parent, int n_parent, const float* zp, or_obj o,
                      int K_total, float* zc, or_pt* pts, int32_t* rec) {
  int64_t N = (int64_t)w->W * w->H, culled = 0;
  for (int64_t i = 0; i < N; ++i) zc[i] = INFINITY;
  render_object(w, c, o, zc, &culled);
  int64_t viol = 0, n_new = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (!isfinite(zc[i])) continue;
    if (!isfinite(zp[i])) n_new++;         /* dR: child visible, parent empty */
    else if (zc[i] < zp[i]) viol++;        /* child occludes the parent's render */
  }
  uint32_t flags = culled ? OR_FLAG_CULLED : 0u;
  memset(rec, 0, sizeof(int32_t) * OR_REC);
  rec[OR_VIOL] = (int32_t)viol;
  rec[OR_NNEW] = (int32_t)n_new;
  if (viol > 0) { rec[OR_FLAGS] = (int32_t)(flags | OR_FLAG_INVALID); return; }
  rec[OR_FLAGS] = (int32_t)flags;

  /* dR_{j+1} as camera-frame points */
  int64_t nd = 0;
  for (int v = 0; v < w->H; ++v)
    for (int u = 0; u < w->W; ++u) {
      int64_t i = (int64_t)v * w->W + u;
      if (isfinite(zc[i]) && !isfinite(zp[i])) pts[nd++] = pixel_point(c, u, v, zc[i]);
    }
  int64_t djr = 0;
  for (int64_t k = 0; k < nd; ++k)
    if (!explained(pts[k], I->cam, I->n, c->delta2)) djr++;
  int64_t djo = 0, nvol = 0;
  for (int64_t k = 0; k < I->n; ++k) {
    if (!in_volume(w, o, I->world[k])) continue;
    if (!explained(I->cam[k], pts, nd, c->delta2)) djo++;
    int in_parent = 0;
    for (int j = 0; j < n_parent && !in_parent; ++j) in_parent = in_volume(w, parent[j], I->world[k]);
    if (!in_parent) nvol++;
  }
  rec[OR_DJR] = (int32_t)djr;
  rec[OR_DJO] = (int32_t)djo;
  rec[OR_NVOL] = (int32_t)nvol;

  if (n_parent + 1 == K_total) {
    /* residual(K): observed points outside V_K unexplained by R_K */
    for (int64_t i = 0; i < N; ++i) zc[i] = (zc[i] < zp[i]) ? zc[i] : zp[i];
    int64_t nr = zbuf_points(w, c, zc, pts);
    int64_t resid = 0;
    for (int64_t k = 0; k < I->n; ++k) {
      int inside = in_volume(w, o, I->world[k]);
      for (int j = 0; j < n_parent && !inside; ++j) inside = in_volume(w, parent[j], I->world[k]);
      if (inside) continue;
      if (!explained(I->cam[k], pts, nr, c->delta2)) resid++;
    }
    rec[OR_RESID] = (int32_t)resid;
  }
}

/* ------------------------------------------------------------------ ICP */
/* Local alignment of a successor's new object with the observed cloud
 * (Sec. IV-E-1, compensating for discretization: each time a state is
 * rendered with a new object, the object's non-occluded portion is aligned
 * with I by ICP in the local vicinity; Sec. V-B: correspondences are sought
 * only within 2 cm, half the grid step). The paper names ICP without fixing
 * its variant; this restatement fixes every step, so the result is a
 * function of the inputs alone:
 *   model set M: the pixels where the object's own render z_O is finite and
 *     lies strictly in front of the parent's render z_P (+inf where empty),
 *     back-projected to the world frame exactly as the observed cloud is;
 *   motion T = (c, s, t_x, t_y): a turn about the world's vertical axis and
 *     a translation in the table plane (the pose's three degrees of
 *     freedom), applied in binary32 from T's values rounded to binary32:
 *     x' = (c x - s y) + t_x, y' = (s x + c y) + t_y, z' = z;
 *   correspondence of m in M: the point q of I of smallest
 *     d^2 = fma(dz, dz, fma(dy, dy, dx dx)) (d = T m - q) among those with
 *     d^2 <= (float)(r^2); ties go to the smaller index of q in I (pixel
 *     order); none: m is unmatched;
 *   sums over the matched pairs, in fixed point (coordinates times 2^16,
 *     rounded to the nearest integer, ties to even) so that they are exact
 *     and independent of the order of summation: n, sum X_m, sum Y_m,
 *     sum X_q, sum Y_q, sum X_m X_q, sum Y_m Y_q, sum X_m Y_q, sum Y_m X_q
 *     (a pair with |x| or |y| >= 32 m for m or q is left out);
 *   fit: the motion minimising sum |T m - q|^2 over the pairs' (x, y), in
 *     closed form (icp_solve);
 *   iteration k = 1 .. max_iter, from T = identity: match under the current
 *     T; fewer than 3 pairs: stop (FEW); the same sums as the previous
 *     iteration: stop (CONVERGED, the fit would repeat itself); no rotation
 *     defined: stop (DEGENERATE); else T = fit of the pairs. After max_iter
 *     fits: CAP. */
typedef struct { double c, s, tx, ty; int32_t n_model, n_corr, iters, status; } or_icp_rec;
enum { OR_ICP_CONVERGED = 0, OR_ICP_CAP = 1, OR_ICP_FEW = 2, OR_ICP_DEGENERATE = 3 };

typedef struct { int64_t n, sx, sy, qx, qy, xx, yy, xy, yx; } or_icp_sums;

static int64_t icp_fixed(float v) { return (int64_t)llrintf(v * 65536.0f); }

/* a 128-bit integer as hi 2^64 + lo, each part rounded to double, then one
 * rounded addition */
static double i128_to_double(__int128 v) {
  int64_t hi = (int64_t)(v >> 64);
  uint64_t lo = (uint64_t)v;
  return (double)hi * 18446744073709551616.0 + (double)lo;
}

static void icp_add_pair(or_icp_sums* S, or_pt m, or_pt q) {
  if (!(fabsf(m.x) < 32.0f && fabsf(m.y) < 32.0f && fabsf(q.x) < 32.0f && fabsf(q.y) < 32.0f)) return;
  int64_t X = icp_fixed(m.x), Y = icp_fixed(m.y), QX = icp_fixed(q.x), QY = icp_fixed(q.y);
  S->n += 1;
  S->sx += X; S->sy += Y; S->qx += QX; S->qy += QY;
  S->xx += X * QX; S->yy += Y * QY; S->xy += X * QY; S->yx += Y * QX;
}

/* Planar Procrustes: with centred sums C = n sum(m . q) - sum m . sum q and
 * S = n sum(m x q) - sum m x sum q (exact integers), the best turn has
 * (cos, sin) = (C, S) / |(C, S)| and the best translation moves the turned
 * centroid of M onto that of Q: t = (sum q - R sum m) / n. Returns 1 when
 * C = S = 0 (no turn is better than another). */
static int icp_solve(const or_icp_sums* S, double* c, double* s, double* tx, double* ty) {
  const __int128 n = S->n;
  const __int128 C = n * ((__int128)S->xx + S->yy) - ((__int128)S->sx * S->qx + (__int128)S->sy * S->qy);
  const __int128 X = n * ((__int128)S->xy - S->yx) - ((__int128)S->sx * S->qy - (__int128)S->sy * S->qx);
  if (C == 0 && X == 0) return 1;
  const double Cd = i128_to_double(C), Xd = i128_to_double(X);
  const double h = sqrt(Cd * Cd + Xd * Xd);
  const double cc = Cd / h, ss = Xd / h;
  const double nd = (double)S->n, sx = (double)S->sx, sy = (double)S->sy;
  *c = cc;
  *s = ss;
  *tx = (((double)S->qx - (cc * sx - ss * sy)) / nd) * (1.0 / 65536.0);
  *ty = (((double)S->qy - (ss * sx + cc * sy)) / nd) * (1.0 / 65536.0);
  return 0;
}

/* observed world points ordered by x (then by index): a candidate whose x
 * differs from the query's by more than 1.001 r cannot be within r (its
 * rounded dx^2 alone already exceeds the rounded r^2), so the scan of the
 * ordered list stops there; every other point is tested in full */
static const or_pt* g_sort_pts;
static int cmp_by_x(const void* a, const void* b) {
  int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  float xi = g_sort_pts[i].x, xj = g_sort_pts[j].x;
  if (xi < xj) return -1;
  if (xi > xj) return 1;
  return (i > j) - (i < j);
}

static int64_t* order_by_x(const or_cloud* I) {
  int64_t* o = (int64_t*)malloc(sizeof(int64_t) * (size_t)(I->n > 0 ? I->n : 1));
  if (!o) return NULL;
  for (int64_t k = 0; k < I->n; ++k) o[k] = k;
  g_sort_pts = I->world;
  qsort(o, (size_t)I->n, sizeof(int64_t), cmp_by_x);
  return o;
}

/* the correspondence of world point p (index into I, or -1) */
static int64_t icp_match(const or_cloud* I, const int64_t* by_x, or_pt p, double r, float r2) {
  const double lo = (double)p.x - 1.001 * r, hi = (double)p.x + 1.001 * r;
  int64_t a = 0, b = I->n;
  while (a < b) {  /* first point with x >= lo */
    int64_t mid = a + (b - a) / 2;
    if ((double)I->world[by_x[mid]].x < lo) a = mid + 1; else b = mid;
  }
  int64_t best = -1;
  float bd = 0.0f;
  for (int64_t k = a; k < I->n && (double)I->world[by_x[k]].x <= hi; ++k) {
    const int64_t j = by_x[k];
    const float d = dist2(p, I->world[j]);
    if (!(d <= r2)) continue;
    if (best < 0 || d < bd || (d == bd && j < best)) { best = j; bd = d; }
  }
  return best;
}

static or_pt icp_apply(float c, float s, float tx, float ty, or_pt m) {
  or_pt p = {(c * m.x - s * m.y) + tx, (s * m.x + c * m.y) + ty, m.z};
  return p;
}

/* ICP of one model set against I (the iteration stated above) */
static void icp_run(const or_cloud* I, const int64_t* by_x, const or_pt* M, int64_t nm, double r,
                    int32_t max_iter, or_icp_rec* out) {
  const float r2 = (float)(r * r);
  double c = 1.0, s = 0.0, tx = 0.0, ty = 0.0;
  or_icp_sums prev;
  int have_prev = 0;
  out->status = OR_ICP_CAP;
  out->iters = 0;
  out->n_corr = 0;
  out->n_model = (int32_t)nm;
  for (int32_t k = 1; k <= max_iter; ++k) {
    const float cf = (float)c, sf = (float)s, txf = (float)tx, tyf = (float)ty;
    or_icp_sums S;
    memset(&S, 0, sizeof S);
    for (int64_t i = 0; i < nm; ++i) {
      const int64_t j = icp_match(I, by_x, icp_apply(cf, sf, txf, tyf, M[i]), r, r2);
      if (j >= 0) icp_add_pair(&S, M[i], I->world[j]);
    }
    out->n_corr = (int32_t)S.n;
    if (S.n < 3) { out->status = OR_ICP_FEW; break; }
    if (have_prev && memcmp(&S, &prev, sizeof S) == 0) { out->status = OR_ICP_CONVERGED; break; }
    double c1, s1, tx1, ty1;
    if (icp_solve(&S, &c1, &s1, &tx1, &ty1)) { out->status = OR_ICP_DEGENERATE; break; }
    c = c1; s = s1; tx = tx1; ty = ty1;
    prev = S;
    have_prev = 1;
    out->iters = k;
  }
  out->c = c; out->s = s; out->tx = tx; out->ty = ty;
}

/* model set of one successor: the new object's pixels in front of the
 * parent's render, in the world frame */
static int64_t icp_model(const or_world* w, const or_cam* c, const float* zo, const float* zp, or_pt* M) {
  int64_t n = 0;
  for (int v = 0; v < w->H; ++v)
    for (int u = 0; u < w->W; ++u) {
      const int64_t i = (int64_t)v * w->W + u;
      if (isfinite(zo[i]) && zo[i] < zp[i]) M[n++] = cam_to_world(c, pixel_point(c, u, v, zo[i]));
    }
  return n;
}

/* ================================================================ exports */

/* z-buffer render of n objects (min z; +inf where empty). Returns the
 * number of culled triangles, or -1 on allocation failure. */
int64_t or_render(const or_world* w, const or_obj* objs, int32_t n, float* zbuf) {
  or_cam c;
  if (cam_init(w, &c)) return -1;
  int64_t culled = 0;
  render_scene(w, &c, objs, n, zbuf, &culled);
  cam_free(&c);
  return culled;
}

/* observed cloud I in camera and world frames; returns |I| (arrays must hold
 * W*H points of 3 floats) */
int64_t or_observed(const or_world* w, const float* depth, float* cam_xyz, float* world_xyz) {
  or_cam c;
  if (cam_init(w, &c)) return -1;
  or_cloud I;
  if (observed_cloud(w, &c, depth, &I)) { cam_free(&c); return -1; }
  for (int64_t k = 0; k < I.n; ++k) {
    cam_xyz[3 * k] = I.cam[k].x; cam_xyz[3 * k + 1] = I.cam[k].y; cam_xyz[3 * k + 2] = I.cam[k].z;
    world_xyz[3 * k] = I.world[k].x; world_xyz[3 * k + 1] = I.world[k].y; world_xyz[3 * k + 2] = I.world[k].z;
  }
  int64_t n = I.n;
  free(I.cam); free(I.world); cam_free(&c);
  return n;
}

/* V(O) membership of n world points for one object (the test above) */
int32_t or_in_volume(const or_world* w, or_obj o, const float* pts, int64_t n, int32_t* out) {
  for (int64_t k = 0; k < n; ++k) {
    or_pt q = {pts[3 * k], pts[3 * k + 1], pts[3 * k + 2]};
    out[k] = in_volume(w, o, q);
  }
  return 0;
}

/* Eq. (1) over explicit clouds: out[k] = 1 iff P[k] is unexplained by Q */
int32_t or_unexplained(const float* P, int64_t np, const float* Q, int64_t nq, float delta, int32_t* out) {
  float d2 = (float)((double)delta * (double)delta);
  for (int64_t k = 0; k < np; ++k) {
    or_pt p = {P[3 * k], P[3 * k + 1], P[3 * k + 2]};
    int ex = 0;
    for (int64_t i = 0; i < nq && !ex; ++i) {
      or_pt q = {Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]};
      ex = dist2(p, q) <= d2;
    }
    out[k] = !ex;
  }
  return 0;
}

/* Undecomposed explanation cost of Sec. III-B for a full assignment:
 * out[0] = J_o (observed points unexplained by R_K), out[1] = J_r. */
int32_t or_cost_J(const or_world* w, const float* depth, const or_obj* objs, int32_t K, int64_t* out) {
  or_cam c;
  if (cam_init(w, &c)) return -1;
  or_cloud I;
  if (observed_cloud(w, &c, depth, &I)) { cam_free(&c); return -1; }
  int64_t N = (int64_t)w->W * w->H, culled = 0;
  float* z = (float*)malloc(sizeof(float) * (size_t)N);
  or_pt* R = (or_pt*)malloc(sizeof(or_pt) * (size_t)N);
  if (!z || !R) { free(z); free(R); free(I.cam); free(I.world); cam_free(&c); return -1; }
  render_scene(w, &c, objs, K, z, &culled);
  int64_t nr = zbuf_points(w, &c, z, R);
  int64_t jo = 0, jr = 0;
  for (int64_t k = 0; k < I.n; ++k) jo += !explained(I.cam[k], R, nr, c.delta2);
  for (int64_t k = 0; k < nr; ++k) jr += !explained(R[k], I.cam, I.n, c.delta2);
  out[0] = jo; out[1] = jr;
  free(z); free(R); free(I.cam); free(I.world); cam_free(&c);
  return 0;
}

/* Edge costs for a batch of successors. parents: n_par x k_max objects,
 * parent_len[i] of them used; hypothesis h adds hyps[h] to parent
 * hyp_parent[h]; K_total = objects in a complete scene. recs: n_hyp x 7. */
int32_t or_eval_batch(const or_world* w, const float* depth,
                      const or_obj* parents, const int32_t* parent_len, int32_t n_par, int32_t k_max,
                      const int32_t* hyp_parent, const or_obj* hyps, int64_t n_hyp,
                      int32_t K_total, int32_t* recs, int32_t n_threads) {
  or_cam c;
  if (cam_init(w, &c)) return -1;
  or_cloud I;
  if (observed_cloud(w, &c, depth, &I)) { cam_free(&c); return -1; }
  int64_t N = (int64_t)w->W * w->H;
  float* zp = (float*)malloc(sizeof(float) * (size_t)N * (size_t)(n_par > 0 ? n_par : 1));
  if (!zp) { free(I.cam); free(I.world); cam_free(&c); return -1; }
  for (int32_t p = 0; p < n_par; ++p) {
    int64_t culled = 0;
    render_scene(w, &c, parents + (int64_t)p * k_max, parent_len[p], zp + (int64_t)p * N, &culled);
  }
  int err = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
#pragma omp parallel
  {
    float* zc = (float*)malloc(sizeof(float) * (size_t)N);
    or_pt* pts = (or_pt*)malloc(sizeof(or_pt) * (size_t)N);
    if (!zc || !pts) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t h = 0; h < n_hyp; ++h) {
        int32_t p = hyp_parent[h];
        edge_cost(w, &c, &I, parents + (int64_t)p * k_max, parent_len[p], zp + (int64_t)p * N,
                  hyps[h], K_total, zc, pts, recs + h * OR_REC);
      }
    }
    free(zc); free(pts);
  }
  free(zp); free(I.cam); free(I.world); cam_free(&c);
  return err ? -1 : 0;
}

/* ICP refinement of n_hyp successors (the restatement above). parents,
 * parent_len, hyp_parent, hyps as in or_eval_batch; radius = the
 * correspondence distance r in metres; out[n_hyp]. */
int32_t or_icp_refine(const or_world* w, const float* depth,
                      const or_obj* parents, const int32_t* parent_len, int32_t n_par, int32_t k_max,
                      const int32_t* hyp_parent, const or_obj* hyps, int64_t n_hyp,
                      float radius, int32_t max_iter, or_icp_rec* out, int32_t n_threads) {
  or_cam c;
  if (cam_init(w, &c)) return -1;
  or_cloud I;
  if (observed_cloud(w, &c, depth, &I)) { cam_free(&c); return -1; }
  int64_t* by_x = order_by_x(&I);
  int64_t N = (int64_t)w->W * w->H;
  float* zp = (float*)malloc(sizeof(float) * (size_t)N * (size_t)(n_par > 0 ? n_par : 1));
  if (!zp || !by_x) { free(zp); free(by_x); free(I.cam); free(I.world); cam_free(&c); return -1; }
  for (int32_t p = 0; p < n_par; ++p) {
    int64_t culled = 0;
    render_scene(w, &c, parents + (int64_t)p * k_max, parent_len[p], zp + (int64_t)p * N, &culled);
  }
  int err = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
#pragma omp parallel
  {
    float* zo = (float*)malloc(sizeof(float) * (size_t)N);
    or_pt* M = (or_pt*)malloc(sizeof(or_pt) * (size_t)N);
    if (!zo || !M) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t h = 0; h < n_hyp; ++h) {
        int64_t culled = 0;
        render_scene(w, &c, hyps + h, 1, zo, &culled);
        const int64_t nm = icp_model(w, &c, zo, zp + (int64_t)hyp_parent[h] * N, M);
        icp_run(&I, by_x, M, nm, (double)radius, max_iter, out + h);
      }
    }
    free(zo); free(M);
  }
  free(zp); free(by_x); free(I.cam); free(I.world); cam_free(&c);
  return err ? -1 : 0;
}

/* The closed-form fit alone, on n explicit pairs (m[k], q[k]) (world
 * frame, n x 3 floats): out = (c, s, t_x, t_y). Returns 0, 1 when no turn
 * is defined, 2 with fewer than 3 pairs kept. */
int32_t or_icp_fit(const float* m, const float* q, int64_t n, double* out) {
  or_icp_sums S;
  memset(&S, 0, sizeof S);
  for (int64_t k = 0; k < n; ++k) {
    or_pt a = {m[3 * k], m[3 * k + 1], m[3 * k + 2]}, b = {q[3 * k], q[3 * k + 1], q[3 * k + 2]};
    icp_add_pair(&S, a, b);
  }
  if (S.n < 3) return 2;
  return icp_solve(&S, out, out + 1, out + 2, out + 3);
}

/* The correspondence rule alone: idx[k] = index in I (pixel order) of the
 * correspondence of world point p[k] within radius, or -1. */
int32_t or_icp_match(const or_world* w, const float* depth, const float* p, int64_t n, float radius, int64_t* idx) {
  or_cam c;
  if (cam_init(w, &c)) return -1;
  or_cloud I;
  if (observed_cloud(w, &c, depth, &I)) { cam_free(&c); return -1; }
  int64_t* by_x = order_by_x(&I);
  if (!by_x) { free(I.cam); free(I.world); cam_free(&c); return -1; }
  const double r = (double)radius;
  const float r2 = (float)(r * r);
  for (int64_t k = 0; k < n; ++k) {
    or_pt a = {p[3 * k], p[3 * k + 1], p[3 * k + 2]};
    idx[k] = icp_match(&I, by_x, a, r, r2);
  }
  free(by_x); free(I.cam); free(I.world); cam_free(&c);
  return 0;
}

int32_t or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
