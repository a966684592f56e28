/*
 * Simulated depth sensor used to make synthetic observations.
 *
 * This is input generation, not the method: it casts one ray per pixel
 * centre through a pinhole camera (double precision, Moller-Trumbore
 * ray/triangle intersection) against triangle soups already placed in the
 * world frame, and returns the camera-frame Z of the nearest hit (0 where
 * no triangle is hit). The method itself renders by z-buffer rasterisation
 * with a fixed-point snap; this ray caster shares no arithmetic with it.
 *
 * Acceleration: each object's triangles are binned into 8x8-pixel screen
 * tiles by the bounding box of their projected vertices (plus one pixel),
 * so a pixel only tests the triangles whose projection can contain it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TILE 8

static int project(const double Rcw[9], const double tcw[3], double fx, double fy,
                   double cx, double cy, const double* p, double* u, double* v) {
  double x = Rcw[0] * p[0] + Rcw[1] * p[1] + Rcw[2] * p[2] + tcw[0];
  double y = Rcw[3] * p[0] + Rcw[4] * p[1] + Rcw[5] * p[2] + tcw[1];
  double z = Rcw[6] * p[0] + Rcw[7] * p[1] + Rcw[8] * p[2] + tcw[2];
  if (!(z > 1e-6)) return 0;
  *u = fx * x / z + cx;
  *v = fy * y / z + cy;
  return 1;
}

/* T_wc: row-major 3x4 camera->world. tris: n_tri_total*9 doubles (world
 * frame, three vertices per triangle); tri_obj (may be NULL): the object id
 * of each triangle, written per pixel to obj_out (-1 = no hit) when both are
 * given. Returns 0 on success. */
int synth_raycast_ids(int W, int H, double fx, double fy, double cx, double cy,
                      const double* T_wc, const double* tris, long n_tri, const int* tri_obj,
                      double* depth_out, int* obj_out) {
  double Rwc[9] = {T_wc[0], T_wc[1], T_wc[2], T_wc[4], T_wc[5],
                   T_wc[6], T_wc[8], T_wc[9], T_wc[10]};
  double twc[3] = {T_wc[3], T_wc[7], T_wc[11]};
  double Rcw[9], tcw[3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Rcw[r * 3 + c] = Rwc[c * 3 + r];
  for (int r = 0; r < 3; ++r)
    tcw[r] = -(Rcw[r * 3 + 0] * twc[0] + Rcw[r * 3 + 1] * twc[1] + Rcw[r * 3 + 2] * twc[2]);

  int TX = (W + TILE - 1) / TILE, TY = (H + TILE - 1) / TILE;
  long n_tiles = (long)TX * TY;
  int* counts = (int*)calloc(n_tiles + 1, sizeof(int));
  int* bbox = (int*)malloc(sizeof(int) * 4 * (n_tri > 0 ? n_tri : 1));
  if (!counts || !bbox) { free(counts); free(bbox); return -1; }
  for (long t = 0; t < n_tri; ++t) {
    double umin = 1e30, umax = -1e30, vmin = 1e30, vmax = -1e30;
    int ok = 1;
    for (int k = 0; k < 3; ++k) {
      double u, v;
      if (!project(Rcw, tcw, fx, fy, cx, cy, tris + t * 9 + k * 3, &u, &v)) { ok = 0; break; }
      if (u < umin) umin = u; if (u > umax) umax = u;
      if (v < vmin) vmin = v; if (v > vmax) vmax = v;
    }
    int* b = bbox + 4 * t;
    if (!ok) { b[0] = 0; b[1] = TX - 1; b[2] = 0; b[3] = TY - 1; }
    else {
      double lo_u = floor(umin) - 1, hi_u = ceil(umax) + 1;
      double lo_v = floor(vmin) - 1, hi_v = ceil(vmax) + 1;
      if (hi_u < 0 || hi_v < 0 || lo_u > W - 1 || lo_v > H - 1) { b[0] = 1; b[1] = 0; b[2] = 1; b[3] = 0; continue; }
      if (lo_u < 0) lo_u = 0; if (lo_v < 0) lo_v = 0;
      if (hi_u > W - 1) hi_u = W - 1; if (hi_v > H - 1) hi_v = H - 1;
      b[0] = (int)lo_u / TILE; b[1] = (int)hi_u / TILE;
      b[2] = (int)lo_v / TILE; b[3] = (int)hi_v / TILE;
    }
    for (int ty = b[2]; ty <= b[3]; ++ty)
      for (int tx = b[0]; tx <= b[1]; ++tx) counts[ty * TX + tx + 1]++;
  }
  for (long i = 0; i < n_tiles; ++i) counts[i + 1] += counts[i];
  long total = counts[n_tiles];
  int* list = (int*)malloc(sizeof(int) * (total > 0 ? total : 1));
  int* cursor = (int*)malloc(sizeof(int) * n_tiles);
  if (!list || !cursor) { free(counts); free(bbox); free(list); free(cursor); return -1; }
  memcpy(cursor, counts, sizeof(int) * n_tiles);
  for (long t = 0; t < n_tri; ++t) {
    int* b = bbox + 4 * t;
    for (int ty = b[2]; ty <= b[3]; ++ty)
      for (int tx = b[0]; tx <= b[1]; ++tx) list[cursor[ty * TX + tx]++] = (int)t;
  }

#pragma omp parallel for schedule(dynamic, 4)
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      double dc[3] = {(u - cx) / fx, (v - cy) / fy, 1.0};
      double d[3];
      for (int r = 0; r < 3; ++r) d[r] = Rwc[r * 3 + 0] * dc[0] + Rwc[r * 3 + 1] * dc[1] + Rwc[r * 3 + 2] * dc[2];
      double best = INFINITY;
      int best_obj = -1;
      int tile = (v / TILE) * TX + (u / TILE);
      for (int li = counts[tile]; li < counts[tile + 1]; ++li) {
        const double* tr = tris + (long)list[li] * 9;
        double e1[3], e2[3], s[3], h[3], q[3];
        for (int r = 0; r < 3; ++r) { e1[r] = tr[3 + r] - tr[r]; e2[r] = tr[6 + r] - tr[r]; s[r] = twc[r] - tr[r]; }
        h[0] = d[1] * e2[2] - d[2] * e2[1];
        h[1] = d[2] * e2[0] - d[0] * e2[2];
        h[2] = d[0] * e2[1] - d[1] * e2[0];
        double a = e1[0] * h[0] + e1[1] * h[1] + e1[2] * h[2];
        if (fabs(a) < 1e-18) continue;
        double f = 1.0 / a;
        double bu = f * (s[0] * h[0] + s[1] * h[1] + s[2] * h[2]);
        if (bu < 0.0 || bu > 1.0) continue;
        q[0] = s[1] * e1[2] - s[2] * e1[1];
        q[1] = s[2] * e1[0] - s[0] * e1[2];
        q[2] = s[0] * e1[1] - s[1] * e1[0];
        double bv = f * (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]);
        if (bv < 0.0 || bu + bv > 1.0) continue;
        double t = f * (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]);
        if (t > 1e-6 && t < best) {
          best = t;
          best_obj = tri_obj ? tri_obj[list[li]] : 0;
        }
      }
      /* the ray direction has camera-frame z = 1, so t is camera-frame Z */
      depth_out[(long)v * W + u] = isinf(best) ? 0.0 : best;
      if (obj_out) obj_out[(long)v * W + u] = best_obj;
    }
  }
  free(counts); free(bbox); free(list); free(cursor);
  return 0;
}

int synth_raycast(int W, int H, double fx, double fy, double cx, double cy,
                  const double* T_wc, const double* tris, long n_tri, double* depth_out) {
  return synth_raycast_ids(W, H, fx, fy, cx, cy, T_wc, tris, n_tri, NULL, depth_out, NULL);
}
