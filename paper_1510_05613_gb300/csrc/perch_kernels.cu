// PERCH successor evaluation: device kernels for sm_103a.
//
// Arithmetic contract: every floating-point step on the evaluation path is a
// single IEEE binary32 operation rounded to nearest-even (__fadd_rn,
// __fmul_rn, __fmaf_rn, __frcp_rn, __int2float_rn, __float2int_rn); a fused
// multiply-add appears only where written as ffma (one rounding, as IEEE 754
// defines it) and the library is compiled with -fmad=false so nothing else is
// contracted. Coverage and z-buffer resolution are exact integer /
// order-independent min operations, so every count is bit-exact with the CPU
// oracle, which writes out the same arithmetic.
#include <climits>

#include "perch_internal.h"

namespace perch {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ int ford(float f) {  // order-preserving float -> int
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}

// squared camera-frame distance, d^2 = fma(dz, dz, fma(dy, dy, dx dx))
__device__ __forceinline__ float dist2(float px, float py, float pz, float4 q) {
  const float dx = fsub(px, q.x), dy = fsub(py, q.y), dz = fsub(pz, q.z);
  return ffma(dz, dz, ffma(dy, dy, fmul(dx, dx)));
}

// V(O) of Sec. III-A for mesh m at pose (ox, oy, yaw iyaw): the inscribed
// vertical cylinder (kind 0) or the closed-form solid (kinds 1-3), tested in
// the object frame: x' = fma(s, dy, c dx), y' = fma(c, dy, -(s dx)) with the
// pose table's (c, s); z is the world height.
__device__ __forceinline__ bool in_volume(const Geometry& g, const DevMesh& m, float ox, float oy, int iyaw,
                                          float4 qw) {
  const float dx = fsub(qw.x, ox), dy = fsub(qw.y, oy);
  if (m.vol_kind == 0) {
    const float d2 = ffma(dy, dy, fmul(dx, dx));
    return d2 <= m.vol_r2 && m.vol_zlo <= qw.z && qw.z <= m.vol_zhi;
  }
  const float2 cs = g.cs[iyaw];
  const float xo = ffma(cs.y, dy, fmul(cs.x, dx));
  const float yo = ffma(cs.x, dy, -fmul(cs.y, dx));
  if (m.vol_kind == 1)
    return fabsf(xo) <= m.vol_p[0] && fabsf(yo) <= m.vol_p[1] && m.vol_z0 <= qw.z && qw.z <= m.vol_z1;
  if (m.vol_kind == 2) {
    if (!(m.vol_z0 <= qw.z && qw.z <= m.vol_z1)) return false;
    // every face test passes inside the inscribed circle shrunk by 2^-12 in
    // r^2, and one fails outside the circumscribed circle grown by 2^-12,
    // whatever the binary32 rounding of the face tests (n <= 256 sides);
    // only the thin annulus between them needs the faces
    const float d2 = ffma(yo, yo, fmul(xo, xo));
    if (d2 <= m.vol_p[1]) return true;
    if (d2 >= m.vol_p[2]) return false;
    const float2* nr = g.vol_normals + m.vol_nrm;
    for (int k = 0; k < m.vol_n; ++k)
      if (ffma(nr[k].y, yo, fmul(nr[k].x, xo)) > m.vol_p[0]) return false;
    return true;
  }
  const float X = fmul(xo, m.vol_p[0]), Y = fmul(yo, m.vol_p[1]), Z = fmul(fsub(qw.z, m.vol_p[3]), m.vol_p[2]);
  const float t = ffma(Y, Y, fmul(X, X));
  const float z2 = fmul(Z, Z);
  const float F = m.vol_n == 2 ? ffma(t, t, fmul(z2, z2)) : fadd(t, z2);
  return F <= 1.0f;
}

struct Vtx {
  int X, Y;   // snapped pixel coordinates, 1/16 px (absolute or tile-relative)
  float iz;   // 1 / z_c; negative marks a culled vertex
};

// Camera-frame vertex (table entry M_yaw v plus the pose offset b) -> pixel:
// 1/z = 1/c_z; u = fma(fx, c_x (1/z), cx); X = rint(16 u).
__device__ __forceinline__ Vtx project_vertex(const Camera& c, float4 mv, float4 b) {
  const float xc = fadd(mv.x, b.x), yc = fadd(mv.y, b.y), zc = fadd(mv.z, b.z);
  bool bad = !(zc > kNearZ);
  const float iz = __frcp_rn(zc);
  const float u = ffma(c.fx, fmul(xc, iz), c.cx);
  const float v = ffma(c.fy, fmul(yc, iz), c.cy);
  bad = bad || !(fabsf(u) <= kGuard) || !(fabsf(v) <= kGuard);
  Vtx o;
  if (bad) {
    o.X = 0; o.Y = 0; o.iz = -1.0f;
    return o;
  }
  o.X = __float2int_rn(fmul(16.0f, u));
  o.Y = __float2int_rn(fmul(16.0f, v));
  o.iz = iz;
  return o;
}

__device__ __forceinline__ int floor16(int a) { return a >> 4; }
__device__ __forceinline__ int ceil16(int a) { return -((-a) >> 4); }

// depth at a covered pixel centre: b_i = E_i / A, 1/z = fma(b2, 1/z2,
// fma(b1, 1/z1, b0/z0)), z = 1/(1/z); returned as the float's bits
__device__ __forceinline__ uint32_t pixel_depth_bits(int w0, int w1, int w2, float invA, float iz0, float iz1,
                                                     float iz2) {
  const float b0 = fmul(__int2float_rn(w0), invA);
  const float b1 = fmul(__int2float_rn(w1), invA);
  const float b2 = fmul(__int2float_rn(w2), invA);
  const float iz = ffma(b2, iz2, ffma(b1, iz1, fmul(b0, iz0)));
  return __float_as_uint(__frcp_rn(iz));
}

// edge ownership for the top-left tie rule (front faces in this orientation)
__device__ __forceinline__ bool owns(int dx, int dy) { return dy > 0 || (dy == 0 && dx < 0); }

// Rasterise one triangle (any size) into a tile of tw x th pixels whose
// top-left pixel is at (ox16 / 16, oy16 / 16): exact edge functions, top-left
// tie rule, min-z resolve through `sink`. Used for full-image parent renders.
template <typename Sink>
__device__ __forceinline__ void raster_tri(Vtx a, Vtx b, Vtx c, int ox16, int oy16, int tw, int th,
                                           unsigned& culled, Sink sink) {
  if (a.iz < 0.0f || b.iz < 0.0f || c.iz < 0.0f) {
    culled = 1u;
    return;
  }
  const int X0 = a.X - ox16, Y0 = a.Y - oy16;
  const int X1 = b.X - ox16, Y1 = b.Y - oy16;
  const int X2 = c.X - ox16, Y2 = c.Y - oy16;
  const int xmin = min(X0, min(X1, X2)), xmax = max(X0, max(X1, X2));
  const int ymin = min(Y0, min(Y1, Y2)), ymax = max(Y0, max(Y1, Y2));
  if (xmax - xmin >= kMaxExtent || ymax - ymin >= kMaxExtent) {
    long long A64 = (long long)(Y1 - Y0) * (X2 - X0) - (long long)(X1 - X0) * (Y2 - Y0);
    if (A64 > 0) culled = 1u;
    return;
  }
  const int A = (Y1 - Y0) * (X2 - X0) - (X1 - X0) * (Y2 - Y0);
  if (A <= 0) return;  // back-facing or degenerate
  const int px0 = max(ceil16(xmin), 0), px1 = min(floor16(xmax), tw - 1);
  const int py0 = max(ceil16(ymin), 0), py1 = min(floor16(ymax), th - 1);
  if (px0 > px1 || py0 > py1) return;
  const bool own12 = owns(X2 - X1, Y2 - Y1), own20 = owns(X0 - X2, Y0 - Y2), own01 = owns(X1 - X0, Y1 - Y0);
  const float invA = __frcp_rn(__int2float_rn(A));
  for (int py = py0; py <= py1; ++py) {
    const int Py = 16 * py;
    for (int px = px0; px <= px1; ++px) {
      const int Px = 16 * px;
      const int w0 = (Y2 - Y1) * (Px - X1) - (X2 - X1) * (Py - Y1);
      const int w1 = (Y0 - Y2) * (Px - X2) - (X0 - X2) * (Py - Y2);
      const int w2 = (Y1 - Y0) * (Px - X0) - (X1 - X0) * (Py - Y0);
      const bool in = (w0 > 0 || (w0 == 0 && own12)) && (w1 > 0 || (w1 == 0 && own20)) &&
                      (w2 > 0 || (w2 == 0 && own01));
      if (in) sink(py * tw + px, pixel_depth_bits(w0, w1, w2, invA, a.iz, b.iz, c.iz));
    }
  }
}

// Eq. (1) against the observed cloud: is some observed point within delta of
// p? 3x3x3 neighbourhood of a grid whose cells are at least delta wide; three
// consecutive x-cells are one contiguous range of the bucketed array.
__device__ __forceinline__ bool explained_by_obs(const ObsIndex& o, float px, float py, float pz, float d2max) {
  if (o.n == 0) return false;
  const float fx = fmul(fsub(px, o.g3x), o.inv3);
  const float fy = fmul(fsub(py, o.g3y), o.inv3);
  const float fz = fmul(fsub(pz, o.g3z), o.inv3);
  const int ix = (int)floorf(fminf(fmaxf(fx, -2.0f), (float)o.n3x + 1.0f));
  const int iy = (int)floorf(fminf(fmaxf(fy, -2.0f), (float)o.n3y + 1.0f));
  const int iz = (int)floorf(fminf(fmaxf(fz, -2.0f), (float)o.n3z + 1.0f));
  if (ix >= 0 && ix < o.n3x && iy >= 0 && iy < o.n3y && iz >= 0 && iz < o.n3z) {
    // one bit says whether the 3x3x3 neighbourhood holds any point at all
    const int c = (iz * o.n3y + iy) * o.n3x + ix;
    if (!((__ldg(&o.dil3[c >> 5]) >> (c & 31)) & 1u)) return false;
  }
  const int x0 = max(ix - 1, 0), x1 = min(ix + 1, o.n3x - 1);
  if (x0 > x1) return false;
  for (int a = 0; a < 3; ++a) {  // the centre row first: the likeliest to hold a match
    const int cz = iz + (a == 0 ? 0 : (a == 1 ? -1 : 1));
    if (cz < 0 || cz >= o.n3z) continue;
    for (int bq = 0; bq < 3; ++bq) {
      const int cy = iy + (bq == 0 ? 0 : (bq == 1 ? -1 : 1));
      if (cy < 0 || cy >= o.n3y) continue;
      const int base = (cz * o.n3y + cy) * o.n3x;
      const int s = __ldg(&o.start3[base + x0]), e = __ldg(&o.start3[base + x1 + 1]);
      for (int k = s; k < e; ++k)
        if (dist2(px, py, pz, __ldg(&o.cam3[k])) <= d2max) return true;
    }
  }
  return false;
}

// Conservative pixel window around observed point q that contains the pixel
// of every rendered point within delta of q: for |p - q| <= delta and
// z_q > delta, |x_p/z_p - x_q/z_q| <= delta * sqrt(1 + (x_q/z_q)^2) / (z_q - delta);
// (1 + |t|) bounds the square root and one pixel of slack absorbs rounding.
__device__ __forceinline__ void delta_window(const Camera& cam, float4 q, int& u0, int& u1, int& v0, int& v1) {
  const int pix = __float_as_int(q.w);
  const int uq = pix % cam.W, vq = pix / cam.W;
  const float den = q.z - cam.delta;
  if (den > 1e-3f) {
    const float tx = fabsf(q.x / q.z), ty = fabsf(q.y / q.z);
    const float ru = fminf(cam.fx * cam.delta * (1.0f + tx) / den, 1e6f);
    const float rv = fminf(cam.fy * cam.delta * (1.0f + ty) / den, 1e6f);
    const int Ru = (int)ceilf(ru) + 1, Rv = (int)ceilf(rv) + 1;
    u0 = uq - Ru; u1 = uq + Ru; v0 = vq - Rv; v1 = vq + Rv;
  } else {
    u0 = INT_MIN / 2; u1 = INT_MAX / 2; v0 = INT_MIN / 2; v1 = INT_MAX / 2;
  }
}

// The new object's dR over its pose's box (rows of the box width): either a
// z tile with +inf off dR (mask == nullptr), or the staged render (z bits,
// with the explained flag in the sign bit) and a bitmask of dR pixels.
struct DRTile {
  const uint32_t* z;
  const uint32_t* mask;
  __device__ __forceinline__ uint32_t at(int i) const {
    if (!mask) return z[i];
    return ((mask[i >> 5] >> (i & 31)) & 1u) ? (z[i] & 0x7fffffffu) : kInfBits;
  }
};

// Eq. (1) against the new object's dR: is some rendered point within delta
// of the observed point q?
__device__ __forceinline__ bool explained_by_tile(const Camera& cam, float4 q, const DRTile& tile,
                                                  const float* rxs, const float* rys, int4 bb) {
  int u0, u1, v0, v1;
  delta_window(cam, q, u0, u1, v0, v1);
  u0 = max(u0, bb.x); u1 = min(u1, bb.x + bb.z - 1);
  v0 = max(v0, bb.y); v1 = min(v1, bb.y + bb.w - 1);
  for (int v = v0; v <= v1; ++v) {
    const int ly = v - bb.y;
    const float ry = rys[ly];
    for (int u = u0; u <= u1; ++u) {
      const int lx = u - bb.x;
      const uint32_t zb = tile.at(ly * bb.z + lx);
      if (zb == kInfBits) continue;
      const float z = __uint_as_float(zb);
      if (dist2(fmul(rxs[lx], z), fmul(ry, z), z, q) <= cam.delta2) return true;
    }
  }
  return false;
}

__device__ __forceinline__ int warp_sum(int v) { return __reduce_add_sync(0xffffffffu, v); }

// ------------------------------------------------------------------ utility
__global__ void k_fill_u32(uint32_t* p, uint32_t v, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) p[i] = v;
}

cudaError_t launch_fill_u32(uint32_t* p, uint32_t v, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_fill_u32<<<(unsigned)blocks, 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

// exclusive scan: out[0..n] with out[n] = total. 1024 elements per block.
__global__ void k_scan_blocks(const int* in, int* out, int n, int* block_sums) {
  __shared__ int warp_tot[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = blockIdx.x * 1024 + tid * 4;
  int v[4], s = 0;
  for (int k = 0; k < 4; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int incl = s;
  for (int d = 1; d < 32; d <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int woff = 0;
  for (int w = 0; w < warp; ++w) woff += warp_tot[w];
  int run = woff + incl - s;
  for (int k = 0; k < 4; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (tid == 255) block_sums[blockIdx.x] = woff + incl;
}

__global__ void k_scan_single(int* sums, int nb, int* total_out) {
  __shared__ int carry_s;
  __shared__ int warp_tot[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (int off = 0; off < nb; off += 1024) {
    int i = off + tid;
    int v = (i < nb) ? sums[i] : 0;
    int incl = v;
    for (int d = 1; d < 32; d <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int woff = 0;
    for (int w = 0; w < warp; ++w) woff += warp_tot[w];
    int carry = carry_s;
    if (i < nb) sums[i] = carry + woff + incl - v;
    __syncthreads();
    if (tid == 1023) carry_s = carry + woff + incl;
    __syncthreads();
  }
  if (tid == 0) *total_out = carry_s;
}

__global__ void k_scan_add(int* out, int n, const int* block_offsets) {
  const int base = blockIdx.x * 1024;
  const int add = block_offsets[blockIdx.x];
  for (int k = threadIdx.x; k < 1024; k += blockDim.x)
    if (base + k < n) out[base + k] += add;
}

cudaError_t launch_exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s) {
  int nb = (n + 1023) / 1024;
  if (nb == 0) nb = 1;
  k_scan_blocks<<<nb, 256, 0, s>>>(in, out, n, tmp);
  k_scan_single<<<1, 1024, 0, s>>>(tmp, nb, out + n);
  k_scan_add<<<nb, 256, 0, s>>>(out, n, tmp);
  return cudaGetLastError();
}

// ------------------------------------------------------- observation prep
__device__ __forceinline__ bool depth_valid(float d) { return d > 0.0f && isfinite(d); }

__global__ void k_obs_count(const float* depth, int n, int* block_counts) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  const bool ok = i < n && depth_valid(depth[i]);
  int c = __syncthreads_count(ok);
  if (threadIdx.x == 0) block_counts[blockIdx.x] = c;
}

cudaError_t launch_obs_count(const float* depth, int W, int H, int* block_counts, cudaStream_t s) {
  const int n = W * H;
  k_obs_count<<<(n + 255) / 256, 256, 0, s>>>(depth, n, block_counts);
  return cudaGetLastError();
}

// back-project valid pixels (observed cloud I) in pixel order, camera and
// world frames; accumulate bounding boxes for the grids
__global__ void k_obs_write(const float* depth, Camera cam, const float* rx, const float* ry,
                            const int* block_offsets, float4* cam_pts, float4* world_pts, int* bounds) {
  __shared__ int warp_cnt[8];
  const int n = cam.W * cam.H;
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float d = i < n ? depth[i] : 0.0f;
  const bool ok = i < n && depth_valid(d);
  const unsigned bal = __ballot_sync(0xffffffffu, ok);
  if (lane == 0) warp_cnt[warp] = __popc(bal);
  __syncthreads();
  int off = block_offsets[blockIdx.x];
  for (int w = 0; w < warp; ++w) off += warp_cnt[w];
  off += __popc(bal & ((1u << lane) - 1u));
  if (!ok) return;
  const int u = i % cam.W, v = i / cam.W;
  const float x = fmul(rx[u], d), y = fmul(ry[v], d), z = d;
  const float xw = fadd(ffma(cam.Rwc[2], z, ffma(cam.Rwc[1], y, fmul(cam.Rwc[0], x))), cam.twc[0]);
  const float yw = fadd(ffma(cam.Rwc[5], z, ffma(cam.Rwc[4], y, fmul(cam.Rwc[3], x))), cam.twc[1]);
  const float zw = fadd(ffma(cam.Rwc[8], z, ffma(cam.Rwc[7], y, fmul(cam.Rwc[6], x))), cam.twc[2]);
  cam_pts[off] = make_float4(x, y, z, __int_as_float(i));
  world_pts[off] = make_float4(xw, yw, zw, 0.0f);
  atomicMin(&bounds[0], ford(x)); atomicMin(&bounds[1], ford(y)); atomicMin(&bounds[2], ford(z));
  atomicMax(&bounds[3], ford(x)); atomicMax(&bounds[4], ford(y)); atomicMax(&bounds[5], ford(z));
  atomicMin(&bounds[6], ford(xw)); atomicMin(&bounds[7], ford(yw));
  atomicMax(&bounds[8], ford(xw)); atomicMax(&bounds[9], ford(yw));
}

cudaError_t launch_obs_write(const float* depth, const Camera& cam, const float* rx, const float* ry,
                             const int* block_offsets, float4* cam_pts, float4* world_pts, int* bounds,
                             cudaStream_t s) {
  const int n = cam.W * cam.H;
  k_obs_write<<<(n + 255) / 256, 256, 0, s>>>(depth, cam, rx, ry, block_offsets, cam_pts, world_pts, bounds);
  return cudaGetLastError();
}

__device__ __forceinline__ int cell_of(float x, float g, float inv, int n) {
  const float f = fmul(fsub(x, g), inv);
  int c = (int)floorf(fminf(fmaxf(f, -2.0f), (float)n + 1.0f));
  return c;
}

__device__ __forceinline__ int sat_sum(const int* S, int cols, int r0, int r1, int c0, int c1) {  // inclusive
  const int w = cols + 1;
  return S[(r1 + 1) * w + c1 + 1] - S[r0 * w + c1 + 1] - S[(r1 + 1) * w + c0] + S[r0 * w + c0];
}

// Could some observed point lie within delta of a point that object o
// renders? No, when the world (x, y) cells around its footprint disk (radius
// fp_r, plus delta, plus 2 cm for the rounding of the back-projected depth,
// plus a cell either side) hold no point: every rendered point lies within
// that disk horizontally, and Eq. (1) bounds the 3D distance, hence the
// horizontal one (the grid covers the whole cloud, so a disk beyond its
// cells holds none).
__device__ __forceinline__ bool obs_near(const Camera& cam, const Geometry& g, const ObsIndex& obs,
                                         const perch_obj& o) {
  if (obs.n == 0) return false;
  const float R = g.meshes[o.mesh].fp_r + cam.delta + 0.02f;
  const float ox = g.xs[o.ix], oy = g.ys[o.iy];
  const int cx0 = max(cell_of(ox - R, obs.g2x, obs.inv2, obs.n2x) - 1, 0);
  const int cx1 = min(cell_of(ox + R, obs.g2x, obs.inv2, obs.n2x) + 1, obs.n2x - 1);
  const int cy0 = max(cell_of(oy - R, obs.g2y, obs.inv2, obs.n2y) - 1, 0);
  const int cy1 = min(cell_of(oy + R, obs.g2y, obs.inv2, obs.n2y) + 1, obs.n2y - 1);
  return cx0 <= cx1 && cy0 <= cy1 && sat_sum(obs.sat2, obs.n2x, cy0, cy1, cx0, cx1) != 0;
}

__global__ void k_grid3_keys(const float4* pts, int n, float gx, float gy, float gz, float inv, int nx, int ny,
                             int nz, int* keys, int* counts) {
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (k >= n) return;
  const float4 p = pts[k];
  const int ix = min(max(cell_of(p.x, gx, inv, nx), 0), nx - 1);
  const int iy = min(max(cell_of(p.y, gy, inv, ny), 0), ny - 1);
  const int iz = min(max(cell_of(p.z, gz, inv, nz), 0), nz - 1);
  const int key = (iz * ny + iy) * nx + ix;
  keys[k] = key;
  atomicAdd(&counts[key], 1);
}

cudaError_t launch_grid3_keys(const float4* cam_pts, int n, float g3x, float g3y, float g3z, float inv3, int n3x,
                              int n3y, int n3z, int* keys, int* counts, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_grid3_keys<<<(n + 255) / 256, 256, 0, s>>>(cam_pts, n, g3x, g3y, g3z, inv3, n3x, n3y, n3z, keys, counts);
  return cudaGetLastError();
}

__global__ void k_grid2_keys(const float4* pts, int n, float gx, float gy, float inv, int nx, int ny, int* keys,
                             int* counts) {
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (k >= n) return;
  const float4 p = pts[k];
  const int ix = min(max(cell_of(p.x, gx, inv, nx), 0), nx - 1);
  const int iy = min(max(cell_of(p.y, gy, inv, ny), 0), ny - 1);
  const int key = iy * nx + ix;
  keys[k] = key;
  atomicAdd(&counts[key], 1);
}

cudaError_t launch_grid2_keys(const float4* world_pts, int n, float g2x, float g2y, float inv2, int n2x, int n2y,
                              int* keys, int* counts, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_grid2_keys<<<(n + 255) / 256, 256, 0, s>>>(world_pts, n, g2x, g2y, inv2, n2x, n2y, keys, counts);
  return cudaGetLastError();
}

__global__ void k_scatter(const int* keys, int n, int* cursor, const float4* a_in, float4* a_out,
                          const float4* b_in, float4* b_out) {
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (k >= n) return;
  const int pos = atomicAdd(&cursor[keys[k]], 1);
  a_out[pos] = a_in[k];
  if (b_in) b_out[pos] = b_in[k];
}

cudaError_t launch_scatter(const int* keys, int n, int* cursor, const float4* a_in, float4* a_out,
                           const float4* b_in, float4* b_out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_scatter<<<(n + 255) / 256, 256, 0, s>>>(keys, n, cursor, a_in, a_out, b_in, b_out);
  return cudaGetLastError();
}

// ray slopes rx[u] = (u - cx) / fx, ry[v] = (v - cy) / fy in double, rounded once
__global__ void k_rays(Camera cam, float* rx, float* ry) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i < cam.W) rx[i] = (float)__ddiv_rn(__dsub_rn((double)i, (double)cam.cx), (double)cam.fx);
  if (i < cam.H) ry[i] = (float)__ddiv_rn(__dsub_rn((double)i, (double)cam.cy), (double)cam.fy);
}

cudaError_t launch_rays(const Camera& cam, float* rx, float* ry, cudaStream_t s) {
  const int n = cam.W > cam.H ? cam.W : cam.H;
  k_rays<<<(n + 255) / 256, 256, 0, s>>>(cam, rx, ry);
  return cudaGetLastError();
}

// dilated occupancy of the 3D grid: bit c set iff a cell within one step of
// c (in each axis) holds a point; dil3 must be zeroed first
__global__ void k_dilate3(const int* start3, int nx, int ny, int nz, uint32_t* dil3) {
  const long long c = blockIdx.x * 256LL + threadIdx.x;
  const long long n = (long long)nx * ny * nz;
  if (c >= n) return;
  const int ix = (int)(c % nx), iy = (int)((c / nx) % ny), iz = (int)(c / ((long long)nx * ny));
  bool any = false;
  for (int dz = -1; dz <= 1 && !any; ++dz) {
    const int z = iz + dz;
    if (z < 0 || z >= nz) continue;
    for (int dy = -1; dy <= 1 && !any; ++dy) {
      const int y = iy + dy;
      if (y < 0 || y >= ny) continue;
      const int base = (z * ny + y) * nx;
      const int x0 = max(ix - 1, 0), x1 = min(ix + 1, nx - 1);
      any = start3[base + x1 + 1] > start3[base + x0];
    }
  }
  if (any) atomicOr(&dil3[c >> 5], 1u << (c & 31));
}

cudaError_t launch_dilate3(const int* start3, int n3x, int n3y, int n3z, uint32_t* dil3, cudaStream_t s) {
  const long long n = (long long)n3x * n3y * n3z;
  if (n == 0) return cudaSuccess;
  k_dilate3<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(start3, n3x, n3y, n3z, dil3);
  return cudaGetLastError();
}
// Camera-frame pose tables: per yaw M = R_cw Rz(yaw), per (ix, iy)
// b = R_cw (x, y, 0) + t_cw, in double from the binary32 inputs (products of
// two floats are exact in double), rounded once.
__global__ void k_pose_tables(Camera cam, Geometry g, float* yaw_mats, float4* pose_off) {
  const int t = blockIdx.x * 256 + threadIdx.x;
  if (t < g.n_yaw) {
    const double cs = g.cs[t].x, sn = g.cs[t].y;
    for (int r = 0; r < 3; ++r) {
      const double r0 = cam.Rcw[r * 3 + 0], r1 = cam.Rcw[r * 3 + 1];
      yaw_mats[t * 9 + r * 3 + 0] = __double2float_rn(__dadd_rn(__dmul_rn(r0, cs), __dmul_rn(r1, sn)));
      yaw_mats[t * 9 + r * 3 + 1] = __double2float_rn(__dsub_rn(__dmul_rn(r1, cs), __dmul_rn(r0, sn)));
      yaw_mats[t * 9 + r * 3 + 2] = cam.Rcw[r * 3 + 2];
    }
  }
  if (t < g.nx * g.ny) {
    const double x = g.xs[t / g.ny], y = g.ys[t % g.ny];
    float b[3];
    for (int r = 0; r < 3; ++r) {
      const double r0 = cam.Rcw[r * 3 + 0], r1 = cam.Rcw[r * 3 + 1];
      b[r] = __double2float_rn(__dadd_rn(__dadd_rn(__dmul_rn(r0, x), __dmul_rn(r1, y)), (double)cam.tcw[r]));
    }
    pose_off[t] = make_float4(b[0], b[1], b[2], 0.0f);
  }
}

// per (yaw, chunk vertex): M v = fma(M_r2, vz, fma(M_r1, vy, M_r0 vx)) per row
__global__ void k_vertex_table(Geometry g, const float* yaw_mats, float4* vtab) {
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t >= (long long)g.n_yaw * g.n_cverts) return;
  const int k = (int)(t / g.n_cverts), j = (int)(t % g.n_cverts);
  const float* M = yaw_mats + 9 * k;
  const float4 v = g.chunk_verts[j];
  float o[3];
  for (int r = 0; r < 3; ++r) o[r] = ffma(M[r * 3 + 2], v.z, ffma(M[r * 3 + 1], v.y, fmul(M[r * 3 + 0], v.x)));
  vtab[t] = make_float4(o[0], o[1], o[2], 0.0f);
}

cudaError_t launch_pose_tables(const Camera& cam, const Geometry& g, float* yaw_mats, float4* pose_off,
                               float4* vtab, cudaStream_t s) {
  const int n = g.n_yaw > g.nx * g.ny ? g.n_yaw : g.nx * g.ny;
  k_pose_tables<<<(n + 255) / 256, 256, 0, s>>>(cam, g, yaw_mats, pose_off);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long nv = (long long)g.n_yaw * g.n_cverts;
  if (nv == 0) return cudaSuccess;
  k_vertex_table<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(g, yaw_mats, vtab);
  return cudaGetLastError();
}

// conservative screen box of every (mesh, pose) from the 8 corners of the
// mesh's bounding box (a convex hull of its vertices), plus one pixel;
// bad: 1 = a corner at or behind the near plane or far off-screen,
// 2 = the unclipped box is wider or taller than kMaxObjectPixels
__global__ void k_pose_bbox(Camera cam, Geometry g, const float* yaw_mats, int4* bbox, int* max_wh, int* bad_any) {
  const long long n = (long long)g.n_mesh * g.nx * g.ny * g.n_yaw;
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t >= n) return;
  const int iyaw = (int)(t % g.n_yaw);
  const int iy = (int)((t / g.n_yaw) % g.ny);
  const int ix = (int)((t / ((long long)g.n_yaw * g.ny)) % g.nx);
  const int m = (int)(t / ((long long)g.n_yaw * g.ny * g.nx));
  const DevMesh dm = g.meshes[m];
  const float* M = yaw_mats + 9 * iyaw;
  const float4 b = g.pose_off[ix * g.ny + iy];
  float umin = 1e30f, umax = -1e30f, vmin = 1e30f, vmax = -1e30f;
  bool bad = false;
  for (int k = 0; k < 8; ++k) {
    const float vx = (k & 1) ? dm.hi[0] : dm.lo[0];
    const float vy = (k & 2) ? dm.hi[1] : dm.lo[1];
    const float vz = (k & 4) ? dm.hi[2] : dm.lo[2];
    const float xc = M[0] * vx + M[1] * vy + M[2] * vz + b.x;
    const float yc = M[3] * vx + M[4] * vy + M[5] * vz + b.y;
    const float zc = M[6] * vx + M[7] * vy + M[8] * vz + b.z;
    if (!(zc > kNearZ)) { bad = true; break; }
    const float u = cam.fx * (xc / zc) + cam.cx, v = cam.fy * (yc / zc) + cam.cy;
    umin = fminf(umin, u); umax = fmaxf(umax, u);
    vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
  }
  int4 r;
  if (bad || !(umax - umin < 4096.0f) || !(vmax - vmin < 4096.0f)) {
    r = make_int4(0, 0, cam.W, cam.H);
    atomicOr(bad_any, 1);
  } else {
    if (umax - umin > (float)(kMaxObjectPixels - 4) || vmax - vmin > (float)(kMaxObjectPixels - 4))
      atomicOr(bad_any, 2);
    int x0 = (int)floorf(fmaxf(umin, -8.0f)) - 1, x1 = (int)ceilf(fminf(umax, (float)cam.W + 8.0f)) + 1;
    int y0 = (int)floorf(fmaxf(vmin, -8.0f)) - 1, y1 = (int)ceilf(fminf(vmax, (float)cam.H + 8.0f)) + 1;
    x0 = max(x0, 0); y0 = max(y0, 0);
    x1 = min(x1, cam.W - 1); y1 = min(y1, cam.H - 1);
    if (x0 > x1 || y0 > y1) r = make_int4(0, 0, 0, 0);
    else r = make_int4(x0, y0, x1 - x0 + 1, y1 - y0 + 1);
  }
  bbox[t] = r;
  atomicMax(&max_wh[2 * m], r.z);  // per-mesh tile
  atomicMax(&max_wh[2 * m + 1], r.w);
}

cudaError_t launch_pose_bbox(const Camera& cam, const Geometry& g, const float* yaw_mats, int4* bbox, int* max_wh,
                             int* bad, cudaStream_t s) {
  const long long n = (long long)g.n_mesh * g.nx * g.ny * g.n_yaw;
  if (n == 0) return cudaSuccess;
  k_pose_bbox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cam, g, yaw_mats, bbox, max_wh, bad);
  return cudaGetLastError();
}

// ------------------------------------------------------------ parent prep
struct GlobalSink {
  uint32_t* z;
  __device__ __forceinline__ void operator()(int idx, uint32_t zbits) const { atomicMin(&z[idx], zbits); }
};

__device__ __forceinline__ bool obj_ok(const Geometry& g, const perch_obj& o) {
  return o.mesh < g.n_mesh && o.ix >= 0 && o.ix < g.nx && o.iy >= 0 && o.iy < g.ny && o.iyaw < g.n_yaw;
}

// z-buffer render of every parent's objects (R_j) into its own full image.
// Block = one chunk of one (parent, object) pair.
__global__ void __launch_bounds__(256) k_render_parents(Camera cam, Geometry g, Batch b,
                                                        unsigned long long* culled_total) {
  __shared__ int2 sXY[kChunkMaxVerts];
  __shared__ float sIZ[kChunkMaxVerts];
  const int item = blockIdx.y;
  const int p = item / b.parent_stride, k = item % b.parent_stride;
  if (p >= b.n_par) return;
  const int plen = b.parent_len[p];
  if (k >= plen || plen > b.parent_stride) return;
  const perch_obj o = b.parents[(long long)p * b.parent_stride + k];
  if (!obj_ok(g, o)) return;
  const DevMesh m = g.meshes[o.mesh];
  if ((int)blockIdx.x >= m.chunk_count) return;
  const int4 ci = g.chunk_info[m.chunk_begin + blockIdx.x];
  const float4 bo = g.pose_off[o.ix * g.ny + o.iy];
  const float4* V = g.vtab + (size_t)o.iyaw * g.n_cverts;
  for (int v = threadIdx.x; v < ci.y; v += 256) {
    const Vtx r = project_vertex(cam, V[ci.x + v], bo);
    sXY[v] = make_int2(r.X, r.Y);
    sIZ[v] = r.iz;
  }
  __syncthreads();
  unsigned culled = 0;
  uint32_t* z = reinterpret_cast<uint32_t*>(b.parent_z) + (size_t)p * cam.W * cam.H;
  for (int t = threadIdx.x; t < ci.w; t += 256) {
    const uint32_t pk = g.chunk_tris[ci.z + t];
    const int i0 = pk & 1023, i1 = (pk >> 10) & 1023, i2 = (pk >> 20) & 1023;
    raster_tri(Vtx{sXY[i0].x, sXY[i0].y, sIZ[i0]}, Vtx{sXY[i1].x, sXY[i1].y, sIZ[i1]},
               Vtx{sXY[i2].x, sXY[i2].y, sIZ[i2]}, 0, 0, cam.W, cam.H, culled, GlobalSink{z});
  }
  if (culled_total) {
    const int c = __syncthreads_count(culled != 0);
    if (threadIdx.x == 0 && c) atomicAdd(culled_total, (unsigned long long)c);
  }
}

cudaError_t launch_render_parents(const Camera& cam, const Geometry& g, const Batch& b, int max_chunks,
                                  unsigned long long* culled, cudaStream_t s) {
  if (b.n_par == 0 || b.parent_stride == 0 || max_chunks == 0) return cudaSuccess;
  const long long items = (long long)b.n_par * b.parent_stride;
  if (items > 65535) return cudaErrorInvalidValue;
  dim3 grid(max_chunks, (unsigned)items);
  k_render_parents<<<grid, 256, 0, s>>>(cam, g, b, culled);
  return cudaGetLastError();
}

// U set of a parent one object short of a complete scene:
// U = {q in I - V_{K-1} : q unexplained by R_{K-1}}; then for the last object
// O_K, residual(K) = #{q in U : q not in V(O_K), q unexplained by dR_K}.
__global__ void k_uset(Camera cam, Geometry g, ObsIndex obs0, Batch b) {
  const int p = blockIdx.y;
  const int plen = b.parent_len[p];
  const int K_total = b.parent_K ? b.parent_K[p] : b.K_total;
  if (plen + 1 != K_total || plen > b.parent_stride) return;
  const int scene = b.parent_scene ? b.parent_scene[p] : 0;
  if (b.parent_scene && (scene < 0 || scene >= b.n_scenes)) return;
  const ObsIndex& obs = b.parent_scene ? b.scenes[scene] : obs0;
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (k >= obs.n) return;
  const float4 qw = obs.world2[k];
  for (int j = 0; j < plen; ++j) {
    const perch_obj o = b.parents[(long long)p * b.parent_stride + j];
    if (!obj_ok(g, o)) return;
    const DevMesh m = g.meshes[o.mesh];
    if (in_volume(g, m, g.xs[o.ix], g.ys[o.iy], o.iyaw, qw)) return;
  }
  const float4 q = obs.cam2[k];
  if (plen > 0) {
    const float* zp = b.parent_z + (size_t)p * cam.W * cam.H;
    int u0, u1, v0, v1;
    delta_window(cam, q, u0, u1, v0, v1);
    u0 = max(u0, 0); u1 = min(u1, cam.W - 1);
    v0 = max(v0, 0); v1 = min(v1, cam.H - 1);
    for (int v = v0; v <= v1; ++v) {
      const float ry = g.ry[v];
      for (int u = u0; u <= u1; ++u) {
        const float z = zp[(size_t)v * cam.W + u];
        if (__float_as_uint(z) == kInfBits) continue;
        if (dist2(fmul(g.rx[u], z), fmul(ry, z), z, q) <= cam.delta2) return;
      }
    }
  }
  const int slot = atomicAdd(&b.uset_count[p], 1);
  b.uset[(size_t)p * b.uset_stride + slot] = k;
}

cudaError_t launch_uset(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                        cudaStream_t s) {
  const int n_max = b.parent_scene ? b.uset_stride : obs.n;  // the largest cloud of the batch's scenes
  if (b.n_par == 0 || n_max == 0) return cudaSuccess;
  if (b.n_par > 65535) return cudaErrorInvalidValue;
  dim3 grid((n_max + 255) / 256, b.n_par);
  k_uset<<<grid, 256, 0, s>>>(cam, g, obs, b);
  return cudaGetLastError();
}

// ------------------------------------------------------------- evaluation
size_t eval_smem_bytes(int tile_w, int tile_h) {
  return (size_t)kChunkMaxVerts * 16 + (size_t)kChunkMaxTris * 4 + (size_t)kChunkMaxVerts * 8 +
         (size_t)kBigQueue * 8 + (size_t)tile_w * tile_h * 4 + (size_t)(tile_w + tile_h) * 4;
}

bool eval_tile_fits(int device, int tile_w, int tile_h) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return false;
  return eval_smem_bytes(tile_w, tile_h) + 256 <= (size_t)optin;  // 256: static shared memory of k_eval
}

// ---- bulk asynchronous copies (TMA, 1D) into shared memory, with mbarriers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one thread: announce `bytes` of transfer and start the copy gmem -> smem
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase with the given parity. Each poll may suspend the thread
// in hardware (up to 0.1 ms) instead of spinning; the wait gives up after
// `polls` polls or 2 s, whichever comes first, and then returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int polls = kWaitSpins) {
  const uint64_t t0 = global_ns();
  for (int i = 0; i < polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(100000u)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > 2000000000ull) break;
  }
  return false;
}

__device__ __forceinline__ uint32_t pack_xy(int X, int Y) { return (uint32_t)(X & 0xffff) | ((uint32_t)Y << 16); }
__device__ __forceinline__ int2 unpack_xy(uint32_t p) { return make_int2((int)(p << 16) >> 16, (int)p >> 16); }

// Is the pixel centre with edge values (w0, w1, w2) inside the triangle
// under the top-left rule? Exact zeros (rare) look at the edge directions.
__device__ __forceinline__ bool covers(int w0, int w1, int w2, int2 a, int2 b, int2 c) {
  if ((w0 | w1 | w2) < 0) return false;  // strictly outside some edge
  if (w0 == 0 && !owns(c.x - b.x, c.y - b.y)) return false;
  if (w1 == 0 && !owns(a.x - c.x, a.y - c.y)) return false;
  if (w2 == 0 && !owns(b.x - a.x, b.y - a.y)) return false;
  return true;
}

// 1/z at a covered pixel centre: b_i = E_i (1/A), 1/z = fma(b2, 1/z2,
// fma(b1, 1/z1, b0/z0)). The tile keeps the largest 1/z (the nearest
// surface; z = 1/(1/z) is taken once per pixel afterwards).
__device__ __forceinline__ uint32_t pixel_iz_bits(int w0, int w1, int w2, float invA, float iz0, float iz1, float iz2) {
  const float b0 = fmul(__int2float_rn(w0), invA);
  const float b1 = fmul(__int2float_rn(w1), invA);
  const float b2 = fmul(__int2float_rn(w2), invA);
  return __float_as_uint(ffma(b2, iz2, ffma(b1, iz1, fmul(b0, iz0))));
}

// Test the candidate pixel centres [px0, px1] x [py0, py1] of a front-facing
// triangle (tile-relative 1/16-px vertices) and max its 1/z into the tile.
__device__ __forceinline__ void raster_box(int2 a, int2 b, int2 c, int A, int px0, int px1, int py0, int py1,
                                           const float* sIZ, int i0, int i1, int i2, uint32_t* tile, int tw) {
  // edge functions at the first candidate, then stepped by their exact
  // integer increments per pixel (16 sub-pixel units)
  const float invA = __frcp_rn(__int2float_rn(A));
  const int d0x = 16 * (c.y - b.y), d0y = -16 * (c.x - b.x);
  const int d1x = 16 * (a.y - c.y), d1y = -16 * (a.x - c.x);
  const int d2x = 16 * (b.y - a.y), d2y = -16 * (b.x - a.x);
  int r0 = (c.y - b.y) * (16 * px0 - b.x) - (c.x - b.x) * (16 * py0 - b.y);
  int r1 = (a.y - c.y) * (16 * px0 - c.x) - (a.x - c.x) * (16 * py0 - c.y);
  int r2 = (b.y - a.y) * (16 * px0 - a.x) - (b.x - a.x) * (16 * py0 - a.y);
  const float z0 = sIZ[i0], z1 = sIZ[i1], z2 = sIZ[i2];
  for (int py = py0; py <= py1; ++py) {
    int w0 = r0, w1 = r1, w2 = r2;
    for (int px = px0; px <= px1; ++px) {
      if (covers(w0, w1, w2, a, b, c))
        atomicMax(&tile[py * tw + px], pixel_iz_bits(w0, w1, w2, invA, z0, z1, z2));
      w0 += d0x;
      w1 += d1x;
      w2 += d2x;
    }
    r0 += d0y;
    r1 += d1y;
    r2 += d2y;
  }
}

struct EvalShared {
  uint64_t* bar;   // [0]: vertex slice, [1]: triangle list
  int* cnt;        // viol, n_new, culled, djr, djo, resid, n_vol
  int* qn;         // queued larger triangles
  unsigned char* dyn;
  uint32_t pv, pt;  // parity of the next phase of each barrier
};

// Outcome of one render or evaluation: done; a bounded wait gave up but
// every copy it was waiting for has landed since (the record carries
// kFlagTimeout and the CTA may go on); or a copy may still be in flight (the
// CTA must stop).
enum EvalStatus { kEvalDone = 0, kEvalTimedOut = 1, kEvalStop = 2 };

// Dynamic shared memory of a render: the chunk buffers (vertex-table slice,
// triangle list, projected vertices, queue of larger triangles), then the
// tile (rows of the pose's box width). Only vbuf and tbuf receive bulk
// copies; threads never write them.
struct RenderSmem {
  float4* vbuf;
  uint32_t* tbuf;
  uint32_t* sXY;
  float* sIZ;
  uint32_t* queue;  // (triangle, box) pairs
  uint32_t* tile;
};

__device__ __forceinline__ RenderSmem render_smem(unsigned char* smem) {
  RenderSmem s;
  s.vbuf = reinterpret_cast<float4*>(smem);
  s.tbuf = reinterpret_cast<uint32_t*>(s.vbuf + kChunkMaxVerts);
  s.sXY = s.tbuf + kChunkMaxTris;
  s.sIZ = reinterpret_cast<float*>(s.sXY + kChunkMaxVerts);
  s.queue = reinterpret_cast<uint32_t*>(s.sIZ + kChunkMaxVerts);
  s.tile = s.queue + 2 * kBigQueue;
  return s;
}

size_t render_smem_bytes(int tile_w, int tile_h) {
  return (size_t)kChunkMaxVerts * 16 + (size_t)kChunkMaxTris * 4 + (size_t)kChunkMaxVerts * 8 +
         (size_t)kBigQueue * 8 + (size_t)tile_w * tile_h * 4;
}

size_t cost_smem_bytes(int tile_w, int tile_h, int stages) {  // stages, dR bitmask (16-byte multiples), rays
  return (size_t)stages * ((tile_w * tile_h + 3) & ~3) * 4 + (size_t)(((tile_w * tile_h + 31) / 32 + 3) & ~3) * 4 +
         (size_t)(tile_w + tile_h) * 4;
}

// thread 0: start the bulk copies of the first chunk of mesh m at yaw iyaw
__device__ __forceinline__ void render_start(const Geometry& g, const DevMesh& m, int iyaw, const RenderSmem& s,
                                             uint64_t* bar) {
  const float4* V = g.vtab + (size_t)iyaw * g.n_cverts;
  const int4 ci = g.chunk_info[m.chunk_begin];
  bulk_load(s.vbuf, V + ci.x, (uint32_t)ci.y * 16u, &bar[0]);
  bulk_load(s.tbuf, g.chunk_tris + ci.z, (uint32_t)((ci.w + 3) & ~3) * 4u, &bar[1]);
}

// Render mesh m at pose o into the tile (1/z bits, 0 = empty) covering the
// pose's screen box bb. The first chunk's copies must have been started
// (render_start) and the tile cleared before the call; the first CTA barrier
// inside orders those writes.
//
// The mesh is walked in chunks of <= 512 vertices / 1024 triangles. A chunk's
// camera-frame vertex table slice (M_yaw v) and its triangle list are
// brought into shared memory by bulk asynchronous copies (TMA); the copy of
// chunk c+1's vertices is issued as soon as chunk c's vertices are projected,
// and the copy of its triangles as soon as chunk c's triangles are set up, so
// the loads overlap the rasterisation. Each thread sets up triangles; a
// front-facing triangle whose box holds at most INL pixel centres (the inline
// limit, a launch parameter the autotuner picks) is rasterised by its thread,
// a larger one is queued and its pixel centres are split across a warp; a full
// queue falls back to the thread. Coverage resolves by an order-independent
// max, so the tile does not depend on INL. Edge arithmetic stays in int32: every object's
// screen box is at most kMaxObjectPixels wide (checked at set-up), so
// tile-relative coordinates (kept as int16 pairs) and all edge-function
// values are far below 2^31. `culled` is set in the threads that dropped a
// triangle. On kEvalTimedOut / kEvalStop the tile is incomplete; the caller
// reports the failure and must pass a CTA barrier before reusing the tile.
template <int NT, int INL>
__device__ __forceinline__ int render_chunks(const Camera& cam, const Geometry& g, const Batch& b, const DevMesh& m,
                                             const perch_obj& o, int4 bb, const RenderSmem& s, EvalShared& sh,
                                             unsigned& culled, int4& cov) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t* s_bar = sh.bar;
  int& s_qn = *sh.qn;
  float4* vbuf = s.vbuf;
  uint32_t* tbuf = s.tbuf;
  uint32_t* sXY = s.sXY;
  float* sIZ = s.sIZ;
  uint32_t* queue = s.queue;
  uint32_t* tile = s.tile;
  const int tw = bb.z, th = bb.w;
  const float4* V = g.vtab + (size_t)o.iyaw * g.n_cverts;
  const float4 bo = g.pose_off[o.ix * g.ny + o.iy];
  const int ox16 = 16 * bb.x, oy16 = 16 * bb.y;
  uint32_t& pv = sh.pv;
  uint32_t& pt = sh.pt;
  const int qcap = b.queue_cap > 0 && b.queue_cap < kBigQueue ? b.queue_cap : kBigQueue;
  bool v_pending = true, t_pending = true;  // a copy in flight on that barrier
  bool timed_out = false;
  for (int c = 0; c < m.chunk_count; ++c) {
    const int4 ci = g.chunk_info[m.chunk_begin + c];
    // vertices: wait for the slice, project, then reuse its buffer for c+1
    const bool vok = mbar_wait(&s_bar[0], pv, b.wait_polls);
    int bad = 0;
    if (vok) {
      for (int v = tid; v < ci.y; v += NT) {
        const Vtx r = project_vertex(cam, vbuf[v], bo);
        sXY[v] = pack_xy(r.X - ox16, r.Y - oy16);
        sIZ[v] = r.iz;
        bad |= r.iz < 0.0f;
      }
    }
    if (tid == 0) s_qn = 0;
    const int vflags = __syncthreads_or(bad | (vok ? 0 : 2));
    if (vflags & 2) {
      timed_out = true;
      break;
    }
    pv ^= 1u;
    v_pending = false;
    if (c + 1 < m.chunk_count) {
      if (tid == 0) {
        const int4 cn = g.chunk_info[m.chunk_begin + c + 1];
        bulk_load(vbuf, V + cn.x, (uint32_t)cn.y * 16u, &s_bar[0]);
      }
      v_pending = true;
    }
    // triangles
    const bool tok = mbar_wait(&s_bar[1], pt, b.wait_polls);
    if (tok) {
      for (int t = tid; t < ci.w; t += NT) {
        const uint32_t pk = tbuf[t];
        const int i0 = pk & 1023, i1 = (pk >> 10) & 1023, i2 = (pk >> 20) & 1023;
        if ((vflags & 1) && (sIZ[i0] < 0.0f || sIZ[i1] < 0.0f || sIZ[i2] < 0.0f)) {
          culled = 1u;
          continue;
        }
        const int2 va = unpack_xy(sXY[i0]), vb = unpack_xy(sXY[i1]), vc = unpack_xy(sXY[i2]);
        const int A = (vb.y - va.y) * (vc.x - va.x) - (vb.x - va.x) * (vc.y - va.y);
        if (A <= 0) continue;  // back-facing or degenerate
        const int px0 = max(ceil16(min(va.x, min(vb.x, vc.x))), 0);
        const int px1 = min(floor16(max(va.x, max(vb.x, vc.x))), tw - 1);
        const int py0 = max(ceil16(min(va.y, min(vb.y, vc.y))), 0);
        const int py1 = min(floor16(max(va.y, max(vb.y, vc.y))), th - 1);
        if (px0 > px1 || py0 > py1) continue;
        cov.x = min(cov.x, px0);  // every pixel this triangle covers lies in its box
        cov.y = max(cov.y, px1);
        cov.z = min(cov.z, py0);
        cov.w = max(cov.w, py1);
        if ((px1 - px0 + 1) * (py1 - py0 + 1) > INL && px1 - px0 < 64 && py1 - py0 < 64) {
          const int slot = atomicAdd(&s_qn, 1);
          if (slot < qcap) {  // (triangle, box): x0 10 bits, y0 10 bits, w-1 and h-1 6 bits each
            queue[2 * slot] = pk;
            queue[2 * slot + 1] = (uint32_t)px0 | ((uint32_t)py0 << 10) | ((uint32_t)(px1 - px0) << 20) |
                                  ((uint32_t)(py1 - py0) << 26);
            continue;
          }
        }
        raster_box(va, vb, vc, A, px0, px1, py0, py1, sIZ, i0, i1, i2, tile, tw);
      }
    }
    if (__syncthreads_or(tok ? 0 : 1)) {
      timed_out = true;
      break;
    }
    pt ^= 1u;
    t_pending = false;
    if (c + 1 < m.chunk_count) {
      if (tid == 0) {
        const int4 cn = g.chunk_info[m.chunk_begin + c + 1];
        bulk_load(tbuf, g.chunk_tris + cn.z, (uint32_t)((cn.w + 3) & ~3) * 4u, &s_bar[1]);
      }
      t_pending = true;
    }
    // larger triangles: one warp per triangle, its pixel centres across lanes
    const int nq = min(s_qn, qcap);
    for (int e = warp; e < nq; e += NW) {
      const uint32_t pk = queue[2 * e], box = queue[2 * e + 1];
      const int i0 = pk & 1023, i1 = (pk >> 10) & 1023, i2 = (pk >> 20) & 1023;
      const int2 va = unpack_xy(sXY[i0]), vb = unpack_xy(sXY[i1]), vc = unpack_xy(sXY[i2]);
      const int px0 = box & 1023, py0 = (box >> 10) & 1023, bw = (int)((box >> 20) & 63) + 1;
      const int n = bw * ((int)(box >> 26) + 1);
      // k / bw = umulhi(k, ceil(2^32 / bw)) for k, bw < 2^16 (bw = 1 would overflow the magic)
      const uint32_t magic = 0xffffffffu / (uint32_t)bw + 1u;
      float invA = 0.0f;
      for (int k = lane; k < n; k += 32) {
        const int ry = bw == 1 ? k : (int)__umulhi((uint32_t)k, magic);
        const int px = px0 + k - ry * bw, py = py0 + ry;
        const int Px = 16 * px, Py = 16 * py;
        const int w0 = (vc.y - vb.y) * (Px - vb.x) - (vc.x - vb.x) * (Py - vb.y);
        const int w1 = (va.y - vc.y) * (Px - vc.x) - (va.x - vc.x) * (Py - vc.y);
        const int w2 = (vb.y - va.y) * (Px - va.x) - (vb.x - va.x) * (Py - va.y);
        if (!covers(w0, w1, w2, va, vb, vc)) continue;
        if (invA == 0.0f) invA = __frcp_rn(__int2float_rn(w0 + w1 + w2));
        atomicMax(&tile[py * tw + px], pixel_iz_bits(w0, w1, w2, invA, sIZ[i0], sIZ[i1], sIZ[i2]));
      }
    }
    __syncthreads();  // the next chunk reuses sXY, sIZ and the queue
  }
  if (timed_out) {
    // A wait gave up: drain every copy still in flight with the full bound
    // (kWaitSpins polls or 2 s). Once both have landed the barriers' phases
    // are known again and the CTA may take further work; if a drain also
    // gives up, a copy may still be writing into this CTA's shared memory and
    // it must stop.
    bool ok = true;
    if (v_pending) ok = mbar_wait(&s_bar[0], pv) && ok;
    if (t_pending) ok = mbar_wait(&s_bar[1], pt) && ok;
    ok = __syncthreads_and(ok);
    if (ok) {
      if (v_pending) pv ^= 1u;
      if (t_pending) pt ^= 1u;
    }
    return ok ? kEvalTimedOut : kEvalStop;
  }
  return kEvalDone;
}

// What a render source holds per pixel of the pose's box (shared memory,
// rows of the box width): 1/z bits with 0 = empty (the per-hypothesis
// kernel's own tile); z bits with +inf = empty (the tile store); or z bits
// whose sign bit says the rendered point is explained by I (Eq. (1)), which
// k_render decides once per pose for a single-scene batch.
constexpr int kSrcInvZ = 0, kSrcZ = 1, kSrcZExplained = 2;
constexpr uint32_t kExplainedBit = 0x80000000u;  // z > 0: the sign bit is free

// The first part of cost_phase: the monotone test against the parent render
// and dR (Eq. (3)). Reads the render from src, writes z on dR (+inf
// elsewhere) into the tile, and sums violations and |dR| into s_cnt[0],
// s_cnt[1] (with kSrcZExplained also dJ_r, the dR pixels not explained by I,
// into s_cnt[3]); ends with a CTA barrier, after which src is no longer read.
template <int NT, int SRC>
__device__ __forceinline__ void compare_phase(int pid, int plen, int4 bb, const Camera& cam, const Batch& b,
                                              const uint32_t* src, uint32_t* tile, int* s_cnt) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int tw = bb.z, n = bb.z * bb.w;
  int viol = 0, nnew = 0, djr = 0;
  const float* zp = plen > 0 ? b.parent_z + (size_t)pid * cam.W * cam.H : nullptr;
  const uint32_t empty = SRC == kSrcInvZ ? 0u : kInfBits;
  // pixel i of the box is (i mod tw, i div tw); i div tw = umulhi(i, ceil(2^32 / tw)),
  // exact for i tw < 2^32 (the box is at most kMaxObjectPixels wide and high)
  const uint32_t mg = tw > 1 ? 0xffffffffu / (uint32_t)tw + 1u : 0u;
  // U pixels per thread at a time: their parent depths are loaded together
  constexpr int U = 4;
  for (int i0 = tid; i0 < n; i0 += NT * U) {
    uint32_t sv[U];
    float pz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * NT;
      sv[u] = i < n ? src[i] : empty;
      pz[u] = __uint_as_float(kInfBits);
      if (zp && sv[u] != empty) {
        const int ly = tw > 1 ? (int)__umulhi((uint32_t)i, mg) : i;
        pz[u] = __ldg(&zp[(size_t)(bb.y + ly) * cam.W + bb.x + (i - ly * tw)]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * NT;
      if (i >= n) break;
      if (sv[u] == empty) {
        tile[i] = kInfBits;
        continue;
      }
      const uint32_t zb = SRC == kSrcInvZ ? __float_as_uint(__frcp_rn(__uint_as_float(sv[u]))) : (sv[u] & ~kExplainedBit);
      if (__float_as_uint(pz[u]) != kInfBits) {  // hidden by (or hiding) the parent: not in dR
        if (__uint_as_float(zb) < pz[u]) viol++;
        tile[i] = kInfBits;
        continue;
      }
      tile[i] = zb;
      nnew++;
      if (SRC == kSrcZExplained && !(sv[u] & kExplainedBit)) djr++;
    }
  }
  viol = warp_sum(viol);
  nnew = warp_sum(nnew);
  if (SRC == kSrcZExplained) djr = warp_sum(djr);
  if (lane == 0) {
    if (viol) atomicAdd(&s_cnt[0], viol);
    if (nnew) atomicAdd(&s_cnt[1], nnew);
    if (djr) atomicAdd(&s_cnt[3], djr);
  }
  __syncthreads();
}

// compare_phase for a staged render that stays as it is (z bits, +inf =
// empty, with kSrcZExplained the explained flag in the sign bit): the same
// test and counts, but dR goes to a bitmask (bit i of mask[i / 32] = pixel i
// is in dR) instead of a z tile. Warps take 32 consecutive pixels at a time
// (NT is a multiple of 32, so every word is written by one ballot). Ends
// with a CTA barrier.
template <int NT, int SRC>
__device__ __forceinline__ void compare_phase_mask(int pid, int plen, int4 bb, const Camera& cam, const Batch& b,
                                                   const uint32_t* src, uint32_t* mask, int* s_cnt) {
  static_assert(SRC != kSrcInvZ && NT % 32 == 0, "staged z source");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tw = bb.z, n = bb.z * bb.w;
  int viol = 0, nnew = 0, djr = 0;
  const float* zp = plen > 0 ? b.parent_z + (size_t)pid * cam.W * cam.H : nullptr;
  const uint32_t mg = tw > 1 ? 0xffffffffu / (uint32_t)tw + 1u : 0u;  // i / tw, as in compare_phase
  constexpr int U = 4;
  for (int w0 = 32 * warp; w0 < n; w0 += NT * U) {  // warp-uniform
    uint32_t sv[U];
    float pz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = w0 + u * NT + lane;
      sv[u] = i < n ? src[i] : kInfBits;
      pz[u] = __uint_as_float(kInfBits);
      if (zp && sv[u] != kInfBits) {
        const int ly = tw > 1 ? (int)__umulhi((uint32_t)i, mg) : i;
        pz[u] = __ldg(&zp[(size_t)(bb.y + ly) * cam.W + bb.x + (i - ly * tw)]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bool in_dr = false;
      if (sv[u] != kInfBits) {
        const uint32_t zb = sv[u] & ~kExplainedBit;
        if (__float_as_uint(pz[u]) != kInfBits) {  // hidden by (or hiding) the parent: not in dR
          if (__uint_as_float(zb) < pz[u]) viol++;
        } else {
          in_dr = true;
          nnew++;
          if (SRC == kSrcZExplained && !(sv[u] & kExplainedBit)) djr++;
        }
      }
      const unsigned bits = __ballot_sync(0xffffffffu, in_dr);
      if (lane == 0 && w0 + u * NT < n) mask[(w0 + u * NT) >> 5] = bits;
    }
  }
  viol = warp_sum(viol);
  nnew = warp_sum(nnew);
  if (SRC == kSrcZExplained) djr = warp_sum(djr);
  if (lane == 0) {
    if (viol) atomicAdd(&s_cnt[0], viol);
    if (nnew) atomicAdd(&s_cnt[1], nnew);
    if (djr) atomicAdd(&s_cnt[3], djr);
  }
  __syncthreads();
}

// The rest of cost_phase, after compare_phase: the record of an invalid
// child, or dJ_r (unless DJR_DONE: compare_phase counted it), dJ_o,
// residual(K) and n_vol from the tile (z on dR, +inf elsewhere). Ends with a
// CTA barrier.
template <int NT, bool DJR_DONE>
__device__ __forceinline__ void finish_phase(long long h, int pid, int plen, int K_total, const perch_obj& o,
                                             int4 bb, const DevMesh& m, const Camera& cam, const Geometry& g,
                                             const ObsIndex& obs, const Batch& b, const DRTile& tile,
                                             const float* rxs, const float* rys, int* s_cnt) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tw = bb.z, th = bb.w;
  const float ox = g.xs[o.ix], oy = g.ys[o.iy];
  const uint32_t flags = s_cnt[2] ? PERCH_FLAG_CULLED : 0u;
  if (s_cnt[0] > 0) {
    if (tid == 0) {
      perch_cost r = {0, 0, 0, s_cnt[0], s_cnt[1], flags | PERCH_FLAG_INVALID, 0};
      b.out[h] = r;
    }
    __syncthreads();  // s_cnt is reset by the next hypothesis
    return;
  }

  // ---- dJ_r: dR points with no observed point within delta (with no
  // observed point near the footprint, all |dR| of them, s_cnt[1])
  int djr = 0;
  const bool probe = !DJR_DONE && obs_near(cam, g, obs, o);
  if (!DJR_DONE && !probe && tid == 0) djr = s_cnt[1];
  for (int ly = warp; probe && ly < th; ly += NW) {
    const float ry = rys[ly];
    for (int lx = lane; lx < tw; lx += 32) {
      const uint32_t zb = tile.at(ly * tw + lx);
      if (zb == kInfBits) continue;
      const float z = __uint_as_float(zb);
      if (!explained_by_obs(obs, fmul(rxs[lx], z), fmul(ry, z), z, cam.delta2)) djr++;
    }
  }

  // ---- dJ_o: observed points inside V(O) with no dR point within delta
  int djo = 0, nvol = 0;
  if (obs.n > 0) {
    const float r = m.vol_rmax * 1.001f + 1e-6f;
    const int cx0 = max(cell_of(ox - r, obs.g2x, obs.inv2, obs.n2x) - 1, 0);
    const int cx1 = min(cell_of(ox + r, obs.g2x, obs.inv2, obs.n2x) + 1, obs.n2x - 1);
    const int cy0 = max(cell_of(oy - r, obs.g2y, obs.inv2, obs.n2y) - 1, 0);
    const int cy1 = min(cell_of(oy + r, obs.g2y, obs.inv2, obs.n2y) + 1, obs.n2y - 1);
    if (cx0 <= cx1) {
      for (int cy = cy0; cy <= cy1; ++cy) {
        const int s = obs.start2[cy * obs.n2x + cx0], e = obs.start2[cy * obs.n2x + cx1 + 1];
        for (int k = s + tid; k < e; k += NT) {
          const float4 qw = obs.world2[k];
          if (!in_volume(g, m, ox, oy, o.iyaw, qw)) continue;
          if (!explained_by_tile(cam, obs.cam2[k], tile, rxs, rys, bb)) djo++;
          bool in_parent = false;  // already inside an assigned volume?
          for (int j = 0; j < plen && !in_parent; ++j) {
            const perch_obj po = b.parents[(long long)pid * b.parent_stride + j];
            in_parent = in_volume(g, g.meshes[po.mesh], g.xs[po.ix], g.ys[po.iy], po.iyaw, qw);
          }
          if (!in_parent) nvol++;
        }
      }
    }
  }

  // ---- residual(K) on edges into the last level
  int resid = 0;
  if (plen + 1 == K_total) {
    const int nu = b.uset_count[pid];
    const int* U = b.uset + (size_t)pid * b.uset_stride;
    for (int k = tid; k < nu; k += NT) {
      const int qi = U[k];
      if (in_volume(g, m, ox, oy, o.iyaw, obs.world2[qi])) continue;
      if (explained_by_tile(cam, obs.cam2[qi], tile, rxs, rys, bb)) continue;
      resid++;
    }
  }
  djr = warp_sum(djr);
  djo = warp_sum(djo);
  resid = warp_sum(resid);
  nvol = warp_sum(nvol);
  if (lane == 0) {
    if (djr) atomicAdd(&s_cnt[3], djr);
    if (djo) atomicAdd(&s_cnt[4], djo);
    if (resid) atomicAdd(&s_cnt[5], resid);
    if (nvol) atomicAdd(&s_cnt[6], nvol);
  }
  __syncthreads();
  if (tid == 0) {
    perch_cost r = {s_cnt[3], s_cnt[4], s_cnt[5], 0, s_cnt[1], flags, s_cnt[6]};
    b.out[h] = r;
  }
  __syncthreads();  // s_cnt and the tile are reused by the next hypothesis
}

// Cost of hypothesis h (Eq. (3), Eq. (4)) from its new object's render,
// which the shared tile holds as 1/z bits (0 = empty) over the pose's box bb,
// rows of bb.z pixels; the tile then receives z on dR and +inf elsewhere.
// rxs / rys hold the ray slopes of the box's columns and rows; s_cnt is zero
// except the culled flag s_cnt[2]; a CTA barrier must separate those writes
// from the call. Ends with a CTA barrier (s_cnt and the tile may be reused
// after it).
template <int NT>
__device__ __forceinline__ void cost_phase(long long h, int pid, int plen, int K_total, const perch_obj& o, int4 bb,
                                           const DevMesh& m, const Camera& cam, const Geometry& g,
                                           const ObsIndex& obs, const Batch& b, uint32_t* tile, const float* rxs,
                                           const float* rys, int* s_cnt) {
  compare_phase<NT, kSrcInvZ>(pid, plen, bb, cam, b, tile, tile, s_cnt);
  finish_phase<NT, false>(h, pid, plen, K_total, o, bb, m, cam, g, obs, b, DRTile{tile, nullptr}, rxs, rys, s_cnt);
}

// The checks every evaluation of hypothesis h makes before it touches its
// parent or pose: false means the record is the bad-index record.
struct HypArgs {
  perch_obj o;
  int pid, plen, scene, K_total;
  long long pose;
};

__device__ __forceinline__ bool hyp_args(const Geometry& g, const Batch& b, long long h, HypArgs& a) {
  a.o = b.hyp[h];
  a.pid = b.hyp_parent[h];
  bool bad = a.pid < 0 || a.pid >= b.n_par || !obj_ok(g, a.o);
  a.plen = bad ? 0 : b.parent_len[a.pid];
  bad = bad || a.plen < 0 || a.plen > b.parent_stride;
  a.scene = (bad || !b.parent_scene) ? 0 : b.parent_scene[a.pid];
  a.K_total = (bad || !b.parent_K) ? b.K_total : b.parent_K[a.pid];
  bad = bad || (b.parent_scene && (a.scene < 0 || a.scene >= b.n_scenes));
  a.pose = bad ? 0 : (((long long)a.o.mesh * g.nx + a.o.ix) * g.ny + a.o.iy) * g.n_yaw + a.o.iyaw;
  return !bad;
}

// One CTA per hypothesis: render the new object into a shared-memory z tile
// covering its screen box (render_chunks), test it against the parent render
// (Eq. (3)), and count dJ_r, dJ_o and residual(K) (Sec. IV-A, Eq. (4))
// (cost_phase). The CTA's two mbarriers persist across hypotheses (their
// phase parities are in sh).
template <int NT, bool MULTI>
__device__ int eval_one(long long h, const Camera& cam, const Geometry& g, const ObsIndex& obs0, const Batch& b,
                        EvalShared& sh, ObsIndex* s_obs) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int* s_cnt = sh.cnt;
  HypArgs a;
  const bool ok = hyp_args(g, b, h, a);
  const int4 bb = ok ? g.pose_bbox[a.pose] : make_int4(0, 0, 0, 0);
  if (!ok || bb.z > b.tile_w || bb.w > b.tile_h) {
    if (tid == 0) {
      perch_cost r = {0, 0, 0, 0, 0, kFlagBadIndex, 0};
      b.out[h] = r;
    }
    return kEvalDone;
  }
  if (MULTI && tid < (int)(sizeof(ObsIndex) / 4))  // this scene's index, read from shared memory below
    reinterpret_cast<int*>(s_obs)[tid] = reinterpret_cast<const int*>(&b.scenes[a.scene])[tid];
  const ObsIndex& obs = MULTI ? *s_obs : obs0;
  const RenderSmem s = render_smem(sh.dyn);
  float* rxs = reinterpret_cast<float*>(s.tile + b.tile_w * b.tile_h);
  float* rys = rxs + b.tile_w;
  const int tw = bb.z, th = bb.w;
  const DevMesh m = g.meshes[a.o.mesh];
  if (tid == 0) render_start(g, m, a.o.iyaw, s, sh.bar);
  for (int ly = warp; ly < th; ly += NW)
    for (int lx = lane; lx < tw; lx += 32) s.tile[ly * tw + lx] = 0u;  // 1/z = 0: empty
  for (int i = tid; i < tw; i += NT) rxs[i] = g.rx[bb.x + i];
  for (int i = tid; i < th; i += NT) rys[i] = g.ry[bb.y + i];
  if (tid < 7) s_cnt[tid] = 0;

  unsigned culled = 0;
  int4 cov = make_int4(0x7fffffff, -1, 0x7fffffff, -1);  // not needed here
  const int st = render_chunks<NT, kInlinePixels>(cam, g, b, m, a.o, bb, s, sh, culled, cov);
  if (st != kEvalDone) {
    if (tid == 0) {
      perch_cost r = {0, 0, 0, 0, 0, kFlagTimeout, 0};
      b.out[h] = r;
    }
    __syncthreads();  // s_cnt and the tile are reused by the next hypothesis
    return st;
  }
  if (culled) s_cnt[2] = 1;
  __syncthreads();
  cost_phase<NT>(h, a.pid, a.plen, a.K_total, a.o, bb, m, cam, g, obs, b, s.tile, rxs, rys, s_cnt);
  return kEvalDone;
}

// A group of hypotheses evaluated by one persistent launch: items
// order[offset .. offset + count) (order == nullptr: hypotheses 0 .. count-1),
// claimed one at a time from the device counter `next`.
struct EvalGroup {
  const int* order;
  const int* offset;  // device scalar
  const int* count;   // device scalar
  int* next;          // device counter, zero before the launch
};

template <int NT, bool MULTI>
__global__ void __launch_bounds__(NT, 1024 / NT) k_eval(Camera cam, Geometry g, ObsIndex obs, Batch b, EvalGroup grp) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(16) ObsIndex s_obs;
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_cnt[7];
  __shared__ int s_qn;
  __shared__ int s_item;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  EvalShared sh{s_bar, s_cnt, &s_qn, smem, 0u, 0u};
  const int count = *grp.count, offset = grp.order ? *grp.offset : 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(grp.next, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= count) break;
    const long long h = grp.order ? grp.order[offset + item] : item;
    if (eval_one<NT, MULTI>(h, cam, g, obs, b, sh, &s_obs) == kEvalStop) break;
  }
}

// ---- shared renders: one render per distinct pose of a batch, then one
// cost per hypothesis. The new object's render depends on its mesh and pose
// alone, not on its parent, so k_render rasterises each distinct (mesh,
// pose) of the batch once into the tile store (global memory, 1/z bits of
// the pose's screen box at 16-byte offset tile_off[pose]), and k_cost gives
// every hypothesis its own comparison with its parent and its own costs
// from that stored tile, read with plain coalesced loads.
template <int NT, bool EXPL, int INL>
__global__ void __launch_bounds__(NT, 1024 / NT) k_render(Camera cam, Geometry g, ObsIndex obs, Batch b,
                                                          RenderWork w) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_qn;
  __shared__ int s_item;
  __shared__ int s_box[4];  // the covered pixels' box within the pose's box: x0, x1, y0, y1
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  EvalShared sh{s_bar, nullptr, &s_qn, smem, 0u, 0u};
  const RenderSmem s = render_smem(smem);
  const int count = *w.count, offset = *w.offset;
  const long long per_x = (long long)g.ny * g.n_yaw, per_mesh = (long long)g.nx * per_x;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(w.next, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= count) break;
    const long long p = w.gpose[offset + item];
    perch_obj o;
    o.mesh = (uint16_t)(p / per_mesh);
    o.ix = (int16_t)((p / per_x) % g.nx);
    o.iy = (int16_t)((p / g.n_yaw) % g.ny);
    o.iyaw = (uint16_t)(p % g.n_yaw);
    const int4 bb = g.pose_bbox[p];
    if (bb.z > b.tile_w || bb.w > b.tile_h) {  // never for a valid pose: the mesh's tile is its largest box
      if (tid == 0) w.pose_flags[p] = kPoseFailed;
      continue;
    }
    const int tw = bb.z, th = bb.w;
    const DevMesh m = g.meshes[o.mesh];
    if (tid == 0) render_start(g, m, o.iyaw, s, sh.bar);
    for (int ly = warp; ly < th; ly += NW)
      for (int lx = lane; lx < tw; lx += 32) s.tile[ly * tw + lx] = 0u;  // 1/z = 0: empty
    if (tid < 4) s_box[tid] = (tid & 1) ? -1 : 0x7fffffff;  // ordered by render_chunks' first barrier
    unsigned culled = 0;
    int4 cov = make_int4(0x7fffffff, -1, 0x7fffffff, -1);  // x0, x1, y0, y1 of this thread's triangle boxes
    const int st = render_chunks<NT, INL>(cam, g, b, m, o, bb, s, sh, culled, cov);
    if (st != kEvalDone) {
      if (tid == 0) w.pose_flags[p] = kPoseFailed;
      __syncthreads();  // the tile is cleared by the next pose
      if (st == kEvalStop) break;
      continue;
    }
    {  // the union of the front faces' candidate boxes holds every covered pixel:
       // the store (and every cost of this pose) keeps only that box
      const int x0 = __reduce_min_sync(0xffffffffu, cov.x), x1 = __reduce_max_sync(0xffffffffu, cov.y);
      const int y0 = __reduce_min_sync(0xffffffffu, cov.z), y1 = __reduce_max_sync(0xffffffffu, cov.w);
      if (lane == 0 && x1 >= 0) {
        atomicMin(&s_box[0], x0);
        atomicMax(&s_box[1], x1);
        atomicMin(&s_box[2], y0);
        atomicMax(&s_box[3], y1);
      }
    }
    const int any_culled = __syncthreads_or(culled != 0);  // also publishes s_box
    const bool empty = s_box[1] < 0;
    const int cx0 = empty ? 0 : s_box[0], cy0 = empty ? 0 : s_box[2];
    const int cw = empty ? 0 : s_box[1] - s_box[0] + 1, ch = empty ? 0 : s_box[3] - s_box[2] + 1;
    // the store gets z = 1/(1/z) (+inf where empty) over that box, rows of
    // its width, and, for a single-scene batch (EXPL), the Eq. (1) test of
    // each rendered point against I in the sign bit: it depends on the pose
    // and the scene, not on the parent. A pose with no observed point near
    // its footprint explains no point.
    const bool probe = EXPL && obs_near(cam, g, obs, o);
    uint32_t* dst = w.store + 4 * (size_t)w.tile_off[p];
    for (int ly = warp; ly < ch; ly += NW) {
      const float ry = EXPL ? g.ry[bb.y + cy0 + ly] : 0.0f;
      for (int lx = lane; lx < cw; lx += 32) {
        const uint32_t izb = s.tile[(cy0 + ly) * tw + cx0 + lx];
        uint32_t v = kInfBits;
        if (izb != 0u) {
          const float z = __frcp_rn(__uint_as_float(izb));
          v = __float_as_uint(z);
          if (probe && explained_by_obs(obs, fmul(g.rx[bb.x + cx0 + lx], z), fmul(ry, z), z, cam.delta2))
            v |= kExplainedBit;
        }
        dst[ly * cw + lx] = v;
      }
    }
    if (tid == 0) {
      w.pose_flags[p] = any_culled ? kPoseCulled : 0;
      w.tile_box[p] = make_int4(bb.x + cx0, bb.y + cy0, cw, ch);
      if (w.valid) w.valid[p] = w.tag;  // read by later launches only
    }
    __syncthreads();  // the tile is cleared by the next pose
  }
}

// k_cost: one persistent CTA per SM slot costs hypotheses, sorted by pose,
// from the tile store. A hypothesis's tile is brought into one of NS shared
// stage buffers by a 1D bulk copy (TMA), which threads only read: the compare
// pass marks dR in a bitmask beside it, and dJ_r, dJ_o and the residual read
// z from the stage through that mask. Thread 0 claims the next hypothesis and
// looks up its arguments, box and tile while the rest of the CTA finishes the
// current one. A hypothesis of a pose whose tile a stage already holds (the
// batch is sorted by pose) takes it as it is, with no copy. With one stage
// (NS = 1) the copy starts once the current hypothesis is done, and the
// smaller footprint lets more CTAs share an SM to cover each other's copies;
// with two (NS = 2, where the tiles are small) it starts into the other stage
// as soon as the next hypothesis is claimed, and overlaps dJ_o and the
// residual.
template <int NT, bool MULTI, int NS>
__global__ void __launch_bounds__(NT) k_cost(Camera cam, Geometry g, ObsIndex obs0, Batch b, CostWork w) {
  static_assert(NS == 1 || NS == 2, "one or two stages");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(16) ObsIndex s_obs;
  __shared__ __align__(8) uint64_t s_bar[NS];
  __shared__ int s_cnt[7];
  // the claimed item: its index, hypothesis, arguments, box, pose flags, tile
  // offset, stage and how its tile reaches the stage (thread 0 writes it,
  // everyone reads it)
  enum { kItemBad = 0, kItemFailed = 1, kItemCopy = 2, kItemReuse = 3 };
  __shared__ struct {
    int item, state, pf, off, sidx;
    long long h;
    HypArgs a;
    int4 bb;
  } s_nx;
  const int tid = threadIdx.x;
  const int stage_words = (b.tile_w * b.tile_h + 3) & ~3;  // 16-byte multiples
  uint32_t* mask = reinterpret_cast<uint32_t*>(smem) + NS * stage_words;
  float* rxs = reinterpret_cast<float*>(mask + (((b.tile_w * b.tile_h + 31) / 32 + 3) & ~3));
  float* rys = rxs + b.tile_w;
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&s_bar[k], 1);
    fence_barrier_init();
  }
  __syncthreads();
  const int count = *w.count, offset = *w.offset;
  // thread 0: the pose whose tile each stage holds or will receive, and the
  // stage of the last claimed item
  long long stage_pose[NS];
  for (int k = 0; k < NS; ++k) stage_pose[k] = -1;
  int cur = 0;
  auto stage_of = [&](int k) { return reinterpret_cast<uint32_t*>(smem) + k * stage_words; };
  auto copy = [&](int k, int off, int4 bb) {
    bulk_load(stage_of(k), w.store + 4 * (size_t)off, 16u * (uint32_t)((bb.z * bb.w + 3) >> 2), &s_bar[k]);
  };
  // thread 0: claim the next item and look it up; with two stages also start
  // its copy into the stage the current item does not use. No barrier (the
  // caller's next one publishes it)
  auto claim = [&]() {
    const int it = atomicAdd(w.next, 1);
    s_nx.item = it;
    if (it >= count) return;
    const long long h = w.order[offset + it];
    HypArgs a;
    int state = kItemBad, pf = 0, off = 0, sidx = cur;
    int4 bb = make_int4(0, 0, 0, 0);
    if (hyp_args(g, b, h, a)) {
      bb = w.tile_box[a.pose];  // the covered pixels' box (k_render)
      pf = w.pose_flags[a.pose];
      if (pf & kPoseFailed) {
        state = kItemFailed;
      } else if (bb.z <= b.tile_w && bb.w <= b.tile_h) {
        if (bb.z == 0 || bb.w == 0) {
          state = kItemReuse;  // nothing rendered: no pixel to copy or compare
        } else if (a.pose == stage_pose[cur]) {
          state = kItemReuse;
        } else if (NS == 2 && a.pose == stage_pose[NS - 1 - cur]) {
          state = kItemReuse;
          sidx = NS - 1 - cur;
        } else {
          state = kItemCopy;
          off = w.tile_off[a.pose];
          sidx = NS - 1 - cur;  // the other stage (the same one with NS = 1)
          stage_pose[sidx] = a.pose;
          if (NS == 2) copy(sidx, off, bb);  // the other stage's last reader has finished
        }
        cur = sidx;
      }
    }
    s_nx.h = h;
    s_nx.state = state;
    s_nx.pf = pf;
    s_nx.off = off;
    s_nx.sidx = sidx;
    s_nx.a = a;
    s_nx.bb = bb;
  };
  if (tid == 0) claim();
  __syncthreads();
  uint32_t parity[NS];
  for (int k = 0; k < NS; ++k) parity[k] = 0;
  for (;;) {
    const int item = s_nx.item;
    if (item >= count) break;
    const long long h = s_nx.h;
    const int state = s_nx.state, pf = s_nx.pf, sidx = s_nx.sidx;
    const HypArgs a = s_nx.a;
    const int4 bb = s_nx.bb;
    if (state == kItemBad || state == kItemFailed) {  // no copy for it
      __syncthreads();  // every thread has read s_nx
      if (tid == 0) {
        perch_cost r = {0, 0, 0, 0, 0, state == kItemFailed ? kFlagTimeout : kFlagBadIndex, 0};
        b.out[h] = r;
        claim();
      }
      __syncthreads();
      continue;
    }
    // one stage: the previous hypothesis's last barrier has passed, the stage is free
    if (NS == 1 && state == kItemCopy && tid == 0) copy(0, s_nx.off, bb);
    if (MULTI && tid < (int)(sizeof(ObsIndex) / 4))
      reinterpret_cast<int*>(&s_obs)[tid] = reinterpret_cast<const int*>(&b.scenes[a.scene])[tid];
    const ObsIndex& obs = MULTI ? s_obs : obs0;
    for (int i = tid; i < bb.z; i += NT) rxs[i] = g.rx[bb.x + i];
    for (int i = tid; i < bb.w; i += NT) rys[i] = g.ry[bb.y + i];
    if (tid < 7) s_cnt[tid] = tid == 2 ? (pf & kPoseCulled) : 0;
    if (state == kItemCopy) {
      // wait for the stage (bounded); on give-up drain the copy with the
      // full bound, report the hypothesis and go on, or stop if it is still
      // in flight
      if (!__syncthreads_and(mbar_wait(&s_bar[sidx], parity[sidx], b.wait_polls))) {
        const bool drained = __syncthreads_and(mbar_wait(&s_bar[sidx], parity[sidx]));
        if (tid == 0) {
          perch_cost r = {0, 0, 0, 0, 0, kFlagTimeout, 0};
          b.out[h] = r;
          for (int k = 0; k < NS; ++k) stage_pose[k] = -1;
          if (drained) claim();
        }
        if (!drained) break;
        parity[sidx] ^= 1u;
        __syncthreads();
        continue;
      }
      parity[sidx] ^= 1u;
    } else {
      __syncthreads();  // a stage holds this pose's tile already; rays and counters are written
    }
    const uint32_t* stage = stage_of(sidx);
    // a single-scene store holds z with the explained flag (k_render); a
    // multi-scene one plain z, and dJ_r is counted here against the scene
    compare_phase_mask<NT, MULTI ? kSrcZ : kSrcZExplained>(a.pid, a.plen, bb, cam, b, stage, mask, s_cnt);
    if (tid == 0) claim();  // look the next one up (and with two stages start its copy)
    const DevMesh m = g.meshes[a.o.mesh];
    finish_phase<NT, !MULTI>(h, a.pid, a.plen, a.K_total, a.o, bb, m, cam, g, obs, b, DRTile{stage, mask}, rxs, rys,
                             s_cnt);
  }
}

cudaError_t preload_eval_kernels() {
  cudaFuncAttributes a;
  cudaError_t e;
  if ((e = cudaFuncGetAttributes(&a, k_fill_u32)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&a, k_render_parents)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&a, k_uset)) != cudaSuccess) return e;
  return cudaFuncGetAttributes(&a, k_eval<256, false>);
}

// group hypotheses by mesh: hist -> offsets (exclusive scan) -> order;
// hypotheses whose record the shortcut already wrote (skip[h] = 1) are left out
__global__ void k_group_hist(const perch_obj* hyp, long long n, int n_mesh, int* hist, const uint8_t* skip) {
  const long long h = blockIdx.x * 256LL + threadIdx.x;
  if (h >= n || (skip && skip[h])) return;
  const int m = min((int)hyp[h].mesh, n_mesh - 1);
  atomicAdd(&hist[m], 1);
}

__global__ void k_group_scatter(const perch_obj* hyp, long long n, int n_mesh, int* cursor, int* order,
                                const uint8_t* skip) {
  const long long h = blockIdx.x * 256LL + threadIdx.x;
  if (h >= n || (skip && skip[h])) return;
  const int m = min((int)hyp[h].mesh, n_mesh - 1);
  order[atomicAdd(&cursor[m], 1)] = (int)h;
}

cudaError_t launch_group_by_mesh(const perch_obj* hyp, long long n, int n_mesh, int* hist, int* offsets,
                                 int* cursor, int* order, int* scan_tmp, cudaStream_t s, const uint8_t* skip) {
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * n_mesh, s);
  if (e != cudaSuccess || n == 0) return e;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_group_hist<<<blocks, 256, 0, s>>>(hyp, n, n_mesh, hist, skip);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_exclusive_scan(hist, offsets, n_mesh, scan_tmp, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(cursor, offsets, sizeof(int) * n_mesh, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  k_group_scatter<<<blocks, 256, 0, s>>>(hyp, n, n_mesh, cursor, order, skip);
  return cudaGetLastError();
}

// ---- hypotheses grouped by pose, for shared renders: counts per pose ->
// starts (exclusive scan) -> the distinct poses (scan of cnt > 0) -> each
// mesh's ranges -> hypotheses placed in their pose's range
__global__ void k_pose_count(Geometry g, Batch b, int* cnt) {
  const long long h = blockIdx.x * 256LL + threadIdx.x;
  if (h >= b.n_hyp || (b.skip && b.skip[h])) return;
  HypArgs a;
  if (!hyp_args(g, b, h, a)) {  // the record k_eval would write; joins no group
    perch_cost r = {0, 0, 0, 0, 0, kFlagBadIndex, 0};
    b.out[h] = r;
    return;
  }
  atomicAdd(&cnt[a.pose], 1);
}

// a pose is rendered when some hypothesis has it and (with the render
// cache) the store does not hold its render under this batch's tag already
__global__ void k_pose_nonzero(const int* cnt, int P, const uint32_t* valid, uint32_t tag, int* flag) {
  const int p = blockIdx.x * 256 + threadIdx.x;
  if (p < P) flag[p] = cnt[p] > 0 && !(valid && valid[p] == tag) ? 1 : 0;
}

__global__ void k_pose_list(const int* flag, const int* gix, int P, int* gpose) {
  const int p = blockIdx.x * 256 + threadIdx.x;
  if (p < P && flag[p]) gpose[gix[p]] = p;
}

// mesh m owns poses [m * per_mesh, (m + 1) * per_mesh): its hypotheses are
// order[start[m * per_mesh] ..) and its distinct poses gpose[gix[m * per_mesh] ..)
__global__ void k_mesh_ranges(const int* start, const int* gix, int n_mesh, int per_mesh, int* ranges) {
  const int m = blockIdx.x * 256 + threadIdx.x;
  if (m >= n_mesh) return;
  const int a = m * per_mesh, e = a + per_mesh;
  ranges[4 * m + 0] = start[a];
  ranges[4 * m + 1] = start[e] - start[a];
  ranges[4 * m + 2] = gix[a];
  ranges[4 * m + 3] = gix[e] - gix[a];
}

__global__ void k_pose_place(Geometry g, Batch b, const int* start, int* cnt, int* order) {
  const long long h = blockIdx.x * 256LL + threadIdx.x;
  if (h >= b.n_hyp || (b.skip && b.skip[h])) return;
  HypArgs a;
  if (!hyp_args(g, b, h, a)) return;
  order[start[a.pose] + atomicSub(&cnt[a.pose], 1) - 1] = (int)h;
}

cudaError_t launch_group_by_pose(const Geometry& g, const Batch& b, const PoseGroups& pg, const uint32_t* valid,
                                 uint32_t tag, cudaStream_t s) {
  const int per_mesh = g.nx * g.ny * g.n_yaw, P = g.n_mesh * per_mesh;
  const unsigned pb = (unsigned)((P + 255) / 256), hb = (unsigned)((b.n_hyp + 255) / 256);
  cudaError_t e = cudaMemsetAsync(pg.cnt, 0, sizeof(int) * (size_t)P, s);
  if (e != cudaSuccess) return e;
  if (b.n_hyp > 0) k_pose_count<<<hb, 256, 0, s>>>(g, b, pg.cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_exclusive_scan(pg.cnt, pg.start, P, pg.tmp, s)) != cudaSuccess) return e;
  k_pose_nonzero<<<pb, 256, 0, s>>>(pg.cnt, P, valid, tag, pg.flag);
  if ((e = launch_exclusive_scan(pg.flag, pg.gix, P, pg.tmp, s)) != cudaSuccess) return e;
  k_pose_list<<<pb, 256, 0, s>>>(pg.flag, pg.gix, P, pg.gpose);
  k_mesh_ranges<<<(unsigned)((g.n_mesh + 255) / 256), 256, 0, s>>>(pg.start, pg.gix, g.n_mesh, per_mesh, pg.ranges);
  if (b.n_hyp > 0) k_pose_place<<<hb, 256, 0, s>>>(g, b, pg.start, pg.cnt, pg.order);
  return cudaGetLastError();
}

__global__ void k_tile_sizes(Geometry g, int P, int* sizes) {
  const int p = blockIdx.x * 256 + threadIdx.x;
  if (p >= P) return;
  const int4 bb = g.pose_bbox[p];
  sizes[p] = (bb.z * bb.w + 3) >> 2;  // 16-byte units: every tile starts 16-byte aligned
}

cudaError_t launch_tile_offsets(const Geometry& g, int* sizes, int* tile_off, int* tmp, cudaStream_t s) {
  const int P = g.n_mesh * g.nx * g.ny * g.n_yaw;
  k_tile_sizes<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(g, P, sizes);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_exclusive_scan(sizes, tile_off, P, tmp, s);
}

// ------------------------------------------------------------ exact shortcut
// A hypothesis whose parent render is empty over its screen box and which has
// no observed point within (footprint radius + delta + 2 cm) of its (x, y)
// in the world plane has a record fixed by its solo render alone: every
// rendered pixel is new (dR = R(O)) and in no conflict with the parent
// (viol = 0); no observed point is within delta of a rendered point (all of
// dR unexplained: dJ_r = |dR|); none lies in V(O) (dJ_o = 0, n_vol = 0); and on
// a last-level edge every q of U is outside V(O) and unexplained (residual =
// |U|). |dR| and the cull flag come from the same rasteriser run once per
// (mesh, pose) against an empty parent and an empty observation.

// summed-area table S[(r + 1) (cols + 1) + c + 1] = sum of counts[0..r][0..c]
// of `mats` matrices (one block each); S's first row and column are zero
__global__ void k_sat(const int* counts, int rows, int cols, int* sat) {
  const int* cnt = counts + (size_t)blockIdx.x * rows * cols;
  int* S = sat + (size_t)blockIdx.x * (rows + 1) * (cols + 1);
  for (int c = threadIdx.x; c <= cols; c += blockDim.x) S[c] = 0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    int* row = S + (size_t)(r + 1) * (cols + 1);
    row[0] = 0;
    int a = 0;
    for (int c = 0; c < cols; ++c) {
      a += cnt[(size_t)r * cols + c];
      row[c + 1] = a;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < cols; c += blockDim.x)
    for (int r = 1; r < rows; ++r) S[(size_t)(r + 1) * (cols + 1) + c + 1] += S[(size_t)r * (cols + 1) + c + 1];
}

__global__ void k_cell_counts(const int* start2, int n, int* counts) {
  const int c = blockIdx.x * 256 + threadIdx.x;
  if (c < n) counts[c] = start2[c + 1] - start2[c];
}

cudaError_t launch_grid2_sat(const int* start2, int n2x, int n2y, int* counts, int* sat, cudaStream_t s) {
  const int n = n2x * n2y;
  k_cell_counts<<<(n + 255) / 256, 256, 0, s>>>(start2, n, counts);
  k_sat<<<1, 1024, 0, s>>>(counts, n2y, n2x, sat);
  return cudaGetLastError();
}

// occupied pixels of each parent render per 8x8 tile
__global__ void k_parent_tile_counts(Camera cam, Batch b, int* counts) {
  const int p = blockIdx.y;
  const int t = blockIdx.x * 256 + threadIdx.x;
  if (t >= b.tiles_w * b.tiles_h) return;
  const int tx = t % b.tiles_w, ty = t / b.tiles_w;
  const float* z = b.parent_z + (size_t)p * cam.W * cam.H;
  int c = 0;
  for (int v = ty * 8; v < min(ty * 8 + 8, cam.H); ++v)
    for (int u = tx * 8; u < min(tx * 8 + 8, cam.W); ++u) c += __float_as_uint(z[(size_t)v * cam.W + u]) != kInfBits;
  counts[(size_t)p * b.tiles_w * b.tiles_h + t] = c;
}

cudaError_t launch_parent_tiles(const Camera& cam, const Batch& b, int* counts, int* sat, cudaStream_t s) {
  if (b.n_par > 65535) return cudaErrorInvalidValue;
  dim3 grid((b.tiles_w * b.tiles_h + 255) / 256, b.n_par);
  k_parent_tile_counts<<<grid, 256, 0, s>>>(cam, b, counts);
  k_sat<<<b.n_par, 128, 0, s>>>(counts, b.tiles_h, b.tiles_w, sat);
  return cudaGetLastError();
}

__global__ void k_shortcut(Camera cam, Geometry g, ObsIndex obs0, Batch b) {
  const long long h = blockIdx.x * 256LL + threadIdx.x;
  int fast = 0;
  if (h < b.n_hyp) {
    const perch_obj o = b.hyp[h];
    const int pid = b.hyp_parent[h];
    bool ok = pid >= 0 && pid < b.n_par && obj_ok(g, o);
    const int plen = ok ? b.parent_len[pid] : 0;
    ok = ok && plen >= 0 && plen <= b.parent_stride;
    const int scene = (ok && b.parent_scene) ? b.parent_scene[pid] : 0;
    ok = ok && (!b.parent_scene || (scene >= 0 && scene < b.n_scenes));
    const long long pose = (((long long)o.mesh * g.nx + o.ix) * g.ny + o.iy) * g.n_yaw + o.iyaw;
    const int4 bb = ok ? g.pose_bbox[pose] : make_int4(0, 0, 0, 0);
    ok = ok && bb.z <= b.tile_w && bb.w <= b.tile_h;
    if (ok && plen > 0 && bb.z > 0 && bb.w > 0) {  // parent render empty over the screen box?
      const int tx0 = max(bb.x, 0) >> 3, tx1 = min(bb.x + bb.z - 1, cam.W - 1) >> 3;
      const int ty0 = max(bb.y, 0) >> 3, ty1 = min(bb.y + bb.w - 1, cam.H - 1) >> 3;
      if (tx0 <= tx1 && ty0 <= ty1) {
        const int* S = b.parent_sat + (size_t)pid * (b.tiles_h + 1) * (b.tiles_w + 1);
        ok = sat_sum(S, b.tiles_w, ty0, ty1, tx0, tx1) == 0;
      }
    }
    if (ok) ok = !obs_near(cam, g, b.parent_scene ? b.scenes[scene] : obs0, o);  // no observed point near (x, y)
    if (ok) {
      const int K_total = b.parent_K ? b.parent_K[pid] : b.K_total;
      const int2 so = b.solo[pose];
      perch_cost r;
      r.djr = so.x;
      r.djo = 0;
      r.resid = plen + 1 == K_total ? b.uset_count[pid] : 0;
      r.viol = 0;
      r.n_new = so.x;
      r.flags = (uint32_t)so.y;
      r.n_vol = 0;
      b.out[h] = r;
      fast = 1;
    }
    b.skip[h] = (uint8_t)fast;
  }
  const int n_fast = __syncthreads_count(fast);
  if (threadIdx.x == 0 && n_fast && b.n_short) atomicAdd(b.n_short, (unsigned long long)n_fast);
}

cudaError_t launch_shortcut(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                            cudaStream_t s) {
  if (b.n_hyp == 0) return cudaSuccess;
  k_shortcut<<<(unsigned)((b.n_hyp + 255) / 256), 256, 0, s>>>(cam, g, obs, b);
  return cudaGetLastError();
}

// solo table entry from a record evaluated against an empty parent and an
// empty observation: (|dR| = pixels covered, cull flag)
__global__ void k_solo_pack(const perch_cost* rec, long long n, int2* solo) {
  const long long h = blockIdx.x * 256LL + threadIdx.x;
  if (h < n) solo[h] = make_int2(rec[h].n_new, (int)(rec[h].flags & 1u));
}

cudaError_t launch_solo_pack(const perch_cost* rec, long long n, int2* solo, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_solo_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rec, n, solo);
  return cudaGetLastError();
}

template <int NT, bool MULTI>
static cudaError_t launch_group_t(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                                  const EvalGroup& grp, long long max_items, int sm_count, cudaStream_t s) {
  const size_t smem = eval_smem_bytes(b.tile_w, b.tile_h);
  auto kern = k_eval<NT, MULTI>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * sm_count;
  if (grid > max_items) grid = max_items;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT, smem, s>>>(cam, g, obs, b, grp);
  return cudaGetLastError();
}

template <int NT, bool EXPL, int INL>
static cudaError_t launch_render_t(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                                   const RenderWork& w, long long max_items, int sm_count, cudaStream_t s) {
  const size_t smem = render_smem_bytes(b.tile_w, b.tile_h);
  auto kern = k_render<NT, EXPL, INL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * sm_count;
  if (grid > max_items) grid = max_items;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT, smem, s>>>(cam, g, obs, b, w);
  return cudaGetLastError();
}

template <int NT, bool EXPL>
static cudaError_t launch_render_i(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                                   const RenderWork& w, long long max_items, int inline_px, int sm_count,
                                   cudaStream_t s) {
  switch (inline_px) {
    case 8: return launch_render_t<NT, EXPL, 8>(cam, g, obs, b, w, max_items, sm_count, s);
    case 32: return launch_render_t<NT, EXPL, 32>(cam, g, obs, b, w, max_items, sm_count, s);
    default: return launch_render_t<NT, EXPL, 16>(cam, g, obs, b, w, max_items, sm_count, s);
  }
}

// One persistent launch rendering one mesh's distinct poses of a batch into
// the tile store, with CTAs of `threads` (128, 256 or 512), the inline limit
// `inline_px` (8, 16 or 32 candidate pixel centres) and the mesh's tile
// (b.tile_w x b.tile_h). A single-scene batch also stores each rendered
// point's Eq. (1) test against `obs`.
cudaError_t launch_render_group(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                                const RenderWork& w, long long max_items, int threads, int inline_px,
                                int sm_count, cudaStream_t s) {
  if (max_items <= 0) return cudaSuccess;
  const bool expl = b.parent_scene == nullptr;
  switch (threads) {
    case 128: return expl ? launch_render_i<128, true>(cam, g, obs, b, w, max_items, inline_px, sm_count, s)
                          : launch_render_i<128, false>(cam, g, obs, b, w, max_items, inline_px, sm_count, s);
    case 512: return expl ? launch_render_i<512, true>(cam, g, obs, b, w, max_items, inline_px, sm_count, s)
                          : launch_render_i<512, false>(cam, g, obs, b, w, max_items, inline_px, sm_count, s);
    default: return expl ? launch_render_i<256, true>(cam, g, obs, b, w, max_items, inline_px, sm_count, s)
                         : launch_render_i<256, false>(cam, g, obs, b, w, max_items, inline_px, sm_count, s);
  }
}

template <int NT, bool MULTI, int NS>
static cudaError_t launch_cost_t(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                                 const CostWork& w, long long max_items, int sm_count, cudaStream_t s) {
  const size_t smem = cost_smem_bytes(b.tile_w, b.tile_h, NS);
  auto kern = k_cost<NT, MULTI, NS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * sm_count;
  if (grid > max_items) grid = max_items;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT, smem, s>>>(cam, g, obs, b, w);
  return cudaGetLastError();
}

template <int NS>
static cudaError_t launch_cost_s(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                                 const CostWork& w, long long max_items, int threads, int sm_count, cudaStream_t s) {
  const bool multi = b.parent_scene != nullptr;
  if (threads == 256)
    return multi ? launch_cost_t<256, true, NS>(cam, g, obs, b, w, max_items, sm_count, s)
                 : launch_cost_t<256, false, NS>(cam, g, obs, b, w, max_items, sm_count, s);
  return multi ? launch_cost_t<128, true, NS>(cam, g, obs, b, w, max_items, sm_count, s)
               : launch_cost_t<128, false, NS>(cam, g, obs, b, w, max_items, sm_count, s);
}

// One persistent launch costing one mesh's hypotheses of a batch from the
// tile store, with CTAs of `threads` (128 or 256) and `stages` (1 or 2) stage
// buffers; two stages fall back to one where they do not fit.
bool cost_stages_fit(int device, int tile_w, int tile_h, int stages) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return false;
  return cost_smem_bytes(tile_w, tile_h, stages) + 1024 <= (size_t)optin;  // 1024: static shared memory
}

cudaError_t launch_cost_group(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                              const CostWork& w, long long max_items, int threads, int stages, int sm_count,
                              cudaStream_t s) {
  if (max_items <= 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (stages == 2 && cost_stages_fit(dev, b.tile_w, b.tile_h, 2))
    return launch_cost_s<2>(cam, g, obs, b, w, max_items, threads, sm_count, s);
  return launch_cost_s<1>(cam, g, obs, b, w, max_items, threads, sm_count, s);
}

// One persistent launch for one group of hypotheses with CTAs of `threads`
// (128, 256 or 512) and the group's tile (b.tile_w x b.tile_h).
cudaError_t launch_eval_group(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                              const int* order, const int* offset, const int* count, int* next, long long max_items,
                              int threads, int sm_count, cudaStream_t s) {
  if (max_items <= 0) return cudaSuccess;
  EvalGroup grp{order, offset, count, next};
  const bool multi = b.parent_scene != nullptr;
  switch (threads) {
    case 128: return multi ? launch_group_t<128, true>(cam, g, obs, b, grp, max_items, sm_count, s)
                           : launch_group_t<128, false>(cam, g, obs, b, grp, max_items, sm_count, s);
    case 512: return multi ? launch_group_t<512, true>(cam, g, obs, b, grp, max_items, sm_count, s)
                           : launch_group_t<512, false>(cam, g, obs, b, grp, max_items, sm_count, s);
    default: return multi ? launch_group_t<256, true>(cam, g, obs, b, grp, max_items, sm_count, s)
                          : launch_group_t<256, false>(cam, g, obs, b, grp, max_items, sm_count, s);
  }
}

// -------------------------------------------------------------------- ICP
// Local alignment of each successor's new object with the observed cloud
// (Sec. IV-E-1: the object's non-occluded portion, aligned by ICP; Sec. V-B:
// correspondences only within 2 cm), step by step as the public header
// states it. The render, the model set and every distance are the binary32
// arithmetic of the evaluation path; the pairs' sums are exact 64-bit
// integers (coordinates in units of 2^-16 m), so the order in which the
// warps add them does not matter; the fit from those sums is double
// arithmetic in a fixed order, made by one thread.

// the observed world points with their index in I, and their bounds
__global__ void k_icp_points(const float4* world2, const float4* cam2, int n, float4* pts, int* bounds) {
  const int k = blockIdx.x * 256 + threadIdx.x;
  const bool ok = k < n;
  const float4 w = ok ? world2[k] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (ok) pts[k] = make_float4(w.x, w.y, w.z, cam2[k].w);
  const int lo[3] = {ok ? ford(w.x) : INT_MAX, ok ? ford(w.y) : INT_MAX, ok ? ford(w.z) : INT_MAX};
  const int hi[3] = {ok ? ford(w.x) : INT_MIN, ok ? ford(w.y) : INT_MIN, ok ? ford(w.z) : INT_MIN};
  for (int d = 0; d < 3; ++d) {
    const int a = __reduce_min_sync(0xffffffffu, lo[d]), b = __reduce_max_sync(0xffffffffu, hi[d]);
    if ((threadIdx.x & 31) == 0 && a <= b) {
      atomicMin(&bounds[d], a);
      atomicMax(&bounds[3 + d], b);
    }
  }
}

cudaError_t launch_icp_points(const float4* world2, const float4* cam2, int n, float4* pts, int* bounds,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_icp_points<<<(n + 255) / 256, 256, 0, s>>>(world2, cam2, n, pts, bounds);
  return cudaGetLastError();
}

__device__ __forceinline__ long long icp_fixed(float v) { return __float2ll_rn(fmul(v, 65536.0f)); }

// hi 2^64 + lo: each part rounded to double, then one rounded addition
__device__ __forceinline__ double icp_i128_to_double(__int128 v) {
  const long long hi = (long long)(v >> 64);
  const unsigned long long lo = (unsigned long long)v;
  return __dadd_rn(__dmul_rn(__ll2double_rn(hi), 18446744073709551616.0), __ull2double_rn(lo));
}

// one pair's terms: n, sum X_m, sum Y_m, sum X_q, sum Y_q, sum X_m X_q,
// sum Y_m Y_q, sum X_m Y_q, sum Y_m X_q (|x|, |y| < 32 m: |X|, |Y| < 2^21)
__device__ __forceinline__ void icp_add_pair(long long* L, float mx, float my, float qx, float qy) {
  if (!(fabsf(mx) < 32.0f && fabsf(my) < 32.0f && fabsf(qx) < 32.0f && fabsf(qy) < 32.0f)) return;
  const long long X = icp_fixed(mx), Y = icp_fixed(my), QX = icp_fixed(qx), QY = icp_fixed(qy);
  L[0] += 1;
  L[1] += X;
  L[2] += Y;
  L[3] += QX;
  L[4] += QY;
  L[5] += X * QX;
  L[6] += Y * QY;
  L[7] += X * QY;
  L[8] += Y * QX;
}

// Planar Procrustes from the sums: C = n sum(m . q) - sum m . sum q and
// S = n sum(m x q) - sum m x sum q (exact), (c, s) = (C, S) / |(C, S)|,
// t = (sum q - R sum m) / n. False when C = S = 0.
__device__ bool icp_solve(const long long* S, double* T) {
  const __int128 n = S[0];
  const __int128 C = n * ((__int128)S[5] + S[6]) - ((__int128)S[1] * S[3] + (__int128)S[2] * S[4]);
  const __int128 X = n * ((__int128)S[7] - S[8]) - ((__int128)S[1] * S[4] - (__int128)S[2] * S[3]);
  if (C == 0 && X == 0) return false;
  const double Cd = icp_i128_to_double(C), Xd = icp_i128_to_double(X);
  const double h = __dsqrt_rn(__dadd_rn(__dmul_rn(Cd, Cd), __dmul_rn(Xd, Xd)));
  const double c = __ddiv_rn(Cd, h), s = __ddiv_rn(Xd, h);
  const double nd = __ll2double_rn(S[0]), sx = __ll2double_rn(S[1]), sy = __ll2double_rn(S[2]);
  T[0] = c;
  T[1] = s;
  T[2] = __dmul_rn(__ddiv_rn(__dsub_rn(__ll2double_rn(S[3]), __dsub_rn(__dmul_rn(c, sx), __dmul_rn(s, sy))), nd),
                   1.0 / 65536.0);
  T[3] = __dmul_rn(__ddiv_rn(__dsub_rn(__ll2double_rn(S[4]), __dadd_rn(__dmul_rn(s, sx), __dmul_rn(c, sy))), nd),
                   1.0 / 65536.0);
  return true;
}

struct IcpClaim {
  int* next;  // device counter, zero before the launch
};

// One CTA per hypothesis at a time (claimed from a counter): render the new
// object into the shared-memory tile over its screen box (render_chunks),
// keep the pixels in front of the parent's render as the model set (z bits;
// 0 elsewhere), then iterate. In each matching a thread takes one model
// pixel: it back-projects and moves the point and scans the grid cells that
// meet a cube of half-width rho about it, where rho is the radius, or from
// the second matching on the distance to the point the pixel was paired with
// last time, when that point is still within the radius (the nearest point
// can only be nearer). It keeps the nearest point (ties: smaller index),
// adds the pair to its own sums, and the warps reduce those into shared
// 64-bit counters. Thread 0 then decides and fits.
template <int NT>
__global__ void __launch_bounds__(NT) k_icp(Camera cam, Geometry g, Batch b, IcpGrid q, IcpWork w, IcpClaim cl) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ __align__(8) unsigned long long s_sum[9];
  __shared__ double s_T[4];
  __shared__ int s_qn, s_item, s_stop, s_nm;
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  EvalShared sh{s_bar, nullptr, &s_qn, smem, 0u, 0u};
  const RenderSmem s = render_smem(smem);
  uint32_t* tile = s.tile;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(cl.next, 1);
    __syncthreads();
    const long long h = s_item;
    __syncthreads();
    if (h >= b.n_hyp) break;
    HypArgs a;
    const bool ok = hyp_args(g, b, h, a);
    const int4 bb = ok ? g.pose_bbox[a.pose] : make_int4(0, 0, 0, 0);
    if (!ok || bb.z > b.tile_w || bb.w > b.tile_h) {
      if (tid == 0) w.out[h] = perch_icp{0.0, 0.0, 0.0, 0.0, 0, 0, 0, (int32_t)kFlagBadIndex};
      continue;
    }
    const int tw = bb.z, area = bb.z * bb.w;
    const DevMesh m = g.meshes[a.o.mesh];
    if (tid == 0) render_start(g, m, a.o.iyaw, s, sh.bar);
    for (int i = tid; i < area; i += NT) tile[i] = 0u;  // 1/z = 0: empty
    if (tid == 0) {
      s_nm = 0;
      s_T[0] = 1.0;
      s_T[1] = s_T[2] = s_T[3] = 0.0;
    }
    unsigned culled = 0;
    int4 cov = make_int4(0x7fffffff, -1, 0x7fffffff, -1);  // not needed here
    const int st = render_chunks<NT, kInlinePixels>(cam, g, b, m, a.o, bb, s, sh, culled, cov);
    if (st != kEvalDone) {
      if (tid == 0) w.out[h] = perch_icp{0.0, 0.0, 0.0, 0.0, 0, 0, 0, (int32_t)kFlagTimeout};
      __syncthreads();  // the tile is cleared by the next hypothesis
      if (st == kEvalStop) break;
      continue;
    }
    // model set: z where the object lies strictly in front of the parent,
    // and the list of those pixels (in any order: every sum is order-free)
    const float* zp = b.parent_z + (size_t)a.pid * cam.W * cam.H;
    const size_t cap = (size_t)b.tile_w * b.tile_h;
    int* list = w.prev + 2 * cap * blockIdx.x;  // this CTA's slice: model pixels, then their last pairs
    int* prev_t = list + cap;
    for (int i0 = 0; i0 < area; i0 += NT) {  // the same trip count in every lane (ballots below)
      const int i = i0 + tid;
      uint32_t v = 0u;
      if (i < area) {
        const uint32_t izb = tile[i];
        if (izb != 0u) {
          const int ly = i / tw, lx = i - ly * tw;
          const float z = __frcp_rn(__uint_as_float(izb));
          if (z < zp[(size_t)(bb.y + ly) * cam.W + bb.x + lx]) v = __float_as_uint(z);
        }
        tile[i] = v;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, v != 0u);
      int base = 0;
      if (lane == 0 && mask) base = atomicAdd(&s_nm, __popc(mask));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (v != 0u) list[base + __popc(mask & ((1u << lane) - 1u))] = i;
    }
    __syncthreads();  // |M|, the model set and its list are complete
    const int nm = s_nm;
    long long prev[9];  // thread 0: the previous matching's sums
    bool have_prev = false;
    int iters = 0, n_corr = 0, status = PERCH_ICP_CAP;
    for (int k = 1; k <= w.max_iter; ++k) {
      if (tid < 9) s_sum[tid] = 0ull;
      __syncthreads();  // also publishes s_T
      const float cf = __double2float_rn(s_T[0]), sf = __double2float_rn(s_T[1]);
      const float txf = __double2float_rn(s_T[2]), tyf = __double2float_rn(s_T[3]);
      long long L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int e = tid; e < nm; e += NT) {
        const int i = list[e];
        const int ly = i / tw, lx = i - ly * tw;
        const float z = __uint_as_float(tile[i]);
        const float xc = fmul(g.rx[bb.x + lx], z), yc = fmul(g.ry[bb.y + ly], z);
        const float mx = fadd(ffma(cam.Rwc[2], z, ffma(cam.Rwc[1], yc, fmul(cam.Rwc[0], xc))), cam.twc[0]);
        const float my = fadd(ffma(cam.Rwc[5], z, ffma(cam.Rwc[4], yc, fmul(cam.Rwc[3], xc))), cam.twc[1]);
        const float mz = fadd(ffma(cam.Rwc[8], z, ffma(cam.Rwc[7], yc, fmul(cam.Rwc[6], xc))), cam.twc[2]);
        const float px = fadd(fsub(fmul(cf, mx), fmul(sf, my)), txf);
        const float py = fadd(fadd(fmul(sf, mx), fmul(cf, my)), tyf);
        // Search window: the radius, or, when the previous matching's point
        // is still within it, that point's distance (the nearest point is no
        // farther). The margins cover the rounding of d^2 (relative 2^-22)
        // and of the window's ends (1e-6 m), so every point whose d^2 can
        // tie or beat the bound lies inside.
        float rho = w.rwin;
        if (k > 1) {
          const int t0 = prev_t[e];
          if (t0 >= 0) {
            const float d0 = dist2(px, py, mz, q.pts[t0]);
            if (d0 <= w.r2) rho = fminf(rho, __fsqrt_rn(d0) * 1.001f + 1e-6f);
          }
        }
        const int x0 = max(cell_of(px - rho, q.gx, q.inv, q.nx), 0), x1 = min(cell_of(px + rho, q.gx, q.inv, q.nx), q.nx - 1);
        const int y0 = max(cell_of(py - rho, q.gy, q.inv, q.ny), 0), y1 = min(cell_of(py + rho, q.gy, q.inv, q.ny), q.ny - 1);
        const int z0 = max(cell_of(mz - rho, q.gz, q.inv, q.nz), 0), z1 = min(cell_of(mz + rho, q.gz, q.inv, q.nz), q.nz - 1);
        uint32_t bd = 0xffffffffu;  // no candidate (every d^2 <= r^2 has smaller bits)
        int bj = INT_MAX, bt = -1;
        float bqx = 0.0f, bqy = 0.0f;
        if (x0 <= x1) {
          for (int iz = z0; iz <= z1; ++iz)
            for (int iy = y0; iy <= y1; ++iy) {
              const int row = (iz * q.ny + iy) * q.nx;
              const int end = q.start[row + x1 + 1];
              for (int t = q.start[row + x0]; t < end; ++t) {
                const float4 o = q.pts[t];
                const float d = dist2(px, py, mz, o);
                if (d <= w.r2) {
                  const uint32_t db = __float_as_uint(d);
                  const int j = __float_as_int(o.w);
                  if (db < bd || (db == bd && j < bj)) {
                    bd = db;
                    bj = j;
                    bt = t;
                    bqx = o.x;
                    bqy = o.y;
                  }
                }
              }
            }
        }
        prev_t[e] = bt;
        if (bt >= 0) icp_add_pair(L, mx, my, bqx, bqy);
      }
      for (int t = 0; t < 9; ++t) {
        long long v = L[t];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0 && v != 0) atomicAdd(&s_sum[t], (unsigned long long)v);
      }
      __syncthreads();
      if (tid == 0) {
        long long S[9];
        for (int t = 0; t < 9; ++t) S[t] = (long long)s_sum[t];
        n_corr = (int)S[0];
        int stop = 0;
        bool same = have_prev;
        for (int t = 0; t < 9 && same; ++t) same = S[t] == prev[t];
        if (S[0] < 3) {
          status = PERCH_ICP_FEW;
          stop = 1;
        } else if (same) {
          status = PERCH_ICP_CONVERGED;
          stop = 1;
        } else {
          double T[4];
          if (!icp_solve(S, T)) {
            status = PERCH_ICP_DEGENERATE;
            stop = 1;
          } else {
            for (int t = 0; t < 4; ++t) s_T[t] = T[t];
            for (int t = 0; t < 9; ++t) prev[t] = S[t];
            have_prev = true;
            iters = k;
          }
        }
        s_stop = stop;
      }
      __syncthreads();
      if (s_stop) break;
    }
    if (tid == 0) w.out[h] = perch_icp{s_T[0], s_T[1], s_T[2], s_T[3], s_nm, n_corr, iters, status};
    __syncthreads();  // the tile, s_T and s_nm are reused by the next hypothesis
  }
}

cudaError_t launch_icp(const Camera& cam, const Geometry& g, const Batch& b, const IcpGrid& q, const IcpWork& w,
                       long long prev_elems, int* next, int sm_count, cudaStream_t s) {
  if (b.n_hyp <= 0) return cudaSuccess;
  const size_t smem = render_smem_bytes(b.tile_w, b.tile_h);
  auto kern = k_icp<256>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * sm_count;
  if (grid > b.n_hyp) grid = b.n_hyp;
  const long long cap = 2LL * b.tile_w * b.tile_h;  // each CTA's slice of w.prev
  if (cap > 0 && grid > prev_elems / cap) grid = prev_elems / cap;
  if (grid < 1) return cudaErrorInvalidValue;
  kern<<<(unsigned)grid, 256, smem, s>>>(cam, g, b, q, w, IcpClaim{next});
  return cudaGetLastError();
}

}  // namespace perch
