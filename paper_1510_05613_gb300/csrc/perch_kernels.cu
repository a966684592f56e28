// PERCH successor evaluation: device kernels for sm_103a.
//
// Arithmetic contract: every floating-point step on the evaluation path is a
// single binary32 operation rounded to nearest-even (__fadd_rn, __fmul_rn,
// __fdiv_rn, __frcp_rn, __int2float_rn, __float2int_rn); nothing is fused.
// The library is also compiled with -fmad=false. Coverage and z-buffer
// resolution are exact integer / order-independent min operations, so every
// count is bit-exact with the CPU oracle.
#include <climits>

#include "perch_internal.h"

namespace perch {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }

__device__ __forceinline__ int ford(float f) {  // order-preserving float -> int
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}

__device__ __forceinline__ float dist2(float px, float py, float pz, float4 q) {
  float dx = fsub(px, q.x), dy = fsub(py, q.y), dz = fsub(pz, q.z);
  return fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz));
}

// V(O): the inscribed vertical cylinder of Sec. III-A at pose (ox, oy)
__device__ __forceinline__ bool in_volume(float4 qw, float ox, float oy, float r2, float zlo, float zhi) {
  float dx = fsub(qw.x, ox), dy = fsub(qw.y, oy);
  float d2 = fadd(fmul(dx, dx), fmul(dy, dy));
  return d2 <= r2 && zlo <= qw.z && qw.z <= zhi;
}

struct Vtx {
  int X, Y;   // snapped pixel coordinates, 1/16 px
  float iz;   // 1 / z_c; negative marks a culled vertex
};

// object frame -> world (yaw, then table translation) -> camera -> pixel
__device__ __forceinline__ Vtx transform_vertex(const Camera& c, float vx, float vy, float vz,
                                                float x, float y, float cs, float sn) {
  float xw = fadd(fsub(fmul(cs, vx), fmul(sn, vy)), x);
  float yw = fadd(fadd(fmul(sn, vx), fmul(cs, vy)), y);
  float zw = vz;
  float xc = fadd(fadd(fadd(fmul(c.Rcw[0], xw), fmul(c.Rcw[1], yw)), fmul(c.Rcw[2], zw)), c.tcw[0]);
  float yc = fadd(fadd(fadd(fmul(c.Rcw[3], xw), fmul(c.Rcw[4], yw)), fmul(c.Rcw[5], zw)), c.tcw[1]);
  float zc = fadd(fadd(fadd(fmul(c.Rcw[6], xw), fmul(c.Rcw[7], yw)), fmul(c.Rcw[8], zw)), c.tcw[2]);
  bool bad = !(zc > kNearZ);
  float u = fadd(fmul(c.fx, __fdiv_rn(xc, zc)), c.cx);
  float v = fadd(fmul(c.fy, __fdiv_rn(yc, zc)), c.cy);
  bad = bad || !(fabsf(u) <= kGuard) || !(fabsf(v) <= kGuard);
  Vtx o;
  if (bad) {
    o.X = 0; o.Y = 0; o.iz = -1.0f;
    return o;
  }
  o.X = __float2int_rn(fmul(16.0f, u));
  o.Y = __float2int_rn(fmul(16.0f, v));
  o.iz = __frcp_rn(zc);
  return o;
}

__device__ __forceinline__ int floor16(int a) { return a >> 4; }
__device__ __forceinline__ int ceil16(int a) { return -((-a) >> 4); }

struct SmemSink {
  uint32_t* tile;
  __device__ __forceinline__ void operator()(int idx, uint32_t zbits) const { atomicMin(&tile[idx], zbits); }
};
struct GlobalSink {
  uint32_t* z;
  __device__ __forceinline__ void operator()(int idx, uint32_t zbits) const { atomicMin(&z[idx], zbits); }
};

// Rasterise one triangle into a tile of tw x th pixels whose top-left pixel
// is at (ox16 / 16, oy16 / 16): exact edge functions, top-left tie rule,
// 1/z interpolation with screen-space barycentrics, min-z resolve.
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
  const bool own12 = (Y2 - Y1) > 0 || ((Y2 - Y1) == 0 && (X2 - X1) < 0);
  const bool own20 = (Y0 - Y2) > 0 || ((Y0 - Y2) == 0 && (X0 - X2) < 0);
  const bool own01 = (Y1 - Y0) > 0 || ((Y1 - Y0) == 0 && (X1 - X0) < 0);
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
      if (!in) continue;
      const float b0 = fmul(__int2float_rn(w0), invA);
      const float b1 = fmul(__int2float_rn(w1), invA);
      const float b2 = fmul(__int2float_rn(w2), invA);
      const float iz = fadd(fadd(fmul(b0, a.iz), fmul(b1, b.iz)), fmul(b2, c.iz));
      sink(py * tw + px, __float_as_uint(__frcp_rn(iz)));
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
  const int x0 = max(ix - 1, 0), x1 = min(ix + 1, o.n3x - 1);
  if (x0 > x1) return false;
  for (int dz = -1; dz <= 1; ++dz) {
    const int cz = iz + dz;
    if (cz < 0 || cz >= o.n3z) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int cy = iy + dy;
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

// Eq. (1) against the new object's dR (the z tile, +inf off dR): is some
// rendered point within delta of the observed point q?
__device__ __forceinline__ bool explained_by_tile(const Camera& cam, float4 q, const uint32_t* tile,
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
      const uint32_t zb = tile[ly * bb.z + lx];
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
  const float xw = fadd(fadd(fadd(fmul(cam.Rwc[0], x), fmul(cam.Rwc[1], y)), fmul(cam.Rwc[2], z)), cam.twc[0]);
  const float yw = fadd(fadd(fadd(fmul(cam.Rwc[3], x), fmul(cam.Rwc[4], y)), fmul(cam.Rwc[5], z)), cam.twc[1]);
  const float zw = fadd(fadd(fadd(fmul(cam.Rwc[6], x), fmul(cam.Rwc[7], y)), fmul(cam.Rwc[8], z)), cam.twc[2]);
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

// conservative screen box of every (mesh, pose) from the 8 corners of the
// mesh's bounding box (a convex hull of its vertices), plus one pixel
__global__ void k_pose_bbox(Camera cam, Geometry g, int4* bbox, int* max_wh, int* bad_any) {
  const long long n = (long long)g.n_mesh * g.nx * g.ny * g.n_yaw;
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t >= n) return;
  const int iyaw = (int)(t % g.n_yaw);
  const int iy = (int)((t / g.n_yaw) % g.ny);
  const int ix = (int)((t / ((long long)g.n_yaw * g.ny)) % g.nx);
  const int m = (int)(t / ((long long)g.n_yaw * g.ny * g.nx));
  const DevMesh dm = g.meshes[m];
  const float2 cs = g.cs[iyaw];
  const float x = g.xs[ix], y = g.ys[iy];
  float umin = 1e30f, umax = -1e30f, vmin = 1e30f, vmax = -1e30f;
  bool bad = false;
  for (int k = 0; k < 8; ++k) {
    const float vx = (k & 1) ? dm.hi[0] : dm.lo[0];
    const float vy = (k & 2) ? dm.hi[1] : dm.lo[1];
    const float vz = (k & 4) ? dm.hi[2] : dm.lo[2];
    const float xw = fadd(fsub(fmul(cs.x, vx), fmul(cs.y, vy)), x);
    const float yw = fadd(fadd(fmul(cs.y, vx), fmul(cs.x, vy)), y);
    const float xc = cam.Rcw[0] * xw + cam.Rcw[1] * yw + cam.Rcw[2] * vz + cam.tcw[0];
    const float yc = cam.Rcw[3] * xw + cam.Rcw[4] * yw + cam.Rcw[5] * vz + cam.tcw[1];
    const float zc = cam.Rcw[6] * xw + cam.Rcw[7] * yw + cam.Rcw[8] * vz + cam.tcw[2];
    if (!(zc > kNearZ)) { bad = true; break; }
    const float u = cam.fx * (xc / zc) + cam.cx, v = cam.fy * (yc / zc) + cam.cy;
    umin = fminf(umin, u); umax = fmaxf(umax, u);
    vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
  }
  int4 b;
  if (bad || !(umax - umin < 4096.0f) || !(vmax - vmin < 4096.0f)) {
    b = make_int4(0, 0, cam.W, cam.H);
    atomicOr(bad_any, 1);
  } else {
    int x0 = (int)floorf(fmaxf(umin, -8.0f)) - 1, x1 = (int)ceilf(fminf(umax, (float)cam.W + 8.0f)) + 1;
    int y0 = (int)floorf(fmaxf(vmin, -8.0f)) - 1, y1 = (int)ceilf(fminf(vmax, (float)cam.H + 8.0f)) + 1;
    x0 = max(x0, 0); y0 = max(y0, 0);
    x1 = min(x1, cam.W - 1); y1 = min(y1, cam.H - 1);
    if (x0 > x1 || y0 > y1) b = make_int4(0, 0, 0, 0);
    else b = make_int4(x0, y0, x1 - x0 + 1, y1 - y0 + 1);
  }
  bbox[t] = b;
  atomicMax(&max_wh[0], b.z);
  atomicMax(&max_wh[1], b.w);
}

cudaError_t launch_pose_bbox(const Camera& cam, const Geometry& g, int4* bbox, int* max_wh, int* bad,
                             cudaStream_t s) {
  const long long n = (long long)g.n_mesh * g.nx * g.ny * g.n_yaw;
  if (n == 0) return cudaSuccess;
  k_pose_bbox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cam, g, bbox, max_wh, bad);
  return cudaGetLastError();
}

// ------------------------------------------------------------ parent prep
// z-buffer render of every parent's objects (R_j) into its own full image.
// Block = one meshlet of one (parent, object) pair.
__global__ void __launch_bounds__(64) k_render_parents(Camera cam, Geometry g, Batch b,
                                                       unsigned long long* culled_total) {
  __shared__ int sX[kMeshletMaxVerts], sY[kMeshletMaxVerts];
  __shared__ float sZ[kMeshletMaxVerts];
  const int item = blockIdx.y;
  const int p = item / b.parent_stride, k = item % b.parent_stride;
  if (p >= b.n_par) return;
  const int plen = b.parent_len[p];
  if (k >= plen || plen > b.parent_stride) return;
  const perch_obj o = b.parents[(long long)p * b.parent_stride + k];
  if (o.mesh >= g.n_mesh || o.ix < 0 || o.ix >= g.nx || o.iy < 0 || o.iy >= g.ny || o.iyaw >= g.n_yaw) return;
  const DevMesh m = g.meshes[o.mesh];
  if ((int)blockIdx.x >= m.meshlet_count) return;
  const int4 info = g.ml_info[m.meshlet_begin + blockIdx.x];
  const float x = g.xs[o.ix], y = g.ys[o.iy];
  const float2 cs = g.cs[o.iyaw];
  const int t = threadIdx.x;
  if (t < info.y) {
    const float4 v = g.ml_verts[info.x + t];
    const Vtx r = transform_vertex(cam, v.x, v.y, v.z, x, y, cs.x, cs.y);
    sX[t] = r.X; sY[t] = r.Y; sZ[t] = r.iz;
  }
  __syncthreads();
  unsigned culled = 0;
  if (t < info.w) {
    const uint32_t pk = g.ml_tris[info.z + t];
    const int i0 = pk & 255, i1 = (pk >> 8) & 255, i2 = (pk >> 16) & 255;
    uint32_t* z = reinterpret_cast<uint32_t*>(b.parent_z) + (size_t)p * cam.W * cam.H;
    raster_tri(Vtx{sX[i0], sY[i0], sZ[i0]}, Vtx{sX[i1], sY[i1], sZ[i1]}, Vtx{sX[i2], sY[i2], sZ[i2]}, 0, 0,
               cam.W, cam.H, culled, GlobalSink{z});
  }
  if (culled_total) {
    const int c = __syncthreads_count(culled != 0);
    if (threadIdx.x == 0 && c) atomicAdd(culled_total, (unsigned long long)c);
  }
}

cudaError_t launch_render_parents(const Camera& cam, const Geometry& g, const Batch& b, int max_meshlets,
                                  unsigned long long* culled, cudaStream_t s) {
  if (b.n_par == 0 || b.parent_stride == 0 || max_meshlets == 0) return cudaSuccess;
  const long long items = (long long)b.n_par * b.parent_stride;
  if (items > 65535) return cudaErrorInvalidValue;
  dim3 grid(max_meshlets, (unsigned)items);
  k_render_parents<<<grid, 64, 0, s>>>(cam, g, b, culled);
  return cudaGetLastError();
}

// U set of a parent one object short of a complete scene:
// U = {q in I - V_{K-1} : q unexplained by R_{K-1}}; then for the last object
// O_K, residual(K) = #{q in U : q not in V(O_K), q unexplained by dR_K}.
__global__ void k_uset(Camera cam, Geometry g, ObsIndex obs, Batch b) {
  const int p = blockIdx.y;
  const int plen = b.parent_len[p];
  if (plen + 1 != b.K_total || plen > b.parent_stride) return;
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (k >= obs.n) return;
  const float4 qw = obs.world2[k];
  for (int j = 0; j < plen; ++j) {
    const perch_obj o = b.parents[(long long)p * b.parent_stride + j];
    if (o.mesh >= g.n_mesh || o.ix < 0 || o.ix >= g.nx || o.iy < 0 || o.iy >= g.ny || o.iyaw >= g.n_yaw) return;
    const DevMesh m = g.meshes[o.mesh];
    if (in_volume(qw, g.xs[o.ix], g.ys[o.iy], m.vol_r2, m.vol_zlo, m.vol_zhi)) return;
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
  if (b.n_par == 0 || obs.n == 0) return cudaSuccess;
  if (b.n_par > 65535) return cudaErrorInvalidValue;
  dim3 grid((obs.n + 255) / 256, b.n_par);
  k_uset<<<grid, 256, 0, s>>>(cam, g, obs, b);
  return cudaGetLastError();
}

// ------------------------------------------------------------- evaluation
size_t eval_smem_bytes(int tile_w, int tile_h) {
  return (size_t)tile_w * tile_h * 4 + (size_t)(tile_w + tile_h) * 4 +
         (size_t)kEvalWarps * kMeshletMaxVerts * 12;
}

bool eval_tile_fits(int device, int tile_w, int tile_h) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return false;
  return eval_smem_bytes(tile_w, tile_h) + 256 <= (size_t)optin;  // 256: static shared memory of k_eval
}

// One CTA per hypothesis: render the new object into a shared-memory z tile
// covering its screen box, test it against the parent render (Eq. (3)), and
// count dJ_r, dJ_o and residual(K) (Sec. IV-A, Eq. (4)).
__global__ void __launch_bounds__(kEvalThreads) k_eval(Camera cam, Geometry g, ObsIndex obs, Batch b) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_cnt[6];  // viol, n_new, culled, djr, djo, resid
  const long long h = blockIdx.x;
  if (h >= b.n_hyp) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const perch_obj o = b.hyp[h];
  const int pid = b.hyp_parent[h];
  bool badidx = pid < 0 || pid >= b.n_par || o.mesh >= g.n_mesh || o.ix < 0 || o.ix >= g.nx || o.iy < 0 ||
                o.iy >= g.ny || o.iyaw >= g.n_yaw;
  const int plen = badidx ? 0 : b.parent_len[pid];
  badidx = badidx || plen < 0 || plen > b.parent_stride;
  const int4 bb = badidx ? make_int4(0, 0, 0, 0)
                         : g.pose_bbox[(((long long)o.mesh * g.nx + o.ix) * g.ny + o.iy) * g.n_yaw + o.iyaw];
  if (badidx || bb.z > b.tile_w || bb.w > b.tile_h) {
    if (tid == 0) {
      perch_cost r = {0, 0, 0, 0, 0, kFlagBadIndex};
      b.out[h] = r;
    }
    return;
  }
  uint32_t* tile = reinterpret_cast<uint32_t*>(smem);
  float* rxs = reinterpret_cast<float*>(tile + b.tile_w * b.tile_h);
  float* rys = rxs + b.tile_w;
  int* vX = reinterpret_cast<int*>(rys + b.tile_h);
  int* vY = vX + kEvalWarps * kMeshletMaxVerts;
  float* vZ = reinterpret_cast<float*>(vY + kEvalWarps * kMeshletMaxVerts);
  const int npx = bb.z * bb.w;
  for (int i = tid; i < npx; i += kEvalThreads) tile[i] = kInfBits;
  for (int i = tid; i < bb.z; i += kEvalThreads) rxs[i] = g.rx[bb.x + i];
  for (int i = tid; i < bb.w; i += kEvalThreads) rys[i] = g.ry[bb.y + i];
  if (tid < 6) s_cnt[tid] = 0;
  __syncthreads();

  // ---- render the new object (warp per meshlet)
  const DevMesh m = g.meshes[o.mesh];
  const float ox = g.xs[o.ix], oy = g.ys[o.iy];
  const float2 cs = g.cs[o.iyaw];
  int* wX = vX + warp * kMeshletMaxVerts;
  int* wY = vY + warp * kMeshletMaxVerts;
  float* wZ = vZ + warp * kMeshletMaxVerts;
  const int ox16 = 16 * bb.x, oy16 = 16 * bb.y;
  unsigned culled = 0;
  SmemSink sink{tile};
  for (int mi = warp; mi < m.meshlet_count; mi += kEvalWarps) {
    const int4 info = g.ml_info[m.meshlet_begin + mi];
    for (int v = lane; v < info.y; v += 32) {
      const float4 p = g.ml_verts[info.x + v];
      const Vtx r = transform_vertex(cam, p.x, p.y, p.z, ox, oy, cs.x, cs.y);
      wX[v] = r.X; wY[v] = r.Y; wZ[v] = r.iz;
    }
    __syncwarp();
    for (int t = lane; t < info.w; t += 32) {
      const uint32_t pk = g.ml_tris[info.z + t];
      const int i0 = pk & 255, i1 = (pk >> 8) & 255, i2 = (pk >> 16) & 255;
      raster_tri(Vtx{wX[i0], wY[i0], wZ[i0]}, Vtx{wX[i1], wY[i1], wZ[i1]}, Vtx{wX[i2], wY[i2], wZ[i2]}, ox16,
                 oy16, bb.z, bb.w, culled, sink);
    }
    __syncwarp();
  }
  if (culled) s_cnt[2] = 1;
  __syncthreads();

  // ---- monotone test against the parent render and dR (Eq. (3))
  int viol = 0, nnew = 0;
  const float* zp = plen > 0 ? b.parent_z + (size_t)pid * cam.W * cam.H : nullptr;
  for (int i = tid; i < npx; i += kEvalThreads) {
    const uint32_t zb = tile[i];
    if (zb == kInfBits) continue;
    if (zp) {
      const int ly = i / bb.z, lx = i - ly * bb.z;
      const float pz = __ldg(&zp[(size_t)(bb.y + ly) * cam.W + bb.x + lx]);
      if (__float_as_uint(pz) != kInfBits) {
        if (__uint_as_float(zb) < pz) viol++;
        tile[i] = kInfBits;  // hidden by (or hiding) the parent: not in dR
        continue;
      }
    }
    nnew++;
  }
  viol = warp_sum(viol);
  nnew = warp_sum(nnew);
  if (lane == 0) {
    if (viol) atomicAdd(&s_cnt[0], viol);
    if (nnew) atomicAdd(&s_cnt[1], nnew);
  }
  __syncthreads();
  const uint32_t flags = s_cnt[2] ? PERCH_FLAG_CULLED : 0u;
  if (s_cnt[0] > 0) {
    if (tid == 0) {
      perch_cost r = {0, 0, 0, s_cnt[0], s_cnt[1], flags | PERCH_FLAG_INVALID};
      b.out[h] = r;
    }
    return;
  }

  // ---- dJ_r: dR points with no observed point within delta
  int djr = 0;
  for (int i = tid; i < npx; i += kEvalThreads) {
    const uint32_t zb = tile[i];
    if (zb == kInfBits) continue;
    const int ly = i / bb.z, lx = i - ly * bb.z;
    const float z = __uint_as_float(zb);
    if (!explained_by_obs(obs, fmul(rxs[lx], z), fmul(rys[ly], z), z, cam.delta2)) djr++;
  }

  // ---- dJ_o: observed points inside V(O) with no dR point within delta
  int djo = 0;
  if (obs.n > 0) {
    const float r = sqrtf(m.vol_r2) * 1.001f + 1e-6f;
    const int cx0 = max(cell_of(ox - r, obs.g2x, obs.inv2, obs.n2x) - 1, 0);
    const int cx1 = min(cell_of(ox + r, obs.g2x, obs.inv2, obs.n2x) + 1, obs.n2x - 1);
    const int cy0 = max(cell_of(oy - r, obs.g2y, obs.inv2, obs.n2y) - 1, 0);
    const int cy1 = min(cell_of(oy + r, obs.g2y, obs.inv2, obs.n2y) + 1, obs.n2y - 1);
    if (cx0 <= cx1) {
      for (int cy = cy0; cy <= cy1; ++cy) {
        const int s = obs.start2[cy * obs.n2x + cx0], e = obs.start2[cy * obs.n2x + cx1 + 1];
        for (int k = s + tid; k < e; k += kEvalThreads) {
          const float4 qw = obs.world2[k];
          if (!in_volume(qw, ox, oy, m.vol_r2, m.vol_zlo, m.vol_zhi)) continue;
          if (!explained_by_tile(cam, obs.cam2[k], tile, rxs, rys, bb)) djo++;
        }
      }
    }
  }

  // ---- residual(K) on edges into the last level
  int resid = 0;
  if (plen + 1 == b.K_total) {
    const int nu = b.uset_count[pid];
    const int* U = b.uset + (size_t)pid * b.uset_stride;
    for (int k = tid; k < nu; k += kEvalThreads) {
      const int qi = U[k];
      if (in_volume(obs.world2[qi], ox, oy, m.vol_r2, m.vol_zlo, m.vol_zhi)) continue;
      if (explained_by_tile(cam, obs.cam2[qi], tile, rxs, rys, bb)) continue;
      resid++;
    }
  }
  djr = warp_sum(djr);
  djo = warp_sum(djo);
  resid = warp_sum(resid);
  if (lane == 0) {
    if (djr) atomicAdd(&s_cnt[3], djr);
    if (djo) atomicAdd(&s_cnt[4], djo);
    if (resid) atomicAdd(&s_cnt[5], resid);
  }
  __syncthreads();
  if (tid == 0) {
    perch_cost r = {s_cnt[3], s_cnt[4], s_cnt[5], 0, s_cnt[1], flags};
    b.out[h] = r;
  }
}

cudaError_t launch_eval(const Camera& cam, const Geometry& g, const ObsIndex& obs, const Batch& b,
                        cudaStream_t s) {
  if (b.n_hyp == 0) return cudaSuccess;
  if (b.n_hyp > 0x7fffffffLL) return cudaErrorInvalidValue;
  const size_t smem = eval_smem_bytes(b.tile_w, b.tile_h);
  cudaError_t e = cudaFuncSetAttribute(k_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_eval<<<(unsigned)b.n_hyp, kEvalThreads, smem, s>>>(cam, g, obs, b);
  return cudaGetLastError();
}

}  // namespace perch
