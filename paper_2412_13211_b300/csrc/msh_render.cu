// Depth cameras: per env and camera, a depth image ray-cast against the env's
// primitives (the paper's environments render two 128x128 RGB-D cameras per
// env, Sec. 4.2; its graphics renderer is replaced here by the depth channel
// computed directly).
//
// Camera model (readings): pinhole looking along the camera frame's +x, image
// right = -y, image down = -z; pixel (row, col) centre (col + 1/2, row + 1/2);
// focal length in pixels f = (H/2) / tan(fov_y / 2); a camera is mounted on a
// body (its pose composed with the body's) or on the world. The ray through a
// pixel is D = R_cam (1, -(u - W/2)/f, -(v - H/2)/f), so the ray parameter is
// the z-depth; a pixel's depth is the smallest parameter in [near, far] over
// spheres, capsules (cylinder and end spheres), boxes (slabs) and the ground
// plane z = 0, or 0 when nothing is hit. Every closed form is evaluated in
// IEEE FP32 without FMA contraction (the library is built with -fmad=false),
// in a fixed operation order.
//
// Kernel: one CTA (8 warps) per 32x32 tile of one camera of one env. The CTA
// builds the env's primitives in world space with widened bounding spheres;
// each warp then keeps those meeting the view frustum of its own 8x16 pixel
// block and orders them by the smallest z-depth their bounding sphere allows.
// A pixel walks that order and stops at the first primitive that cannot come
// nearer than its current hit. Both tests are conservative (bounding spheres
// widened by 1 % and 1 mm), so the result is the brute-force minimum.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/msh.h"
#include "msh_render.h"

int msh_fail(int code, const char* msg);

namespace {

enum { TILE = 32, RT_THREADS = 256, PRIM_F = 16 };
enum { PR_SPHERE = 0, PR_CAPSULE = 1, PR_BOX = 2 };
enum { SW_C = 0, SW_M = 1, SW_N = 6 };   // static box record layout (RenderScene::sworld)

__device__ __forceinline__ float3 mk3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 scl3(float3 a, float s) { return mk3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// rotation matrix rows of a unit quaternion (w, x, y, z)
__device__ __forceinline__ void qmat3(float w, float x, float y, float z, float M[3][3]) {
  float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
  M[0][0] = 1.f - 2.f * (yy + zz); M[0][1] = 2.f * (xy - wz); M[0][2] = 2.f * (xz + wy);
  M[1][0] = 2.f * (xy + wz); M[1][1] = 1.f - 2.f * (xx + zz); M[1][2] = 2.f * (yz - wx);
  M[2][0] = 2.f * (xz - wy); M[2][1] = 2.f * (yz + wx); M[2][2] = 1.f - 2.f * (xx + yy);
}
__device__ __forceinline__ float3 mul3(const float M[3][3], float3 v) {
  return mk3(M[0][0] * v.x + M[0][1] * v.y + M[0][2] * v.z, M[1][0] * v.x + M[1][1] * v.y + M[1][2] * v.z,
             M[2][0] * v.x + M[2][1] * v.y + M[2][2] * v.z);
}

// Smallest root s >= near of |w + s D|^2 = r^2 (w = origin - centre).
// a = D.D and ia = 1/a belong to the ray (once per pixel): the roots are
// products with the reciprocal, as the oracle forms them.
__device__ __forceinline__ float hit_sphere(float3 w, float3 D, float a, float ia, float r, float near_) {
  const float b = dot3(D, w), c = dot3(w, w) - r * r;
  const float disc = b * b - a * c;
  if (disc < 0.f) return INFINITY;
  const float sq = sqrtf(disc);
  float s = (-b - sq) * ia;
  if (s >= near_) return s;
  s = (-b + sq) * ia;
  return s >= near_ ? s : INFINITY;
}

// Slab test with origin and direction in the box frame.
__device__ __forceinline__ float hit_box(float3 o, float3 D, float3 h, float near_) {
  float tmin = -INFINITY, tmax = INFINITY;
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {D.x, D.y, D.z}, hh[3] = {h.x, h.y, h.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (dd[i] == 0.f) {
      if (oo[i] < -hh[i] || oo[i] > hh[i]) return INFINITY;
      continue;
    }
    const float inv = 1.f / dd[i];
    const float t1 = (-hh[i] - oo[i]) * inv, t2 = (hh[i] - oo[i]) * inv;
    const float lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
    if (lo > tmin) tmin = lo;
    if (hi < tmax) tmax = hi;
  }
  if (tmax < tmin || tmax < near_) return INFINITY;
  return tmin >= near_ ? tmin : tmax;
}

__device__ __forceinline__ float hit_capsule(float3 w, float3 D, float dd, float idd, float3 a, float L, float r,
                                             float near_) {
  float best = INFINITY;
  const float Da = dot3(D, a), wa = dot3(w, a);
  const float3 Dp = sub3(D, scl3(a, Da)), wp = sub3(w, scl3(a, wa));
  const float A = dot3(Dp, Dp), B = dot3(Dp, wp), C = dot3(wp, wp) - r * r;
  if (A > 0.f) {
    const float disc = B * B - A * C;
    if (disc >= 0.f) {
      const float sq = sqrtf(disc);
      const float iA = 1.f / A;
      const float s1 = (-B - sq) * iA, s2 = (-B + sq) * iA;
      if (s1 >= near_ && wa + s1 * Da >= -L && wa + s1 * Da <= L) best = s1;
      else if (s2 >= near_ && wa + s2 * Da >= -L && wa + s2 * Da <= L) best = s2;
    }
  }
  const float e0 = hit_sphere(sub3(w, scl3(a, L)), D, dd, idd, r, near_);
  const float e1 = hit_sphere(add3(w, scl3(a, L)), D, dd, idd, r, near_);
  if (e0 < best) best = e0;
  if (e1 < best) best = e1;
  return best;
}

// The camera's world position and rotation (rows).
__device__ __forceinline__ void camera_pose(const RenderScene& p, const RenderCams& cm, int env, int b0, int c, float3& o,
                                            float Mc[3][3]) {
  const int mb = cm.body[env * cm.ncam + c];
  const float* lp = cm.pose + 7 * (env * cm.ncam + c);
  const float ql[4] = {lp[3], lp[4], lp[5], lp[6]};
  float q[4];
  if (mb >= 0) {
    const int g = b0 + mb;
    const float qb[4] = {p.quat[4 * g], p.quat[4 * g + 1], p.quat[4 * g + 2], p.quat[4 * g + 3]};
    float M[3][3];
    qmat3(qb[0], qb[1], qb[2], qb[3], M);
    const float3 off = mul3(M, mk3(lp[0], lp[1], lp[2]));
    o = mk3(p.pos[3 * g] + off.x, p.pos[3 * g + 1] + off.y, p.pos[3 * g + 2] + off.z);
    q[0] = qb[0] * ql[0] - qb[1] * ql[1] - qb[2] * ql[2] - qb[3] * ql[3];
    q[1] = qb[0] * ql[1] + qb[1] * ql[0] + qb[2] * ql[3] - qb[3] * ql[2];
    q[2] = qb[0] * ql[2] - qb[1] * ql[3] + qb[2] * ql[0] + qb[3] * ql[1];
    q[3] = qb[0] * ql[3] + qb[1] * ql[2] - qb[2] * ql[1] + qb[3] * ql[0];
  } else {
    o = mk3(lp[0], lp[1], lp[2]);
    q[0] = ql[0]; q[1] = ql[1]; q[2] = ql[2]; q[3] = ql[3];
  }
  qmat3(q[0], q[1], q[2], q[3], Mc);
}

// Inward unit normals of the four side planes of the view frustum through
// pixel rectangle [u0, u1] x [v0, v1] (pixel-edge coordinates).
__device__ __forceinline__ void frustum(const float Mc[3][3], float f, float cx, float cy, float u0, float u1,
                                        float v0, float v1, float3 nrm[4]) {
  const float3 cr[4] = {mul3(Mc, mk3(1.f, -((u0 - cx) / f), -((v0 - cy) / f))),
                        mul3(Mc, mk3(1.f, -((u1 - cx) / f), -((v0 - cy) / f))),
                        mul3(Mc, mk3(1.f, -((u1 - cx) / f), -((v1 - cy) / f))),
                        mul3(Mc, mk3(1.f, -((u0 - cx) / f), -((v1 - cy) / f)))};
  const float3 mid = mul3(Mc, mk3(1.f, -((0.5f * (u0 + u1) - cx) / f), -((0.5f * (v0 + v1) - cy) / f)));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float3 a = cr[k], b = cr[(k + 1) & 3];
    float3 n = mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
    if (dot3(n, mid) < 0.f) n = scl3(n, -1.f);
    nrm[k] = scl3(n, 1.f / sqrtf(dot3(n, n)));
  }
}

enum { WB_W = 8, WB_H = 16, WARPS = RT_THREADS / 32 };

__global__ void __launch_bounds__(RT_THREADS) k_render(RenderScene p, RenderCams cm, float* depth) {
  __shared__ float s_prim[MSH_RENDER_MAX_PRIMS * PRIM_F];
  __shared__ float4 s_bs[MSH_RENDER_MAX_PRIMS];                // widened bounding sphere: centre - camera, radius
  __shared__ float s_near[WARPS][MSH_RENDER_MAX_PRIMS];        // per warp: near bound of each kept primitive
  __shared__ unsigned char s_keep[WARPS][MSH_RENDER_MAX_PRIMS];
  __shared__ unsigned char s_order[WARPS][MSH_RENDER_MAX_PRIMS];
  const int env = blockIdx.z, c = blockIdx.y;
  const int tiles_x = (cm.width + TILE - 1) / TILE;
  const int tx0 = (blockIdx.x % tiles_x) * TILE, ty0 = (blockIdx.x / tiles_x) * TILE;
  const int b0 = p.body_off[env], D = p.body_off[env + 1] - b0;
  const int s0 = p.static_off[env], S = p.static_off[env + 1] - s0;
  float3 o;
  float Mc[3][3];
  camera_pose(p, cm, env, b0, c, o, Mc);
  const float f = cm.focal, cx = (float)cm.width * 0.5f, cy = (float)cm.height * 0.5f;
  const float3 fwd = mk3(Mc[0][0], Mc[1][0], Mc[2][0]);
  // the env's primitives in world space
  for (int i = threadIdx.x; i < D + S; i += blockDim.x) {
    float rec[PRIM_F];
    float3 cen;
    float rho;
    if (i < D) {
      const int g = b0 + i;
      const float4 dm = p.bdims[g];
      const int sh = __float_as_int(dm.w);
      cen = mk3(p.pos[3 * g], p.pos[3 * g + 1], p.pos[3 * g + 2]);
      rec[1] = cen.x; rec[2] = cen.y; rec[3] = cen.z;
      if (sh == 0) {
        rec[0] = __int_as_float(PR_SPHERE); rec[4] = dm.x;
        rho = dm.x;
      } else {
        float M[3][3];
        qmat3(p.quat[4 * g], p.quat[4 * g + 1], p.quat[4 * g + 2], p.quat[4 * g + 3], M);
        if (sh == 1) {
          rec[0] = __int_as_float(PR_CAPSULE);
          rec[4] = M[0][0]; rec[5] = M[1][0]; rec[6] = M[2][0];   // axis: local x
          rec[7] = dm.y; rec[8] = dm.x;                           // half length, radius
          rho = dm.y + dm.x;
        } else {
          rec[0] = __int_as_float(PR_BOX);
#pragma unroll
          for (int r = 0; r < 3; ++r) { rec[4 + 3 * r] = M[r][0]; rec[5 + 3 * r] = M[r][1]; rec[6 + 3 * r] = M[r][2]; }
          rec[13] = dm.x; rec[14] = dm.y; rec[15] = dm.z;
          rho = sqrtf(dm.x * dm.x + dm.y * dm.y + dm.z * dm.z);
        }
      }
    } else {
      const float4* sw = p.sworld + (size_t)SW_N * (s0 + i - D);
      const float4 cc = sw[SW_C], m0 = sw[SW_M], m1 = sw[SW_M + 1], m2 = sw[SW_M + 2];
      cen = mk3(cc.x, cc.y, cc.z);
      rec[0] = __int_as_float(PR_BOX);
      rec[1] = cen.x; rec[2] = cen.y; rec[3] = cen.z;
      rec[4] = m0.x; rec[5] = m0.y; rec[6] = m0.z;
      rec[7] = m1.x; rec[8] = m1.y; rec[9] = m1.z;
      rec[10] = m2.x; rec[11] = m2.y; rec[12] = m2.z;
      rec[13] = m0.w; rec[14] = m1.w; rec[15] = m2.w;
      rho = sqrtf(m0.w * m0.w + m1.w * m1.w + m2.w * m2.w);
    }
    float* dst = s_prim + i * PRIM_F;
#pragma unroll
    for (int q = 0; q < PRIM_F; ++q) dst[q] = rec[q];
    // widened by 1 % and 1 mm so that rounding never drops a primitive that a ray hits
    const float3 w = sub3(cen, o);
    s_bs[i] = make_float4(w.x, w.y, w.z, rho * 1.01f + 1e-3f);
  }
  __syncthreads();
  // per warp: the primitives meeting its block's frustum, in near-bound order
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx0 = tx0 + (warp % (TILE / WB_W)) * WB_W, by0 = ty0 + (warp / (TILE / WB_W)) * WB_H;
  float3 nrm[4];
  frustum(Mc, f, cx, cy, (float)bx0, (float)min(bx0 + WB_W, cm.width), (float)by0, (float)min(by0 + WB_H, cm.height),
          nrm);
  int n = 0;
  for (int base = 0; base < D + S; base += 32) {
    const int i = base + lane;
    bool keep = false;
    float nb = 0.f;
    if (i < D + S) {
      const float4 bs = s_bs[i];
      const float3 w = mk3(bs.x, bs.y, bs.z);
      const float zc = dot3(w, fwd);
      keep = zc >= cm.near_ - bs.w && zc <= cm.far_ + bs.w;
#pragma unroll
      for (int k = 0; k < 4; ++k) keep = keep && dot3(nrm[k], w) >= -bs.w;
      nb = zc - bs.w;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int slot = n + __popc(m & ((1u << lane) - 1u));
      s_keep[warp][slot] = (unsigned char)i;
      s_near[warp][slot] = nb;
    }
    n += __popc(m);
  }
  __syncwarp();
  for (int a = lane; a < n; a += 32) {   // rank sort, ties by position
    const float key = s_near[warp][a];
    int rank = 0;
    for (int b = 0; b < n; ++b) {
      const float kb = s_near[warp][b];
      rank += (kb < key) || (kb == key && b < a);
    }
    s_order[warp][rank] = (unsigned char)a;
  }
  __syncwarp();
  const int col = bx0 + (lane % WB_W);
  for (int row = by0 + lane / WB_W; row < by0 + WB_H; row += 32 / WB_W) {
    if (col >= cm.width || row >= cm.height) break;
    const float u = (float)col + 0.5f, v = (float)row + 0.5f;
    const float3 Dw = mul3(Mc, mk3(1.f, -((u - cx) / f), -((v - cy) / f)));
    const float dd = dot3(Dw, Dw), idd = 1.f / dd;
    float best = INFINITY;
    if (Dw.z < 0.f) {   // ground plane z = 0
      const float s = -o.z / Dw.z;
      if (s >= cm.near_) best = s;
    }
    for (int k = 0; k < n; ++k) {
      const int a = s_order[warp][k];
      if (s_near[warp][a] > best) break;   // this and every later primitive lie beyond the current hit
      const float* pr = s_prim + s_keep[warp][a] * PRIM_F;
      const int ty = __float_as_int(pr[0]);
      const float3 w = sub3(o, mk3(pr[1], pr[2], pr[3]));
      float s;
      if (ty == PR_SPHERE) {
        s = hit_sphere(w, Dw, dd, idd, pr[4], cm.near_);
      } else if (ty == PR_CAPSULE) {
        s = hit_capsule(w, Dw, dd, idd, mk3(pr[4], pr[5], pr[6]), pr[7], pr[8], cm.near_);
      } else {
        // box frame: R^T w and R^T D, with R's rows in pr[4..12]
        const float3 ob = mk3(pr[4] * w.x + pr[7] * w.y + pr[10] * w.z, pr[5] * w.x + pr[8] * w.y + pr[11] * w.z,
                              pr[6] * w.x + pr[9] * w.y + pr[12] * w.z);
        const float3 db = mk3(pr[4] * Dw.x + pr[7] * Dw.y + pr[10] * Dw.z,
                              pr[5] * Dw.x + pr[8] * Dw.y + pr[11] * Dw.z,
                              pr[6] * Dw.x + pr[9] * Dw.y + pr[12] * Dw.z);
        s = hit_box(ob, db, mk3(pr[13], pr[14], pr[15]), cm.near_);
      }
      if (s < best) best = s;
    }
    depth[(((size_t)env * cm.ncam + c) * cm.height + row) * cm.width + col] = best <= cm.far_ ? best : 0.f;
  }
}

}  // namespace

int msh_render_launch(const RenderScene& sc, const RenderCams& cm, float* depth, cudaStream_t s) {
  if (sc.E == 0) return MSH_OK;
  const int tiles = ((cm.width + TILE - 1) / TILE) * ((cm.height + TILE - 1) / TILE);
  dim3 grid(tiles, cm.ncam, sc.E);
  k_render<<<grid, RT_THREADS, 0, s>>>(sc, cm, depth);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MSH_OK : msh_fail(MSH_ERR_CUDA, cudaGetErrorString(e));
}
