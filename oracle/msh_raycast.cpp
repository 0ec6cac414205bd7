// CPU oracle of the depth cameras -- TEST INFRASTRUCTURE ONLY.
//
// Only tests/, the smoke check and the benchmark's CPU legs may load this
// code (it is linked into the oracle library). The paper's environments
// render two 128x128 RGB-D cameras per env (Sec. 4.2); the graphics renderer
// it uses is unavailable here, so the depth channel is restated as ray
// casting against the env's primitives. Readings (shared with the CUDA path):
//   * pinhole camera looking along its frame's +x, image right = -y, image
//     down = -z; pixel (row, col) has centre (col + 1/2, row + 1/2); focal
//     length in pixels f = (H/2) / tan(fov_y/2), given by the caller;
//   * a camera is mounted on a body (pose composed with the body's pose) or
//     on the world;
//   * the ray through a pixel is D = R_cam (1, -(u - W/2)/f, -(v - H/2)/f), so
//     its parameter s is the z-depth (distance along the optical axis); the
//     pixel's depth is the smallest s in [near, far] over all spheres,
//     capsules (cylinder plus end spheres), boxes (slabs) and the ground
//     plane, 0 when nothing is hit;
//   * every intersection is the textbook closed form, evaluated without FMA
//     contraction in a fixed order, so FP32 results are reproducible; the
//     distances are products with reciprocals rounded once (1/(D.D) per ray
//     for the sphere roots, 1/A per cylinder, 1/D_i per box axis) rather than
//     quotients.
// Brute force: every pixel tests every primitive.

#include <cmath>
#include <cstdint>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
struct OracleScene;   // defined in msh_oracle.cpp
struct OracleCams {
  int32_t ncam, width, height;
  float focal, near_, far_;
  const int32_t* body;   // [E][ncam] env-local mount body, -1 = world
  const float* pose;     // [E][ncam][7] mount-local (or world) position, quaternion (w,x,y,z)
};
struct OracleRayScene {  // the parts of the scene the cameras see
  int32_t num_envs;
  const int32_t* body_off;
  const int32_t* static_off;
  const int32_t* body_shape;
  const float* body_dims;
  const float* static_pose;
  const float* static_half;
};
}

namespace ray {

template <class R> struct V { R x, y, z; };
template <class R> inline V<R> mk(R x, R y, R z) { V<R> v; v.x = x; v.y = y; v.z = z; return v; }
template <class R> inline V<R> sub(V<R> a, V<R> b) { return mk<R>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class R> inline V<R> add(V<R> a, V<R> b) { return mk<R>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class R> inline V<R> scl(V<R> a, R s) { return mk<R>(a.x * s, a.y * s, a.z * s); }
template <class R> inline R dot(V<R> a, V<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// rotation matrix of a unit quaternion (w, x, y, z)
template <class R> void qmat(R w, R x, R y, R z, R M[3][3]) {
  R xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
  M[0][0] = R(1) - R(2) * (yy + zz); M[0][1] = R(2) * (xy - wz); M[0][2] = R(2) * (xz + wy);
  M[1][0] = R(2) * (xy + wz); M[1][1] = R(1) - R(2) * (xx + zz); M[1][2] = R(2) * (yz - wx);
  M[2][0] = R(2) * (xz - wy); M[2][1] = R(2) * (yz + wx); M[2][2] = R(1) - R(2) * (xx + yy);
}
template <class R> V<R> mul(const R M[3][3], V<R> v) {
  return mk<R>(M[0][0] * v.x + M[0][1] * v.y + M[0][2] * v.z, M[1][0] * v.x + M[1][1] * v.y + M[1][2] * v.z,
               M[2][0] * v.x + M[2][1] * v.y + M[2][2] * v.z);
}
template <class R> V<R> mulT(const R M[3][3], V<R> v) {
  return mk<R>(M[0][0] * v.x + M[1][0] * v.y + M[2][0] * v.z, M[0][1] * v.x + M[1][1] * v.y + M[2][1] * v.z,
               M[0][2] * v.x + M[1][2] * v.y + M[2][2] * v.z);
}
// quaternion product a (x) b
template <class R> void qmul(const R* a, const R* b, R* o) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Smallest root s >= near of |w + s D|^2 = r^2 (w = origin - centre); inf if
// none. a = D.D and ia = 1 / a belong to the ray (formed once per pixel); the
// roots are (-b -+ sqrt(disc)) * ia.
template <class R> R hit_sphere(V<R> w, V<R> D, R a, R ia, R r, R near_) {
  const R b = dot(D, w), c = dot(w, w) - r * r;
  const R disc = b * b - a * c;
  if (disc < R(0)) return std::numeric_limits<R>::infinity();
  const R sq = std::sqrt(disc);
  R s = (-b - sq) * ia;
  if (s >= near_) return s;
  s = (-b + sq) * ia;
  return s >= near_ ? s : std::numeric_limits<R>::infinity();
}

// Slab test in the box frame (o, D already rotated into it).
template <class R> R hit_box(V<R> o, V<R> D, const R* h, R near_) {
  const R inf = std::numeric_limits<R>::infinity();
  R tmin = -inf, tmax = inf;
  const R oo[3] = {o.x, o.y, o.z}, dd[3] = {D.x, D.y, D.z};
  for (int i = 0; i < 3; ++i) {
    if (dd[i] == R(0)) {
      if (oo[i] < -h[i] || oo[i] > h[i]) return inf;
      continue;
    }
    const R inv = R(1) / dd[i];   // one reciprocal per axis, then products
    R t1 = (-h[i] - oo[i]) * inv, t2 = (h[i] - oo[i]) * inv;
    R lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
    if (lo > tmin) tmin = lo;
    if (hi < tmax) tmax = hi;
  }
  if (tmax < tmin || tmax < near_) return inf;
  return tmin >= near_ ? tmin : tmax;
}

// Capsule along unit axis a through centre c, half length L, radius r:
// the cylinder's side between the caps, then the two end spheres.
template <class R> R hit_capsule(V<R> w, V<R> D, R dd, R idd, V<R> a, R L, R r, R near_) {
  const R inf = std::numeric_limits<R>::infinity();
  R best = inf;
  const R Da = dot(D, a), wa = dot(w, a);
  const V<R> Dp = sub(D, scl(a, Da)), wp = sub(w, scl(a, wa));
  const R A = dot(Dp, Dp), B = dot(Dp, wp), C = dot(wp, wp) - r * r;
  if (A > R(0)) {
    const R disc = B * B - A * C;
    if (disc >= R(0)) {
      const R sq = std::sqrt(disc);
      const R iA = R(1) / A;
      const R s1 = (-B - sq) * iA, s2 = (-B + sq) * iA;
      const R ss[2] = {s1, s2};
      for (int k = 0; k < 2; ++k) {
        const R s = ss[k];
        if (s < near_) continue;
        const R ax = wa + s * Da;
        if (ax >= -L && ax <= L) { best = s; break; }
      }
    }
  }
  const R s0 = hit_sphere(sub(w, scl(a, L)), D, dd, idd, r, near_);
  const R s1 = hit_sphere(add(w, scl(a, L)), D, dd, idd, r, near_);
  if (s0 < best) best = s0;
  if (s1 < best) best = s1;
  return best;
}

template <class R, class T>
void render_env(const OracleRayScene& sc, int e, const T* pos, const T* quat, const OracleCams& cm, T* depth) {
  const int b0 = sc.body_off[e], D = sc.body_off[e + 1] - b0;
  const int s0 = sc.static_off[e], S = sc.static_off[e + 1] - s0;
  const int W = cm.width, H = cm.height;
  const R f = R(cm.focal), cx = R(W) * R(0.5), cy = R(H) * R(0.5), near_ = R(cm.near_), far_ = R(cm.far_);
  for (int c = 0; c < cm.ncam; ++c) {
    const int mb = cm.body[e * cm.ncam + c];
    const float* lp = cm.pose + 7 * (e * cm.ncam + c);
    R p[3], q[4];
    const R ql[4] = {R(lp[3]), R(lp[4]), R(lp[5]), R(lp[6])};
    if (mb >= 0) {
      const int g = b0 + mb;
      const R qb[4] = {R(quat[4 * g]), R(quat[4 * g + 1]), R(quat[4 * g + 2]), R(quat[4 * g + 3])};
      R M[3][3];
      qmat(qb[0], qb[1], qb[2], qb[3], M);
      const V<R> o = mul(M, mk<R>(R(lp[0]), R(lp[1]), R(lp[2])));
      p[0] = R(pos[3 * g]) + o.x; p[1] = R(pos[3 * g + 1]) + o.y; p[2] = R(pos[3 * g + 2]) + o.z;
      qmul(qb, ql, q);
    } else {
      p[0] = R(lp[0]); p[1] = R(lp[1]); p[2] = R(lp[2]);
      for (int k = 0; k < 4; ++k) q[k] = ql[k];
    }
    R Mc[3][3];
    qmat(q[0], q[1], q[2], q[3], Mc);
    const V<R> o = mk<R>(p[0], p[1], p[2]);
    T* img = depth + (size_t)(e * cm.ncam + c) * W * H;
    for (int row = 0; row < H; ++row) {
      for (int col = 0; col < W; ++col) {
        const R u = R(col) + R(0.5), v = R(row) + R(0.5);
        const V<R> dc = mk<R>(R(1), -((u - cx) / f), -((v - cy) / f));
        const V<R> Dw = mul(Mc, dc);
        const R dd = dot(Dw, Dw), idd = R(1) / dd;
        R best = std::numeric_limits<R>::infinity();
        for (int i = 0; i < D; ++i) {
          const int g = b0 + i;
          const int sh = sc.body_shape[g];
          const V<R> cen = mk<R>(R(pos[3 * g]), R(pos[3 * g + 1]), R(pos[3 * g + 2]));
          const V<R> w = sub(o, cen);
          R s;
          if (sh == 0) {
            s = hit_sphere(w, Dw, dd, idd, R(sc.body_dims[4 * g]), near_);
          } else {
            R M[3][3];
            qmat(R(quat[4 * g]), R(quat[4 * g + 1]), R(quat[4 * g + 2]), R(quat[4 * g + 3]), M);
            if (sh == 1) {
              s = hit_capsule(w, Dw, dd, idd, mk<R>(M[0][0], M[1][0], M[2][0]), R(sc.body_dims[4 * g + 1]),
                              R(sc.body_dims[4 * g]), near_);
            } else {
              const R h[3] = {R(sc.body_dims[4 * g]), R(sc.body_dims[4 * g + 1]), R(sc.body_dims[4 * g + 2])};
              s = hit_box(mulT(M, w), mulT(M, Dw), h, near_);
            }
          }
          if (s < best) best = s;
        }
        for (int k = 0; k < S; ++k) {
          const float* sp = sc.static_pose + 7 * (s0 + k);
          const float* hh = sc.static_half + 3 * (s0 + k);
          R M[3][3];
          qmat(R(sp[3]), R(sp[4]), R(sp[5]), R(sp[6]), M);
          const V<R> w = sub(o, mk<R>(R(sp[0]), R(sp[1]), R(sp[2])));
          const R h[3] = {R(hh[0]), R(hh[1]), R(hh[2])};
          const R s = hit_box(mulT(M, w), mulT(M, Dw), h, near_);
          if (s < best) best = s;
        }
        if (Dw.z < R(0)) {   // ground plane z = 0
          const R s = -o.z / Dw.z;
          if (s >= near_ && s < best) best = s;
        }
        img[row * W + col] = T(best <= far_ ? best : R(0));
      }
    }
  }
}

}  // namespace ray

extern "C" {
int oracle_render_depth_f32(const OracleRayScene* sc, const float* pos, const float* quat, const OracleCams* cm,
                            float* depth, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int e = 0; e < sc->num_envs; ++e) ray::render_env<float, float>(*sc, e, pos, quat, *cm, depth);
  return 0;
}
int oracle_render_depth_f64(const OracleRayScene* sc, const double* pos, const double* quat, const OracleCams* cm,
                            double* depth, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int e = 0; e < sc->num_envs; ++e) ray::render_env<double, double>(*sc, e, pos, quat, *cm, depth);
  return 0;
}
}
