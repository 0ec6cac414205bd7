// CPU oracle of the batched rigid-body step -- TEST INFRASTRUCTURE ONLY.
//
// Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
// this library. It is a plain, slow, per-environment restatement of the step
// used as the parity reference for the CUDA library, and it shares no code
// with it. Templated on the scalar: float (FP32 oracle), double (FP64 oracle)
// and Dual<N> (forward-mode derivatives for reference gradients).
//
// The ManiSkill-HAB paper (Sec. 4.1-4.2) runs its environments at a 100 Hz
// simulation rate with PD joint targets and base velocity control, but it does
// not describe the physics step itself. The scheme below is the written
// reading of the step (integrate, AABB broadphase, primitive narrowphase to
// contact manifolds, graph-coloured projected Gauss-Seidel or Jacobi solve over
// substeps, position update); each function names the method it follows:
//   * symplectic Euler with world-frame angular velocity, no gyroscopic term;
//     quaternion update q += h/2 (0,w) q, then normalise;
//   * inclusive AABB overlap, pairs in (i<j) lexicographic order, dynamic
//     bodies before static boxes, the ground plane last;
//   * closed-form sphere/plane manifolds, Ericson's segment-segment closest
//     points (Real-Time Collision Detection, 5.1.9), separating-axis test over
//     15 axes with Sutherland-Hodgman clipping for box-box;
//   * sequential impulses (Catto 2005) with speculative contacts, Coulomb
//     friction on two tangents from Duff et al. 2017's orthonormal basis,
//     soft PD drives in Catto's 2011 soft-constraint form, Baumgarte joints;
//   * greedy graph colouring (joints first, then manifolds) for PGS; Jacobi
//     with Tonge et al. 2012 mass splitting as the variant.
// Pinned by brute force (tests/test_oracle_manifolds.py): capsule-capsule,
// capsule-box (outside and entering), box-box face and edge manifolds,
// sphere centres inside boxes, and the clipper's 8-vertex cap (never reached
// on near-degenerate face pairs, in FP32 and FP64); every dynamic pair's
// manifold is equivariant under a rigid motion of both shapes
// (tests/test_oracle_equivariance.py).
//
// Compile with -ffp-contract=off: the collision stages (AABB, broadphase,
// narrowphase) must be bit-reproducible in FP32 from identical inputs.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// --------------------------------------------------------------------------
// Scalars: float, double and forward-mode dual numbers
// --------------------------------------------------------------------------
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0) { for (int i = 0; i < N; ++i) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0; }  // NOLINT
};
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int N> inline bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N> inline bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }
template <int N> inline bool operator<=(const Dual<N>& a, const Dual<N>& b) { return a.v <= b.v; }
template <int N> inline bool operator>=(const Dual<N>& a, const Dual<N>& b) { return a.v >= b.v; }
template <int N> inline bool operator==(const Dual<N>& a, const Dual<N>& b) { return a.v == b.v; }
template <int N> inline bool operator!=(const Dual<N>& a, const Dual<N>& b) { return a.v != b.v; }

inline float sqrt_(float x) { return std::sqrt(x); }
inline double sqrt_(double x) { return std::sqrt(x); }
template <int N> inline Dual<N> sqrt_(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = r.v > 0 ? a.d[i] / (2.0 * r.v) : 0.0;
  return r; }
inline float abs_(float x) { return std::fabs(x); }
inline double abs_(double x) { return std::fabs(x); }
template <int N> inline Dual<N> abs_(const Dual<N>& a) { return a.v < 0 ? -a : a; }
inline float atan2_(float y, float x) { return std::atan2(y, x); }
inline double atan2_(double y, double x) { return std::atan2(y, x); }
template <int N> inline Dual<N> atan2_(const Dual<N>& y, const Dual<N>& x) {
  Dual<N> r; r.v = std::atan2(y.v, x.v);
  double den = x.v * x.v + y.v * y.v;
  for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / den;
  return r; }
// Reverse mode (the basic operator-overloading scheme of Griewank and
// Walther, "Evaluating Derivatives", 2nd ed., Ch. 3 and 6): every result of an
// arithmetic operation on a Rev is a node of the calling thread's tape that
// stores the local partial derivatives with respect to its operands (at most
// two); a sweep over the tape from the last node to the first accumulates the
// adjoints of all nodes. The primal value has its own type P: with P = float
// the primal arithmetic is exactly the FP32 oracle's (same operations in the
// same order), so every branch decision equals the FP32 oracle's; partials and
// adjoints are carried in double. Constants carry id -1 and record nothing.
struct RevNode { int a, b; double da, db; };
struct RevTape {
  std::vector<RevNode> nodes;
  std::vector<double> adj;
  int push(int a, double da, int b, double db) {
    RevNode n; n.a = a; n.b = b; n.da = da; n.db = db;
    nodes.push_back(n);
    return (int)nodes.size() - 1;
  }
  // adjoints of every node, seeded beforehand through adj (sized by seed())
  void seed(int id, double w) {
    if (id < 0) return;
    if (adj.size() != nodes.size()) adj.resize(nodes.size(), 0.0);
    adj[id] += w;
  }
  void sweep() {
    if (adj.size() != nodes.size()) adj.resize(nodes.size(), 0.0);
    for (int i = (int)nodes.size() - 1; i >= 0; --i) {
      const double w = adj[i];
      if (w == 0.0) continue;
      const RevNode& n = nodes[i];
      if (n.a >= 0) adj[n.a] += n.da * w;
      if (n.b >= 0) adj[n.b] += n.db * w;
    }
  }
  double get(int id) const { return id >= 0 && id < (int)adj.size() ? adj[id] : 0.0; }
  void clear() { nodes.clear(); adj.clear(); }
};
inline RevTape*& rev_tape() { static thread_local RevTape* t = nullptr; return t; }

template <class P> struct Rev {
  P v;
  int id;
  Rev() : v(0), id(-1) {}
  Rev(double x) : v(P(x)), id(-1) {}  // NOLINT
  static Rev make(P value, int a, double da, int b, double db) {
    Rev r; r.v = value;
    r.id = (a < 0 && b < 0) ? -1 : rev_tape()->push(a, da, b, db);
    return r;
  }
  static Rev leaf(P value) { Rev r; r.v = value; r.id = rev_tape()->push(-1, 0.0, -1, 0.0); return r; }
};
template <class P> inline Rev<P> operator+(const Rev<P>& a, const Rev<P>& b) {
  return Rev<P>::make(a.v + b.v, a.id, 1.0, b.id, 1.0); }
template <class P> inline Rev<P> operator-(const Rev<P>& a, const Rev<P>& b) {
  return Rev<P>::make(a.v - b.v, a.id, 1.0, b.id, -1.0); }
template <class P> inline Rev<P> operator-(const Rev<P>& a) { return Rev<P>::make(-a.v, a.id, -1.0, -1, 0.0); }
template <class P> inline Rev<P> operator*(const Rev<P>& a, const Rev<P>& b) {
  return Rev<P>::make(a.v * b.v, a.id, (double)b.v, b.id, (double)a.v); }
template <class P> inline Rev<P> operator/(const Rev<P>& a, const Rev<P>& b) {
  const double bv = b.v;
  return Rev<P>::make(a.v / b.v, a.id, 1.0 / bv, b.id, -(double)a.v / (bv * bv)); }
template <class P> inline bool operator<(const Rev<P>& a, const Rev<P>& b) { return a.v < b.v; }
template <class P> inline bool operator>(const Rev<P>& a, const Rev<P>& b) { return a.v > b.v; }
template <class P> inline bool operator<=(const Rev<P>& a, const Rev<P>& b) { return a.v <= b.v; }
template <class P> inline bool operator>=(const Rev<P>& a, const Rev<P>& b) { return a.v >= b.v; }
template <class P> inline bool operator==(const Rev<P>& a, const Rev<P>& b) { return a.v == b.v; }
template <class P> inline bool operator!=(const Rev<P>& a, const Rev<P>& b) { return a.v != b.v; }
template <class P> inline Rev<P> sqrt_(const Rev<P>& a) {
  const P r = std::sqrt(a.v);
  return Rev<P>::make(r, a.id, r > P(0) ? 0.5 / (double)r : 0.0, -1, 0.0); }
template <class P> inline Rev<P> abs_(const Rev<P>& a) { return a.v < P(0) ? -a : a; }
template <class P> inline Rev<P> atan2_(const Rev<P>& y, const Rev<P>& x) {
  const double xv = x.v, yv = y.v, den = xv * xv + yv * yv;
  return Rev<P>::make(std::atan2(y.v, x.v), y.id, xv / den, x.id, -yv / den); }

inline double val(float x) { return x; }
inline double val(double x) { return x; }
template <int N> inline double val(const Dual<N>& a) { return a.v; }
template <class P> inline double val(const Rev<P>& a) { return a.v; }
template <class R> inline bool finite_(const R& x) { return std::isfinite(val(x)); }

template <class R> inline R clampv(R x, R lo, R hi) { return x < lo ? lo : (x > hi ? hi : x); }
// The solver's impulse clamp to [lo, hi]: at an exact tie with a bound the
// bound is returned (the clamp counts as active). The value is the same
// either way, but derivatives then follow the bound; for a zero-width
// interval (lo == hi, e.g. a friction limit mu * lambda_n with lambda_n = 0)
// that is the only consistent choice, since the clamped impulse cannot move
// away from it.
template <class R> inline R clamp_active(R x, R lo, R hi) { return x <= lo ? lo : (x >= hi ? hi : x); }

// Branch decisions of a step whose outcome rounding can decide. The step is
// piecewise smooth; a decision taken at a value within rounding of its
// threshold (an impulse within noise of its clamp bound, a joint-limit error
// or a contact separation within noise of a kink of the bias) could go the
// other way in another correct FP32 evaluation, and with it the derivative.
// While a log is installed (reverse-mode adjoints only), every such decision
// of the step gets the next index; those closer to their threshold than the
// log's margins are listed as fragile, and the ones named in `flip` are taken
// the other way (the other one-sided piece of the step).
struct DecisionLog {
  int next = 0;
  double delta = 1e-4;     // impulse clamps: distance to the bound over the update's magnitude
  double len_tol = 1e-6;   // joint limits and contact biases: absolute distance (m or rad)
  int site = -1;           // solver row of the decision being taken (-1: a geometric branch)
  int choice = 0;          // its natural outcome: 0 free (or the branch's first case), 1 clamped (or the second)
  std::vector<int> fragile, fragile_site, fragile_choice;
  std::vector<double> fragile_margin;
  const int* flip = nullptr;
  int nflip = 0;
};
inline DecisionLog*& dec_log() { static thread_local DecisionLog* d = nullptr; return d; }

// Records the next decision with the given margin and threshold; returns
// whether it is to be inverted. No log: nothing is recorded, nothing inverted.
inline bool decision(double margin, double thr) {
  DecisionLog* d = dec_log();
  if (!d) return false;
  const int idx = d->next++;
  if (margin < thr) {
    d->fragile.push_back(idx);
    d->fragile_site.push_back(d->site);
    d->fragile_choice.push_back(d->choice);
    d->fragile_margin.push_back(margin);
  }
  d->site = -1;
  d->choice = 0;
  for (int i = 0; i < d->nflip; ++i)
    if (d->flip[i] == idx) return true;
  return false;
}
inline double dec_tol() { return dec_log() ? dec_log()->len_tol : 0.0; }
template <class R> inline R maxv(R a, R b) { return a > b ? a : b; }
template <class R> inline R minv(R a, R b) { return a < b ? a : b; }

// --------------------------------------------------------------------------
// Vectors, quaternions (w,x,y,z), 3x3 matrices
// --------------------------------------------------------------------------
template <class R> struct V3 { R x, y, z; };
template <class R> struct Q4 { R w, x, y, z; };
template <class R> struct M3 { R m[3][3]; };

template <class R> inline V3<R> v3(R x, R y, R z) { V3<R> r; r.x = x; r.y = y; r.z = z; return r; }
template <class R> inline V3<R> operator+(const V3<R>& a, const V3<R>& b) { return v3<R>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class R> inline V3<R> operator-(const V3<R>& a, const V3<R>& b) { return v3<R>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class R> inline V3<R> operator-(const V3<R>& a) { return v3<R>(-a.x, -a.y, -a.z); }
template <class R> inline V3<R> operator*(const V3<R>& a, R s) { return v3<R>(a.x * s, a.y * s, a.z * s); }
template <class R> inline R dot(const V3<R>& a, const V3<R>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class R> inline V3<R> cross(const V3<R>& a, const V3<R>& b) {
  return v3<R>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
template <class R> inline R comp(const V3<R>& a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
template <class R> inline void setc(V3<R>& a, int k, R v) { if (k == 0) a.x = v; else if (k == 1) a.y = v; else a.z = v; }
template <class R> inline V3<R> unit(int k) { V3<R> r = v3<R>(R(0), R(0), R(0)); setc(r, k, R(1)); return r; }

template <class R> inline M3<R> qmat(const Q4<R>& q) {
  R xx = q.x * q.x, yy = q.y * q.y, zz = q.z * q.z;
  R xy = q.x * q.y, xz = q.x * q.z, yz = q.y * q.z;
  R wx = q.w * q.x, wy = q.w * q.y, wz = q.w * q.z;
  const R one = R(1), two = R(2);
  M3<R> M;
  M.m[0][0] = one - two * (yy + zz); M.m[0][1] = two * (xy - wz); M.m[0][2] = two * (xz + wy);
  M.m[1][0] = two * (xy + wz); M.m[1][1] = one - two * (xx + zz); M.m[1][2] = two * (yz - wx);
  M.m[2][0] = two * (xz - wy); M.m[2][1] = two * (yz + wx); M.m[2][2] = one - two * (xx + yy);
  return M;
}
template <class R> inline V3<R> mul(const M3<R>& M, const V3<R>& v) {
  return v3<R>(M.m[0][0] * v.x + M.m[0][1] * v.y + M.m[0][2] * v.z,
               M.m[1][0] * v.x + M.m[1][1] * v.y + M.m[1][2] * v.z,
               M.m[2][0] * v.x + M.m[2][1] * v.y + M.m[2][2] * v.z); }
template <class R> inline V3<R> mulT(const M3<R>& M, const V3<R>& v) {
  return v3<R>(M.m[0][0] * v.x + M.m[1][0] * v.y + M.m[2][0] * v.z,
               M.m[0][1] * v.x + M.m[1][1] * v.y + M.m[2][1] * v.z,
               M.m[0][2] * v.x + M.m[1][2] * v.y + M.m[2][2] * v.z); }
template <class R> inline V3<R> col(const M3<R>& M, int k) { return v3<R>(M.m[0][k], M.m[1][k], M.m[2][k]); }

template <class R> inline Q4<R> qmul(const Q4<R>& a, const Q4<R>& b) {
  Q4<R> r;
  r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
  r.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
  r.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
  r.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
  return r; }
template <class R> inline Q4<R> qconj(const Q4<R>& a) { Q4<R> r; r.w = a.w; r.x = -a.x; r.y = -a.y; r.z = -a.z; return r; }

// --------------------------------------------------------------------------
// Scene view (host arrays, same layout as the CUDA library's descriptor)
// --------------------------------------------------------------------------
enum { SPHERE = 0, CAPSULE = 1, BOX = 2, PLANE = 3 };
enum { REVOLUTE = 0, PRISMATIC = 1, PLANAR = 2 };
enum { ST_PAIR_OVERFLOW = 1, ST_CONTACT_OVERFLOW = 2, ST_COLOUR_OVERFLOW = 4, ST_NONFINITE = 8 };

}  // namespace orc

extern "C" {
struct OracleScene {
  int32_t num_envs;
  const int32_t* body_off;
  const int32_t* static_off;
  const int32_t* joint_off;
  int32_t max_dof;
  const int32_t* body_shape;
  const float* body_dims;     // [B,4]
  const float* body_mass;     // [B]
  const float* static_pose;   // [S,7]
  const float* static_half;   // [S,3]
  const int32_t* joint_type;
  const int32_t* joint_parent;
  const int32_t* joint_child;
  const int32_t* joint_dof;
  const float* joint_frame_a;  // [J,7]
  const float* joint_frame_b;  // [J,7]
  const float* joint_gains;    // [J,4]
  const float* joint_limits;   // [J,2]
};
struct OracleCfg {
  double dt;
  int32_t substeps, iterations, mode;
  double gravity[3];
  double friction, restitution, contact_offset, baumgarte, joint_baumgarte, slop;
  int32_t max_contacts, max_pairs;
};
}

namespace orc {

// --------------------------------------------------------------------------
// Per-env working data
// --------------------------------------------------------------------------
template <class R> struct Body {
  V3<R> x; Q4<R> q; V3<R> v, w;
  R mass, invm; V3<R> invI;   // principal inverse inertia (body frame)
  int shape; R dim[3];
};
template <class R> struct Stat { V3<R> x; Q4<R> q; V3<R> h; };
template <class R> struct Joint {
  int type, parent, child, dof;
  V3<R> pa; Q4<R> qa; V3<R> pb; Q4<R> qb;
  R k, d, fmax, lo, hi;
};
template <class R> struct Pt { V3<R> n, pa, pb; R s; };   // n: first -> second shape
template <class R> struct Contact { int a, b; V3<R> n, ra, rb; R s0; };  // b: collision index
struct Manifold { int a, b, first, count; };                  // b: collision index
template <class R> struct Shape { int type; V3<R> c; M3<R> M; R d0, d1, d2; };

// Solid-body inertia of the primitives about their centre, principal axes =
// local axes (sphere 2/5 m r^2; box m/3 (h1^2 + h2^2); capsule = cylinder of
// length 2L plus two hemispheres, axis = local x).
template <class R> V3<R> inv_inertia(int shape, R m, const R* d) {
  const R one = R(1);
  if (shape == SPHERE) {
    R I = R(0.4) * m * d[0] * d[0];
    return v3<R>(one / I, one / I, one / I);
  }
  if (shape == BOX) {
    R hx2 = d[0] * d[0], hy2 = d[1] * d[1], hz2 = d[2] * d[2];
    R k = m / R(3);
    return v3<R>(one / (k * (hy2 + hz2)), one / (k * (hx2 + hz2)), one / (k * (hx2 + hy2)));
  }
  // capsule: radius r = d[0], half segment length L = d[1]
  R r = d[0], L = d[1];
  R pi = R(3.14159265358979323846);
  R vc = pi * r * r * (R(2) * L);
  R vs = R(4) / R(3) * pi * r * r * r;
  R mc = m * vc / (vc + vs);
  R ms = m * vs / (vc + vs);
  R H = R(2) * L;
  R Ia = mc * r * r * R(0.5) + ms * R(0.4) * r * r;
  R Ip = mc * (H * H / R(12) + r * r * R(0.25)) + ms * (R(0.4) * r * r + H * H * R(0.25) + R(0.375) * H * r);
  return v3<R>(one / Ia, one / Ip, one / Ip);
}

// --------------------------------------------------------------------------
// a2: AABBs (exact box extents summed over columns, inflated by the offset)
// --------------------------------------------------------------------------
template <class R> struct AABB { V3<R> lo, hi; };

template <class R> AABB<R> shape_aabb(const Shape<R>& s, R off) {
  V3<R> e;
  if (s.type == SPHERE) {
    e = v3<R>(s.d0, s.d0, s.d0);
  } else if (s.type == CAPSULE) {
    V3<R> a = col(s.M, 0);
    e = v3<R>(abs_(a.x) * s.d1 + s.d0, abs_(a.y) * s.d1 + s.d0, abs_(a.z) * s.d1 + s.d0);
  } else {
    e.x = abs_(s.M.m[0][0]) * s.d0 + abs_(s.M.m[0][1]) * s.d1 + abs_(s.M.m[0][2]) * s.d2;
    e.y = abs_(s.M.m[1][0]) * s.d0 + abs_(s.M.m[1][1]) * s.d1 + abs_(s.M.m[1][2]) * s.d2;
    e.z = abs_(s.M.m[2][0]) * s.d0 + abs_(s.M.m[2][1]) * s.d1 + abs_(s.M.m[2][2]) * s.d2;
  }
  AABB<R> b;
  b.lo = v3<R>((s.c.x - e.x) - off, (s.c.y - e.y) - off, (s.c.z - e.z) - off);
  b.hi = v3<R>((s.c.x + e.x) + off, (s.c.y + e.y) + off, (s.c.z + e.z) + off);
  return b;
}
template <class R> inline bool overlap(const AABB<R>& a, const AABB<R>& b) {
  return a.lo.x <= b.hi.x && b.lo.x <= a.hi.x && a.lo.y <= b.hi.y && b.lo.y <= a.hi.y &&
         a.lo.z <= b.hi.z && b.lo.z <= a.hi.z;
}

// --------------------------------------------------------------------------
// a4: narrowphase. Each routine returns points with the normal pointing from
// its first shape to its second; pa lies on the first, pb on the second, and
// s = n . (pb - pa) is the signed separation.
// --------------------------------------------------------------------------
template <class R> int sphere_sphere(V3<R> c1, R r1, V3<R> c2, R r2, Pt<R>* out) {
  V3<R> d = c2 - c1;
  R dist = sqrt_(dot(d, d));
  V3<R> n;
  if (dist > R(1e-6)) n = v3<R>(d.x / dist, d.y / dist, d.z / dist);
  else n = v3<R>(R(0), R(0), R(1));
  out[0].n = n;
  out[0].s = (dist - r1) - r2;
  out[0].pa = c1 + n * r1;
  out[0].pb = c2 - n * r2;
  return 1;
}

template <class R> int sphere_plane(V3<R> c, R r, Pt<R>* out) {
  out[0].n = v3<R>(R(0), R(0), R(-1));
  out[0].s = c.z - r;
  out[0].pa = v3<R>(c.x, c.y, c.z - r);
  out[0].pb = v3<R>(c.x, c.y, R(0));
  return 1;
}

template <class R> int sphere_capsule(V3<R> c, R r, const Shape<R>& cap, Pt<R>* out) {
  V3<R> a = col(cap.M, 0);
  R t = clampv(dot(c - cap.c, a), -cap.d1, cap.d1);
  V3<R> q = cap.c + a * t;
  return sphere_sphere(c, r, q, cap.d0, out);
}

// Sphere (first) against box (second).
template <class R> int sphere_box(V3<R> c, R r, const Shape<R>& box, Pt<R>* out) {
  V3<R> l = mulT(box.M, c - box.c);
  R h[3] = {box.d0, box.d1, box.d2};
  bool inside = abs_(l.x) <= h[0] && abs_(l.y) <= h[1] && abs_(l.z) <= h[2];
  V3<R> nl, pl;
  R s;
  if (!inside) {
    V3<R> q = v3<R>(clampv(l.x, -h[0], h[0]), clampv(l.y, -h[1], h[1]), clampv(l.z, -h[2], h[2]));
    V3<R> df = l - q;
    R dist = sqrt_(dot(df, df));
    nl = v3<R>(df.x / dist, df.y / dist, df.z / dist);
    s = dist - r;
    pl = q;
  } else {
    R dx = h[0] - abs_(l.x), dy = h[1] - abs_(l.y), dz = h[2] - abs_(l.z);
    int k = 0;
    R best = dx;
    if (dy < best) { k = 1; best = dy; }
    if (dz < best) { k = 2; best = dz; }
    R lk = comp(l, k);
    R sg = lk >= R(0) ? R(1) : R(-1);
    nl = unit<R>(k) * sg;
    s = -best - r;
    pl = l;
    setc(pl, k, sg * h[k]);
  }
  V3<R> nw = mul(box.M, nl);    // box -> sphere
  out[0].n = -nw;
  out[0].s = s;
  out[0].pa = c + out[0].n * r;
  out[0].pb = box.c + mul(box.M, pl);
  return 1;
}

template <class R> int capsule_plane(const Shape<R>& cap, R off, Pt<R>* out) {
  V3<R> a = col(cap.M, 0);
  int n = 0;
  for (int e = 0; e < 2; ++e) {
    R t = e == 0 ? -cap.d1 : cap.d1;
    V3<R> p = cap.c + a * t;
    R s = p.z - cap.d0;
    if (s < off) {
      out[n].n = v3<R>(R(0), R(0), R(-1));
      out[n].s = s;
      out[n].pa = v3<R>(p.x, p.y, p.z - cap.d0);
      out[n].pb = v3<R>(p.x, p.y, R(0));
      ++n;
    }
  }
  return n;
}

template <class R> int capsule_capsule(const Shape<R>& c1, const Shape<R>& c2, Pt<R>* out) {
  V3<R> a1 = col(c1.M, 0), a2 = col(c2.M, 0);
  R L1 = c1.d1, L2 = c2.d1;
  V3<R> rr = c1.c - c2.c;
  R b = dot(a1, a2), cc = dot(a1, rr), f = dot(a2, rr);
  V3<R> cr = cross(a1, a2);
  if (dot(cr, cr) < R(1e-6)) {
    // nearly parallel: up to two points over the overlap of the projections
    R ta = -cc - b * L2, tb = -cc + b * L2;
    R lo = minv(ta, tb), hi = maxv(ta, tb);
    lo = maxv(lo, -L1);
    hi = minv(hi, L1);
    if (lo <= hi) {
      int n = 0;
      for (int e = 0; e < 2; ++e) {
        if (e == 1 && hi == lo) break;
        R t = e == 0 ? lo : hi;
        V3<R> p1 = c1.c + a1 * t;
        R u = clampv(dot(p1 - c2.c, a2), -L2, L2);
        V3<R> p2 = c2.c + a2 * u;
        n += sphere_sphere(p1, c1.d0, p2, c2.d0, out + n);
      }
      return n;
    }
  }
  R denom = R(1) - b * b;
  R s = denom > R(1e-6) ? clampv((b * f - cc) / denom, -L1, L1) : R(0);
  R t = b * s + f;
  if (t < -L2) { t = -L2; s = clampv(b * t - cc, -L1, L1); }
  else if (t > L2) { t = L2; s = clampv(b * t - cc, -L1, L1); }
  V3<R> p1 = c1.c + a1 * s, p2 = c2.c + a2 * t;
  return sphere_sphere(p1, c1.d0, p2, c2.d0, out);
}

// Squared distance from the local point p0 + d t to the box [-h, h].
template <class R> R seg_box_d2(const V3<R>& p0, const V3<R>& d, const R* h, R t) {
  R acc = R(0);
  for (int k = 0; k < 3; ++k) {
    R x = comp(p0, k) + comp(d, k) * t;
    R q = clampv(x, -h[k], h[k]);
    R e = x - q;
    acc = acc + e * e;
  }
  return acc;
}

// Capsule (first) against box (second): sphere-box tests at both segment
// endpoints and at the segment point closest to the box (exact minimiser of
// the piecewise-quadratic squared distance over the slab breakpoints).
template <class R> int capsule_box(const Shape<R>& cap, const Shape<R>& box, R off, Pt<R>* out) {
  V3<R> a = col(cap.M, 0);
  R L = cap.d1;
  R h[3] = {box.d0, box.d1, box.d2};
  V3<R> p0 = mulT(box.M, cap.c - box.c);
  V3<R> d = mulT(box.M, a);
  R brk[8];
  int nb = 0;
  brk[nb++] = -L;
  for (int k = 0; k < 3; ++k) {
    R dk = comp(d, k);
    if (abs_(dk) > R(1e-6)) {
      for (int e = 0; e < 2; ++e) {
        R bound = e == 0 ? -h[k] : h[k];
        R t = (bound - comp(p0, k)) / dk;
        if (t > -L && t < L) brk[nb++] = t;
      }
    }
  }
  brk[nb++] = L;
  for (int i = 1; i < nb; ++i) {   // insertion sort, ascending
    R key = brk[i];
    int j = i - 1;
    while (j >= 0 && brk[j] > key) { brk[j + 1] = brk[j]; --j; }
    brk[j + 1] = key;
  }
  R best_t = -L;
  R best_f = seg_box_d2(p0, d, h, best_t);
  for (int i = 0; i + 1 < nb; ++i) {
    R t0 = brk[i], t1 = brk[i + 1];
    if (!(t1 > t0)) continue;
    R tm = (t0 + t1) * R(0.5);
    R A = R(0), B = R(0);
    for (int k = 0; k < 3; ++k) {
      R x = comp(p0, k) + comp(d, k) * tm;
      R bound;
      if (x > h[k]) bound = h[k];
      else if (x < -h[k]) bound = -h[k];
      else continue;
      R e = comp(p0, k) - bound;
      A = A + comp(d, k) * comp(d, k);
      B = B + comp(d, k) * e;
    }
    R topt = A > R(0) ? clampv(-B / A, t0, t1) : t0;
    R fo = seg_box_d2(p0, d, h, topt);
    if (fo < best_f) { best_f = fo; best_t = topt; }
  }
  R cand[3];
  int nc = 0;
  cand[nc++] = -L;
  cand[nc++] = L;
  if ((best_t + L) > R(1e-3) && (L - best_t) > R(1e-3)) cand[nc++] = best_t;
  int n = 0;
  for (int i = 0; i < nc; ++i) {
    V3<R> q = cap.c + a * cand[i];
    Pt<R> p;
    sphere_box(q, cap.d0, box, &p);
    if (p.s < off) out[n++] = p;
  }
  return n;
}

template <class R> int box_plane(const Shape<R>& box, R off, Pt<R>* out) {
  V3<R> v[8];
  R s[8];
  for (int i = 0; i < 8; ++i) {
    V3<R> l = v3<R>((i & 1) ? box.d0 : -box.d0, (i & 2) ? box.d1 : -box.d1, (i & 4) ? box.d2 : -box.d2);
    v[i] = box.c + mul(box.M, l);
    s[i] = v[i].z;
  }
  bool used[8] = {false, false, false, false, false, false, false, false};
  int n = 0;
  while (n < 4) {
    int k = -1;
    for (int i = 0; i < 8; ++i) {
      if (used[i] || !(s[i] < off)) continue;
      if (k < 0 || s[i] < s[k]) k = i;
    }
    if (k < 0) break;
    used[k] = true;
    out[n].n = v3<R>(R(0), R(0), R(-1));
    out[n].s = s[k];
    out[n].pa = v[k];
    out[n].pb = v3<R>(v[k].x, v[k].y, R(0));
    ++n;
  }
  return n;
}

// One Sutherland-Hodgman pass over a polygon in reference-face coordinates
// (x, y, height), keeping the side where sg * coord - bound <= 0. The output
// is capped at 8 vertices (a convex quad never exceeds it; rounding on a
// nearly degenerate polygon could).
// Number of clip outputs dropped by the 8-vertex cap (tests read it).
inline long long& clip_cap_drops() { static long long n = 0; return n; }

template <class R> int clip_poly(const R (*in)[3], int n, R (*out)[3], int axis, R sg, R bound) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const R* P = in[i];
    const R* Q = in[(i + 1) % n];
    R dp = sg * P[axis] - bound;
    R dq = sg * Q[axis] - bound;
    if (dp <= R(0)) {
      if (m < 8) { out[m][0] = P[0]; out[m][1] = P[1]; out[m][2] = P[2]; ++m; }
      else {
#pragma omp atomic
        ++clip_cap_drops();
      }
    }
    if ((dp < R(0) && dq > R(0)) || (dp > R(0) && dq < R(0))) {
      if (m < 8) {
        R t = dp / (dp - dq);
        for (int k = 0; k < 3; ++k) out[m][k] = P[k] + (Q[k] - P[k]) * t;
        ++m;
      } else {
#pragma omp atomic
        ++clip_cap_drops();
      }
    }
  }
  return m;
}

// Box (first) against box (second): separating-axis test over the 6 face
// normals and 9 edge-edge cross products; face contacts by clipping the
// incident face against the reference face's side planes and reducing to at
// most 4 points; edge contacts at the closest points of the two edges.
template <class R> int box_box(const Shape<R>& A, const Shape<R>& B, R off, Pt<R>* out) {
  V3<R> d = B.c - A.c;
  V3<R> axA[3] = {col(A.M, 0), col(A.M, 1), col(A.M, 2)};
  V3<R> axB[3] = {col(B.M, 0), col(B.M, 1), col(B.M, 2)};
  R hA[3] = {A.d0, A.d1, A.d2}, hB[3] = {B.d0, B.d1, B.d2};
  R C[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = abs_(dot(axA[i], axB[j]));
  R dA[3], dB[3];
  for (int i = 0; i < 3; ++i) { dA[i] = dot(d, axA[i]); dB[i] = dot(d, axB[i]); }
  R best_face_sep = R(0);
  int best_face = -1;
  for (int i = 0; i < 3; ++i) {
    R pB = hB[0] * C[i][0] + hB[1] * C[i][1] + hB[2] * C[i][2];
    R sep = abs_(dA[i]) - (hA[i] + pB);
    if (sep > off) return 0;
    if (best_face < 0 || sep > best_face_sep) { best_face_sep = sep; best_face = i; }
  }
  for (int j = 0; j < 3; ++j) {
    R pA = hA[0] * C[0][j] + hA[1] * C[1][j] + hA[2] * C[2][j];
    R sep = abs_(dB[j]) - (pA + hB[j]);
    if (sep > off) return 0;
    if (sep > best_face_sep) { best_face_sep = sep; best_face = 3 + j; }
  }
  R best_edge_sep = R(0);
  int best_edge = -1;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      V3<R> Lx = cross(axA[i], axB[j]);
      R len = sqrt_(dot(Lx, Lx));
      if (len < R(1e-5)) continue;
      V3<R> L = v3<R>(Lx.x / len, Lx.y / len, Lx.z / len);
      R pA = hA[0] * abs_(dot(L, axA[0])) + hA[1] * abs_(dot(L, axA[1])) + hA[2] * abs_(dot(L, axA[2]));
      R pB = hB[0] * abs_(dot(L, axB[0])) + hB[1] * abs_(dot(L, axB[1])) + hB[2] * abs_(dot(L, axB[2]));
      R sep = abs_(dot(d, L)) - (pA + pB);
      if (sep > off) return 0;
      if (best_edge < 0 || sep > best_edge_sep) { best_edge_sep = sep; best_edge = 3 * i + j; }
    }
  }
  bool use_edge = best_edge >= 0 &&
                  best_edge_sep > best_face_sep + R(1e-4) * (R(1) + abs_(best_face_sep));
  if (use_edge) {
    int i = best_edge / 3, j = best_edge % 3;
    V3<R> Lx = cross(axA[i], axB[j]);
    R len = sqrt_(dot(Lx, Lx));
    V3<R> L = v3<R>(Lx.x / len, Lx.y / len, Lx.z / len);
    V3<R> n = dot(d, L) >= R(0) ? L : -L;
    V3<R> pa = A.c;
    for (int m = 0; m < 3; ++m) {
      if (m == i) continue;
      R sg = dot(n, axA[m]) > R(0) ? R(1) : R(-1);
      pa = pa + axA[m] * (hA[m] * sg);
    }
    V3<R> pb = B.c;
    for (int m = 0; m < 3; ++m) {
      if (m == j) continue;
      R sg = dot(n, axB[m]) > R(0) ? R(-1) : R(1);
      pb = pb + axB[m] * (hB[m] * sg);
    }
    V3<R> rr = pa - pb;
    R b = dot(axA[i], axB[j]), cc = dot(axA[i], rr), f = dot(axB[j], rr);
    R denom = R(1) - b * b;
    R s = denom > R(1e-6) ? (b * f - cc) / denom : R(0);
    s = clampv(s, -hA[i], hA[i]);
    R t = clampv(b * s + f, -hB[j], hB[j]);
    V3<R> qa = pa + axA[i] * s, qb = pb + axB[j] * t;
    R sep = dot(n, qb - qa);
    if (!(sep < off)) return 0;
    out[0].n = n; out[0].pa = qa; out[0].pb = qb; out[0].s = sep;
    return 1;
  }
  // face contact
  bool refA = best_face < 3;
  int k = refA ? best_face : best_face - 3;
  const V3<R>* axR = refA ? axA : axB;
  const V3<R>* axI = refA ? axB : axA;
  const R* hR = refA ? hA : hB;
  const R* hI = refA ? hB : hA;
  V3<R> cR = refA ? A.c : B.c, cI = refA ? B.c : A.c;
  R dist = refA ? dA[k] : dB[k];
  R sgn = refA ? (dist >= R(0) ? R(1) : R(-1)) : (dist >= R(0) ? R(-1) : R(1));
  V3<R> nR = axR[k] * sgn;
  V3<R> fc = cR + nR * hR[k];
  int ku = (k + 1) % 3, kv = (k + 2) % 3;
  V3<R> u = axR[ku], v = axR[kv];
  R hu = hR[ku], hv = hR[kv];
  int m = 0;
  R bestd = abs_(dot(nR, axI[0]));
  R dm = dot(nR, axI[0]);
  for (int q = 1; q < 3; ++q) {
    R dq = dot(nR, axI[q]);
    if (abs_(dq) > bestd) { bestd = abs_(dq); m = q; dm = dq; }
  }
  R sgI = dm > R(0) ? R(-1) : R(1);
  V3<R> ic = cI + axI[m] * (hI[m] * sgI);
  int m1 = (m + 1) % 3, m2 = (m + 2) % 3;
  V3<R> e1 = axI[m1] * hI[m1], e2 = axI[m2] * hI[m2];
  V3<R> vert[4] = {(ic + e1) + e2, (ic - e1) + e2, (ic - e1) - e2, (ic + e1) - e2};
  R P0[8][3], P1[8][3];
  for (int i = 0; i < 4; ++i) {
    V3<R> rel = vert[i] - fc;
    P0[i][0] = dot(rel, u); P0[i][1] = dot(rel, v); P0[i][2] = dot(rel, nR);
  }
  int np = 4;
  np = clip_poly<R>(P0, np, P1, 0, R(1), hu);
  np = clip_poly<R>(P1, np, P0, 0, R(-1), hu);
  np = clip_poly<R>(P0, np, P1, 1, R(1), hv);
  np = clip_poly<R>(P1, np, P0, 1, R(-1), hv);
  int keep[8];
  int nk = 0;
  for (int i = 0; i < np; ++i) if (P0[i][2] < off) keep[nk++] = i;
  int sel[4];
  int ns = 0;
  if (nk <= 4) {
    for (int i = 0; i < nk; ++i) sel[ns++] = keep[i];
  } else {
    // deepest, farthest from it, largest triangle, largest area on the other side
    int i0 = keep[0];
    for (int i = 1; i < nk; ++i) if (P0[keep[i]][2] < P0[i0][2]) i0 = keep[i];
    int i1 = -1; R bd = R(0);
    for (int i = 0; i < nk; ++i) {
      int c = keep[i]; if (c == i0) continue;
      R dx = P0[c][0] - P0[i0][0], dy = P0[c][1] - P0[i0][1];
      R dd = dx * dx + dy * dy;
      if (i1 < 0 || dd > bd) { bd = dd; i1 = c; }
    }
    R ex = P0[i1][0] - P0[i0][0], ey = P0[i1][1] - P0[i0][1];
    int i2 = -1; R ba = R(0), a2 = R(0);
    for (int i = 0; i < nk; ++i) {
      int c = keep[i]; if (c == i0 || c == i1) continue;
      R ar = ex * (P0[c][1] - P0[i0][1]) - ey * (P0[c][0] - P0[i0][0]);
      if (i2 < 0 || abs_(ar) > ba) { ba = abs_(ar); i2 = c; a2 = ar; }
    }
    R flip = a2 >= R(0) ? R(-1) : R(1);
    int i3 = -1; R bv = R(0);
    for (int i = 0; i < nk; ++i) {
      int c = keep[i]; if (c == i0 || c == i1 || c == i2) continue;
      R ar = (ex * (P0[c][1] - P0[i0][1]) - ey * (P0[c][0] - P0[i0][0])) * flip;
      if (i3 < 0 || ar > bv) { bv = ar; i3 = c; }
    }
    sel[0] = i0; sel[1] = i1; sel[2] = i2; sel[3] = i3; ns = 4;
  }
  for (int i = 0; i < ns; ++i) {
    const R* P = P0[sel[i]];
    V3<R> pR = (fc + u * P[0]) + v * P[1];
    V3<R> pI = pR + nR * P[2];
    if (refA) { out[i].n = nR; out[i].pa = pR; out[i].pb = pI; }
    else { out[i].n = -nR; out[i].pa = pI; out[i].pb = pR; }
    out[i].s = P[2];
  }
  return ns;
}

// Dispatch on the shape types of (first = dynamic body, second = body, static
// box or plane). The routines take the lower shape type first; the points are
// flipped back when the pair order is the reverse.
template <class R> int collide(const Shape<R>& S1, const Shape<R>& S2, R off, Pt<R>* out) {
  int n = 0;
  if (S2.type == PLANE) {
    if (S1.type == SPHERE) n = sphere_plane(S1.c, S1.d0, out);
    else if (S1.type == CAPSULE) n = capsule_plane(S1, off, out);
    else n = box_plane(S1, off, out);
  } else {
    bool swap = S1.type > S2.type;
    const Shape<R>& P = swap ? S2 : S1;
    const Shape<R>& Q = swap ? S1 : S2;
    if (P.type == SPHERE) {
      if (Q.type == SPHERE) n = sphere_sphere(P.c, P.d0, Q.c, Q.d0, out);
      else if (Q.type == CAPSULE) n = sphere_capsule(P.c, P.d0, Q, out);
      else n = sphere_box(P.c, P.d0, Q, out);
    } else if (P.type == CAPSULE) {
      if (Q.type == CAPSULE) n = capsule_capsule(P, Q, out);
      else n = capsule_box(P, Q, off, out);
    } else {
      n = box_box(P, Q, off, out);
    }
    if (swap) {
      for (int i = 0; i < n; ++i) {
        out[i].n = -out[i].n;
        V3<R> t = out[i].pa; out[i].pa = out[i].pb; out[i].pb = t;
      }
    }
  }
  int m = 0;
  for (int i = 0; i < n; ++i) if (out[i].s < off) out[m++] = out[i];
  return m;
}

// --------------------------------------------------------------------------
// Rows (sequential impulses)
// --------------------------------------------------------------------------
enum { ROW_BILATERAL = 0, ROW_UNILATERAL = 1, ROW_FRICTION = 2, ROW_SOFT = 3 };

template <class R> struct Row {
  int a, b;              // dynamic body indices, -1 = static/world
  V3<R> la, aa, lb, ab;  // Jacobian blocks
  V3<R> Ia, Ib;          // world inverse inertia times the angular blocks
  R m, bias, gamma, lam, lo, hi, mu;
  int kind, ref;         // ref: normal row of a friction row
};
struct Con { int a, b, first, count; };   // rows [first, first+count), dynamic bodies a,b (-1 none)

// Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin (2017),
// "Building an Orthonormal Basis, Revisited": branchless frame from a unit n.
template <class R> void onb(const V3<R>& n, V3<R>& t1, V3<R>& t2) {
  R sg = n.z >= R(0) ? R(1) : R(-1);
  R a = R(-1) / (sg + n.z);
  R b = n.x * n.y * a;
  t1 = v3<R>(R(1) + sg * n.x * n.x * a, sg * b, -sg * n.x);
  t2 = v3<R>(b, sg + n.y * n.y * a, -n.y);
}

template <class R> struct EnvState {
  int D, S, J;
  std::vector<Body<R>> body;
  std::vector<Stat<R>> stat;
  std::vector<Joint<R>> joint;
};

template <class R> M3<R> world_invI(const Body<R>& b) {
  M3<R> Rm = qmat(b.q);
  M3<R> W;
  R dI[3] = {b.invI.x, b.invI.y, b.invI.z};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      W.m[i][j] = Rm.m[i][0] * dI[0] * Rm.m[j][0] + Rm.m[i][1] * dI[1] * Rm.m[j][1] + Rm.m[i][2] * dI[2] * Rm.m[j][2];
  return W;
}

template <class R> struct Solver {
  const OracleCfg* cfg;
  R h;
  int sub = 0;               // substep of the rows being built
  std::vector<M3<R>> Iw;     // world inverse inertia per dynamic body
  std::vector<R> split;      // Jacobi mass-splitting counts (1 in PGS)
  std::vector<Row<R>> rows;
  std::vector<Con> cons;

  void finish_row(Row<R>& r, const EnvState<R>& E) {
    R K = R(0);
    if (r.a >= 0) {
      const Body<R>& A = E.body[r.a];
      r.Ia = mul(Iw[r.a], r.aa);
      K = K + split[r.a] * (A.invm * dot(r.la, r.la) + dot(r.aa, r.Ia));
    }
    if (r.b >= 0) {
      const Body<R>& B = E.body[r.b];
      r.Ib = mul(Iw[r.b], r.ab);
      K = K + split[r.b] * (B.invm * dot(r.lb, r.lb) + dot(r.ab, r.Ib));
    }
    if (r.kind == ROW_SOFT) r.m = R(1) / (K + r.gamma);
    else r.m = K > R(0) ? R(1) / K : R(0);
    r.lam = R(0);
  }

  Row<R> blank(int a, int b, int kind) {
    Row<R> r;
    V3<R> z = v3<R>(R(0), R(0), R(0));
    r.a = a; r.b = b; r.la = z; r.aa = z; r.lb = z; r.ab = z; r.Ia = z; r.Ib = z;
    r.m = R(0); r.bias = R(0); r.gamma = R(0); r.lam = R(0); r.lo = R(0); r.hi = R(0); r.mu = R(0);
    r.kind = kind; r.ref = -1;
    return r;
  }

  // Row along a linear direction u between anchor points; ra, rb are the lever
  // arms from the body centres (ignored for a static side).
  Row<R> lin_row(int a, int b, const V3<R>& u, const V3<R>& ra, const V3<R>& rb, int kind) {
    Row<R> r = blank(a, b, kind);
    r.la = -u; r.aa = -cross(ra, u); r.lb = u; r.ab = cross(rb, u);
    return r;
  }
  Row<R> ang_row(int a, int b, const V3<R>& u, int kind) {
    Row<R> r = blank(a, b, kind);
    r.aa = -u; r.ab = u;
    return r;
  }
  void soft(Row<R>& r, R C, R k, R d, R fmax) {
    // Catto (2011) soft constraint: gamma = 1/(h(d + h k)), beta = h k/(d + h k)
    R den = d + h * k;
    r.gamma = R(1) / (h * den);
    r.bias = (h * k / den) / h * C;
    r.lo = -fmax * h;
    r.hi = fmax * h;
  }

  void add_con(int a, int b, int first) {
    Con c; c.a = a; c.b = b; c.first = first; c.count = (int)rows.size() - first;
    cons.push_back(c);
  }

  void joint_rows(const Joint<R>& j, const EnvState<R>& E, const R* tgt) {
    R beta = R(cfg->joint_baumgarte) / h;
    int A = j.parent, B = j.child;
    V3<R> xa, ra, pa_w;
    Q4<R> qFA;
    if (A >= 0) {
      const Body<R>& bA = E.body[A];
      xa = bA.x;
      ra = mul(qmat(bA.q), j.pa);
      pa_w = xa + ra;
      qFA = qmul(bA.q, j.qa);
    } else {
      xa = j.pa; ra = v3<R>(R(0), R(0), R(0)); pa_w = j.pa; qFA = j.qa;
    }
    const Body<R>& bB = E.body[B];
    V3<R> rb = mul(qmat(bB.q), j.pb);
    V3<R> pb_w = bB.x + rb;
    Q4<R> qFB = qmul(bB.q, j.qb);
    M3<R> MF = qmat(qFA);
    V3<R> ux = col(MF, 0), uy = col(MF, 1), uz = col(MF, 2);
    V3<R> dp = pb_w - pa_w;
    Q4<R> qr = qmul(qconj(qFA), qFB);
    if (qr.w < R(0)) { qr.w = -qr.w; qr.x = -qr.x; qr.y = -qr.y; qr.z = -qr.z; }
    V3<R> raB = A >= 0 ? pb_w - xa : v3<R>(R(0), R(0), R(0));   // lever to the moving point
    int first = (int)rows.size();
    if (j.type == REVOLUTE) {
      for (int k = 0; k < 3; ++k) {
        Row<R> r = lin_row(A, B, unit<R>(k), ra, rb, ROW_BILATERAL);
        r.bias = beta * comp(dp, k);
        rows.push_back(r);
      }
      V3<R> aB = col(qmat(qFB), 0);
      V3<R> cr = cross(ux, aB);
      V3<R> us[2] = {uy, uz};
      for (int k = 0; k < 2; ++k) {
        Row<R> r = ang_row(A, B, us[k], ROW_BILATERAL);
        r.bias = beta * dot(cr, us[k]);
        rows.push_back(r);
      }
      if (j.k > R(0) || j.d > R(0)) {
        Row<R> r = ang_row(A, B, ux, ROW_SOFT);
        R theta = R(2) * atan2_(qr.x, qr.w);
        soft(r, theta - tgt[j.dof], j.k, j.d, j.fmax);
        rows.push_back(r);
      }
      if (j.lo < j.hi) {   // hinge angle limits lo <= theta <= hi, speculative unilateral rows
        R theta = R(2) * atan2_(qr.x, qr.w);
        for (int e = 0; e < 2; ++e) {
          Row<R> r = ang_row(A, B, e == 0 ? ux : -ux, ROW_UNILATERAL);
          R C = e == 0 ? theta - j.lo : j.hi - theta;
          bool open = C > R(0);
          if (decision(std::fabs(val(C)), dec_tol())) open = !open;
          r.bias = open ? C / h : beta * C;
          rows.push_back(r);
        }
      }
    } else if (j.type == PRISMATIC) {
      V3<R> us[2] = {uy, uz};
      for (int k = 0; k < 2; ++k) {
        Row<R> r = lin_row(A, B, us[k], raB, rb, ROW_BILATERAL);
        r.bias = beta * dot(dp, us[k]);
        rows.push_back(r);
      }
      V3<R> ua[3] = {ux, uy, uz};
      R qv[3] = {qr.x, qr.y, qr.z};
      for (int k = 0; k < 3; ++k) {
        Row<R> r = ang_row(A, B, ua[k], ROW_BILATERAL);
        r.bias = beta * (R(2) * qv[k]);
        rows.push_back(r);
      }
      R dd = dot(dp, ux);
      if (j.k > R(0) || j.d > R(0)) {
        Row<R> r = lin_row(A, B, ux, raB, rb, ROW_SOFT);
        soft(r, dd - tgt[j.dof], j.k, j.d, j.fmax);
        rows.push_back(r);
      }
      for (int e = 0; e < 2; ++e) {
        Row<R> r = lin_row(A, B, e == 0 ? ux : -ux, raB, rb, ROW_UNILATERAL);
        R C = e == 0 ? dd - j.lo : j.hi - dd;
        bool open = C > R(0);
        if (decision(std::fabs(val(C)), dec_tol())) open = !open;
        r.bias = open ? C / h : beta * C;
        rows.push_back(r);
      }
    } else {  // PLANAR: normal = frame z; free x, y, yaw
      {
        Row<R> r = lin_row(A, B, uz, raB, rb, ROW_BILATERAL);
        r.bias = beta * dot(dp, uz);
        rows.push_back(r);
      }
      V3<R> aB = col(qmat(qFB), 2);
      V3<R> cr = cross(uz, aB);
      V3<R> us[2] = {ux, uy};
      for (int k = 0; k < 2; ++k) {
        Row<R> r = ang_row(A, B, us[k], ROW_BILATERAL);
        r.bias = beta * dot(cr, us[k]);
        rows.push_back(r);
      }
      if (j.k > R(0) || j.d > R(0)) {
        for (int k = 0; k < 2; ++k) {
          Row<R> r = lin_row(A, B, us[k], raB, rb, ROW_SOFT);
          soft(r, dot(dp, us[k]) - tgt[j.dof + k], j.k, j.d, j.fmax);
          rows.push_back(r);
        }
        Row<R> r = ang_row(A, B, uz, ROW_SOFT);
        R theta = R(2) * atan2_(qr.z, qr.w);
        soft(r, theta - tgt[j.dof + 2], j.k, j.d, j.fmax);
        rows.push_back(r);
      }
    }
    for (int i = first; i < (int)rows.size(); ++i) finish_row(rows[i], E);
    add_con(A, B, first);
  }

  void contact_rows(const Manifold& mf, const std::vector<Contact<R>>& ct, const EnvState<R>& E) {
    const Body<R>& bA = E.body[mf.a];
    int bdyn = mf.b < E.D ? mf.b : -1;
    M3<R> MA = qmat(bA.q);
    M3<R> MB;
    if (bdyn >= 0) MB = qmat(E.body[bdyn].q);
    R mu = R(cfg->friction);
    R beta = R(cfg->baumgarte);
    R slop = R(cfg->slop);
    R rest = R(cfg->restitution);
    int first = (int)rows.size();
    for (int p = mf.first; p < mf.first + mf.count; ++p) {
      const Contact<R>& c = ct[p];
      V3<R> ra = mul(MA, c.ra);
      V3<R> pa_w = bA.x + ra;
      V3<R> rb, pb_w;
      if (bdyn >= 0) { rb = mul(MB, c.rb); pb_w = E.body[bdyn].x + rb; }
      else { pb_w = c.rb; rb = v3<R>(R(0), R(0), R(0)); }
      R s = dot(c.n, pb_w - pa_w);
      Row<R> rn = lin_row(mf.a, bdyn, c.n, ra, rb, ROW_UNILATERAL);
      // speculative above s = 0, nothing down to -slop, Baumgarte below; from
      // the second substep on the poses carry the solver's rounding, so a
      // separation within noise of a kink is a fragile decision there
      bool spec = s > R(0);
      if (sub > 0 && decision(std::fabs(val(s)), dec_tol())) spec = !spec;
      if (spec) {
        rn.bias = s / h;
      } else {
        // (at pen == 0 exactly the bias is 0 either way; the Baumgarte case is
        // taken only for pen > 0, so a contact resting exactly at -slop has no
        // bias derivative)
        const R pen = -s - slop;
        bool deep = pen > R(0);
        if (sub > 0 && decision(std::fabs(val(pen)), dec_tol())) deep = !deep;
        rn.bias = -(beta / h) * (deep ? pen : R(0));
      }
      finish_row(rn, E);
      if (rest > R(0)) {
        R vn = jv(rn, E);
        if (vn < R(-1)) rn.bias = minv(rn.bias, rest * vn);
      }
      int nrow = (int)rows.size();
      rows.push_back(rn);
      V3<R> t1, t2;
      onb(c.n, t1, t2);
      V3<R> ts[2] = {t1, t2};
      for (int k = 0; k < 2; ++k) {
        Row<R> rt = lin_row(mf.a, bdyn, ts[k], ra, rb, ROW_FRICTION);
        rt.mu = mu;
        rt.ref = nrow;
        finish_row(rt, E);
        rows.push_back(rt);
      }
    }
    add_con(mf.a, bdyn, first);
  }

  R jv(const Row<R>& r, const EnvState<R>& E) const {
    R acc = R(0);
    if (r.a >= 0) acc = acc + dot(r.la, E.body[r.a].v) + dot(r.aa, E.body[r.a].w);
    if (r.b >= 0) acc = acc + dot(r.lb, E.body[r.b].v) + dot(r.ab, E.body[r.b].w);
    return acc;
  }

  // Sequential-impulse update of one row on velocities (va, wa, vb, wb); the
  // velocity change uses the (possibly split) inverse masses; the true-mass
  // change is accumulated into (dva, dwa, dvb, dwb) when given.
  void solve_row(Row<R>& r, const EnvState<R>& E, V3<R>* va, V3<R>* wa, V3<R>* vb, V3<R>* wb,
                 V3<R>* dva, V3<R>* dwa, V3<R>* dvb, V3<R>* dwb) {
    R acc = R(0);
    if (r.a >= 0) acc = acc + dot(r.la, *va) + dot(r.aa, *wa);
    if (r.b >= 0) acc = acc + dot(r.lb, *vb) + dot(r.ab, *wb);
    R dl = -r.m * (acc + r.bias + r.gamma * r.lam);
    R nl = r.lam + dl;
    if (dec_log() && r.kind != ROW_BILATERAL) {
      // the same clamps, with the decision logged (and possibly inverted)
      R lo, hi, lim = R(0);
      const bool has_hi = r.kind != ROW_UNILATERAL;
      if (r.kind == ROW_UNILATERAL) { lo = R(0); hi = R(0); }
      else if (r.kind == ROW_FRICTION) { lim = r.mu * rows[r.ref].lam; lo = -lim; hi = lim; }
      else { lo = r.lo; hi = r.hi; }
      int choice = r.kind == ROW_UNILATERAL ? (nl > R(0) ? 0 : -1) : (nl <= lo ? -1 : (nl >= hi ? 1 : 0));
      // magnitude of what enters the update: the noise scale of nl
      double a = 0.0;
      if (r.a >= 0) a += std::fabs(val(r.la.x) * val(va->x)) + std::fabs(val(r.la.y) * val(va->y)) +
                         std::fabs(val(r.la.z) * val(va->z)) + std::fabs(val(r.aa.x) * val(wa->x)) +
                         std::fabs(val(r.aa.y) * val(wa->y)) + std::fabs(val(r.aa.z) * val(wa->z));
      if (r.b >= 0) a += std::fabs(val(r.lb.x) * val(vb->x)) + std::fabs(val(r.lb.y) * val(vb->y)) +
                         std::fabs(val(r.lb.z) * val(vb->z)) + std::fabs(val(r.ab.x) * val(wb->x)) +
                         std::fabs(val(r.ab.y) * val(wb->y)) + std::fabs(val(r.ab.z) * val(wb->z));
      const double scale = std::fabs(val(r.lam)) + std::fabs(val(r.m)) * (a + std::fabs(val(r.bias)) +
                           std::fabs(val(r.gamma) * val(r.lam))) + std::fabs(val(lim)) + 1e-300;
      const double dlo = std::fabs(val(nl) - val(lo));
      const double dhi = has_hi ? std::fabs(val(nl) - val(hi)) : INFINITY;
      // a zero-width interval (friction with lambda_n = 0) leaves one choice:
      // its decision is never fragile
      const double margin = has_hi && val(lo) == val(hi) ? INFINITY : std::min(dlo, dhi) / scale;
      dec_log()->site = (int)(&r - rows.data());
      dec_log()->choice = choice != 0;
      if (decision(margin, dec_log()->delta))
        choice = choice != 0 ? 0 : (dlo <= dhi ? -1 : 1);
      nl = choice == 0 ? nl : (choice < 0 ? lo : hi);
    } else if (r.kind == ROW_UNILATERAL) nl = maxv(nl, R(0));
    else if (r.kind == ROW_FRICTION) { R lim = r.mu * rows[r.ref].lam; nl = clamp_active(nl, -lim, lim); }
    else if (r.kind == ROW_SOFT) nl = clamp_active(nl, r.lo, r.hi);
    dl = nl - r.lam;
    r.lam = nl;
    if (r.a >= 0) {
      R im = E.body[r.a].invm, sp = split[r.a];
      *va = *va + r.la * (sp * im * dl);
      *wa = *wa + r.Ia * (sp * dl);
      if (dva) { *dva = *dva + r.la * (im * dl); *dwa = *dwa + r.Ia * dl; }
    }
    if (r.b >= 0) {
      R im = E.body[r.b].invm, sp = split[r.b];
      *vb = *vb + r.lb * (sp * im * dl);
      *wb = *wb + r.Ib * (sp * dl);
      if (dvb) { *dvb = *dvb + r.lb * (im * dl); *dwb = *dwb + r.Ib * dl; }
    }
  }
};

template <class R> struct Detect {
  std::vector<AABB<R>> aabb;          // D + S
  std::vector<std::pair<int, int>> pairs;
  std::vector<Contact<R>> contacts;
  std::vector<Manifold> manifolds;
  std::vector<int> colour;            // per constraint: joints then manifolds
  int ncolours = 0;
  int status = 0;
};

template <class R> Shape<R> body_shape(const EnvState<R>& E, int i) {
  Shape<R> s;
  if (i < E.D) {
    const Body<R>& b = E.body[i];
    s.type = b.shape; s.c = b.x; s.M = qmat(b.q); s.d0 = b.dim[0]; s.d1 = b.dim[1]; s.d2 = b.dim[2];
  } else if (i < E.D + E.S) {
    const Stat<R>& b = E.stat[i - E.D];
    s.type = BOX; s.c = b.x; s.M = qmat(b.q); s.d0 = b.h.x; s.d1 = b.h.y; s.d2 = b.h.z;
  } else {
    s.type = PLANE; s.c = v3<R>(R(0), R(0), R(0)); s.d0 = s.d1 = s.d2 = R(0);
  }
  return s;
}

// a2-a4 and the colouring, from the poses at the start of the step.
template <class R> void detect(const EnvState<R>& E, const OracleCfg& cfg, Detect<R>& out) {
  R off = R(cfg.contact_offset);
  int D = E.D, S = E.S;
  out.aabb.resize(D + S);
  for (int i = 0; i < D + S; ++i) out.aabb[i] = shape_aabb(body_shape(E, i), off);
  // a3: pairs (i < j), skipping static-static and jointed pairs
  for (int i = 0; i < D; ++i) {
    for (int j = i + 1; j <= D + S; ++j) {
      bool hit;
      if (j == D + S) hit = out.aabb[i].lo.z <= R(0);
      else hit = overlap(out.aabb[i], out.aabb[j]);
      if (!hit) continue;
      if (j < D) {
        bool jointed = false;
        for (int k = 0; k < E.J; ++k) {
          int p = E.joint[k].parent, c = E.joint[k].child;
          if ((p == i && c == j) || (p == j && c == i)) jointed = true;
        }
        if (jointed) continue;
      }
      if ((int)out.pairs.size() < cfg.max_pairs) out.pairs.push_back(std::make_pair(i, j));
      else out.status |= ST_PAIR_OVERFLOW;
    }
  }
  // a4: manifolds in pair order, points in routine order
  for (size_t p = 0; p < out.pairs.size(); ++p) {
    int i = out.pairs[p].first, j = out.pairs[p].second;
    Shape<R> Si = body_shape(E, i), Sj = body_shape(E, j);
    Pt<R> pts[8];
    int n = collide(Si, Sj, off, pts);
    int first = (int)out.contacts.size();
    for (int k = 0; k < n; ++k) {
      if ((int)out.contacts.size() >= cfg.max_contacts) { out.status |= ST_CONTACT_OVERFLOW; break; }
      Contact<R> c;
      c.a = i; c.b = j; c.n = pts[k].n; c.s0 = pts[k].s;
      c.ra = mulT(Si.M, pts[k].pa - Si.c);
      if (j < D) c.rb = mulT(Sj.M, pts[k].pb - Sj.c);
      else c.rb = pts[k].pb;
      out.contacts.push_back(c);
    }
    int cnt = (int)out.contacts.size() - first;
    if (cnt > 0) { Manifold m; m.a = i; m.b = j; m.first = first; m.count = cnt; out.manifolds.push_back(m); }
  }
  // greedy colouring: joints first, then manifolds; static sides never conflict
  std::vector<uint64_t> used(D, 0ull);
  int nc = 0;
  auto colour_of = [&](int a, int b) {
    uint64_t m = 0;
    if (a >= 0) m |= used[a];
    if (b >= 0) m |= used[b];
    if (m == ~0ull) return -1;
    int c = 0;
    while (m & (1ull << c)) ++c;
    if (a >= 0) used[a] |= 1ull << c;
    if (b >= 0) used[b] |= 1ull << c;
    return c;
  };
  for (int k = 0; k < E.J; ++k) {
    int c = colour_of(E.joint[k].parent, E.joint[k].child);
    if (c < 0) out.status |= ST_COLOUR_OVERFLOW;
    out.colour.push_back(c);
    if (c + 1 > nc) nc = c + 1;
  }
  for (size_t k = 0; k < out.manifolds.size(); ++k) {
    int b = out.manifolds[k].b < D ? out.manifolds[k].b : -1;
    int c = colour_of(out.manifolds[k].a, b);
    if (c < 0) out.status |= ST_COLOUR_OVERFLOW;
    out.colour.push_back(c);
    if (c + 1 > nc) nc = c + 1;
  }
  out.ncolours = nc;
}

// Contact report of one env for one step. The paper's event labels and
// success conditions (Sec. 3.3, Appendix A.4-A.5) consume pairwise contact
// forces F_{a,b,t} in N, the robot's cumulative collision force and a grasp
// indicator "computed by the simulator"; it does not say how. Readings:
//   * the force of contact c on its second body is its accumulated impulse
//     over the step's substeps, sum_s (l_n n + l_t1 t1 + l_t2 t2), divided by
//     the step's dt (the mean force over the step); the first body receives
//     the opposite force;
//   * the robot collision force of a step is the sum over robot links of the
//     norm of each link's net force from contacts with static boxes and with
//     dynamic bodies that are neither robot links nor the target (self
//     contacts, the ground plane and the target itself do not count); the
//     cumulative force adds it up step by step;
//   * grasped(x): both fingers touch x with a force of at least f_min whose
//     angle to the finger's opening direction (from the other finger towards
//     it) is at most theta_max, tested as F.o >= cos(theta_max) |F|.
template <class R> struct ReportEnv {
  const int32_t* flags = nullptr;   // env-local body flags: bit 0 robot link, bit 1 end-effector link
  int finger[2] = {-1, -1};
  int target = -1;
  double fmin = 0.0, cosmax = 1.0;
  std::vector<V3<R>> body_force;    // net contact force per dynamic body
  V3<R> target_force, finger_force[2];
  R robot_inc = R(0);
  int grasped = 0;
};

template <class R> R norm3(const V3<R>& a) { return sqrt_(a.x * a.x + a.y * a.y + a.z * a.z); }

template <class R> void contact_report(const EnvState<R>& E, const OracleCfg& cfg, const Detect<R>& det,
                                       const std::vector<V3<R>>& lam_sum, ReportEnv<R>& rp) {
  const int D = E.D, S = E.S;
  const V3<R> z = v3<R>(R(0), R(0), R(0));
  const R dt = R(cfg.dt);
  rp.body_force.assign(D, z);
  rp.target_force = z;
  rp.finger_force[0] = z;
  rp.finger_force[1] = z;
  std::vector<V3<R>> robot_net(D, z);
  auto robot = [&](int i) { return i < D && (rp.flags[i] & 1); };
  auto ee = [&](int i) { return i < D && (rp.flags[i] & 2); };
  auto counts_against = [&](int other) {   // does a contact with `other` count as a robot collision?
    if (other >= D) return other < D + S;   // static boxes count, the plane does not
    return !robot(other) && other != rp.target;
  };
  for (size_t c = 0; c < det.contacts.size(); ++c) {
    const Contact<R>& ct = det.contacts[c];
    V3<R> t1, t2;
    onb(ct.n, t1, t2);
    const V3<R>& L = lam_sum[c];
    V3<R> P = (ct.n * L.x + t1 * L.y) + t2 * L.z;
    V3<R> F = v3<R>(P.x / dt, P.y / dt, P.z / dt);   // on b; -F on a
    const int a = ct.a, b = ct.b;
    rp.body_force[a] = rp.body_force[a] - F;
    if (b < D) rp.body_force[b] = rp.body_force[b] + F;
    if (robot(a) && counts_against(b)) robot_net[a] = robot_net[a] - F;
    if (robot(b) && counts_against(a)) robot_net[b] = robot_net[b] + F;
    if (rp.target >= 0) {
      if (ee(a) && b == rp.target) rp.target_force = rp.target_force + F;
      if (ee(b) && a == rp.target) rp.target_force = rp.target_force - F;
      for (int f = 0; f < 2; ++f) {
        const int fb = rp.finger[f];
        if (fb < 0) continue;
        if (a == fb && b == rp.target) rp.finger_force[f] = rp.finger_force[f] - F;
        if (b == fb && a == rp.target) rp.finger_force[f] = rp.finger_force[f] + F;
      }
    }
  }
  rp.robot_inc = R(0);
  for (int i = 0; i < D; ++i)
    if (robot(i)) rp.robot_inc = rp.robot_inc + norm3(robot_net[i]);
  rp.grasped = 0;
  if (rp.target >= 0 && rp.finger[0] >= 0 && rp.finger[1] >= 0) {
    int ok = 1;
    for (int f = 0; f < 2; ++f) {
      V3<R> o = E.body[rp.finger[f]].x - E.body[rp.finger[1 - f]].x;   // opening direction (unnormalised)
      const V3<R>& Ff = rp.finger_force[f];
      R fn = norm3(Ff);
      R on = norm3(o);
      if (!(fn >= R(rp.fmin)) || !(dot(Ff, o) >= R(rp.cosmax) * fn * on)) ok = 0;
    }
    rp.grasped = ok;
  }
}

// Recorder of the impulses after every sweep of a step (tests): rows of an
// env numbered as joint k row r -> k * 8 + r (jmax joints), then contact
// point c row i -> 8 * jmax + 3 c + i; out holds [substep][sweep][rows].
struct LambdaRec { float* out; int jmax, rows, iterations; };
inline LambdaRec*& lambda_rec() { static thread_local LambdaRec* r = nullptr; return r; }

// One step of one env: detection at the step start, then per substep:
// gravity, rows from the current poses, N solver iterations, position update.
// With `rp`, the contact report of the step is computed at its end.
template <class R> int step_env(EnvState<R>& E, const OracleCfg& cfg, const R* tgt, Detect<R>* dbg,
                                ReportEnv<R>* rp = nullptr) {
  Detect<R> det;
  detect(E, cfg, det);
  int D = E.D;
  int S = cfg.substeps;
  R h = R(cfg.dt) / R(S);
  V3<R> g = v3<R>(R(cfg.gravity[0]), R(cfg.gravity[1]), R(cfg.gravity[2]));
  Solver<R> sv;
  sv.cfg = &cfg;
  sv.h = h;
  sv.Iw.resize(D);
  sv.split.assign(D, R(1));
  bool jacobi = cfg.mode == 1;
  std::vector<V3<R>> lam_sum;
  if (jacobi) {
    std::vector<int> cnt(D, 0);
    for (int k = 0; k < E.J; ++k) {
      if (E.joint[k].parent >= 0) cnt[E.joint[k].parent]++;
      cnt[E.joint[k].child]++;
    }
    for (const Manifold& m : det.manifolds) { cnt[m.a]++; if (m.b < D) cnt[m.b]++; }
    for (int i = 0; i < D; ++i) sv.split[i] = R(cnt[i] > 0 ? cnt[i] : 1);
  }
  for (int s = 0; s < S; ++s) {
    sv.sub = s;
    for (int i = 0; i < D; ++i) E.body[i].v = E.body[i].v + g * h;
    for (int i = 0; i < D; ++i) sv.Iw[i] = world_invI(E.body[i]);
    sv.rows.clear();
    sv.cons.clear();
    for (int k = 0; k < E.J; ++k) sv.joint_rows(E.joint[k], E, tgt);
    for (const Manifold& m : det.manifolds) sv.contact_rows(m, det.contacts, E);
    int ncon = (int)sv.cons.size();
    for (int it = 0; it < cfg.iterations; ++it) {
      if (!jacobi) {
        for (int c = 0; c < det.ncolours; ++c) {
          for (int k = 0; k < ncon; ++k) {
            if (det.colour[k] != c) continue;
            Con& cn = sv.cons[k];
            V3<R> dummy = v3<R>(R(0), R(0), R(0));
            V3<R>* va = cn.a >= 0 ? &E.body[cn.a].v : &dummy;
            V3<R>* wa = cn.a >= 0 ? &E.body[cn.a].w : &dummy;
            V3<R>* vb = cn.b >= 0 ? &E.body[cn.b].v : &dummy;
            V3<R>* wb = cn.b >= 0 ? &E.body[cn.b].w : &dummy;
            for (int r = cn.first; r < cn.first + cn.count; ++r)
              sv.solve_row(sv.rows[r], E, va, wa, vb, wb, nullptr, nullptr, nullptr, nullptr);
          }
        }
      } else {
        // Jacobi: every constraint reads the iteration-start velocities of
        // its split bodies; body velocities then add the true-mass changes
        // in constraint order.
        std::vector<V3<R>> dv(D, v3<R>(R(0), R(0), R(0))), dw(D, v3<R>(R(0), R(0), R(0)));
        for (int k = 0; k < ncon; ++k) {
          Con& cn = sv.cons[k];
          V3<R> z = v3<R>(R(0), R(0), R(0));
          V3<R> va = cn.a >= 0 ? E.body[cn.a].v : z, wa = cn.a >= 0 ? E.body[cn.a].w : z;
          V3<R> vb = cn.b >= 0 ? E.body[cn.b].v : z, wb = cn.b >= 0 ? E.body[cn.b].w : z;
          V3<R> dva = z, dwa = z, dvb = z, dwb = z;
          for (int r = cn.first; r < cn.first + cn.count; ++r)
            sv.solve_row(sv.rows[r], E, &va, &wa, &vb, &wb, &dva, &dwa, &dvb, &dwb);
          if (cn.a >= 0) { dv[cn.a] = dv[cn.a] + dva; dw[cn.a] = dw[cn.a] + dwa; }
          if (cn.b >= 0) { dv[cn.b] = dv[cn.b] + dvb; dw[cn.b] = dw[cn.b] + dwb; }
        }
        for (int i = 0; i < D; ++i) { E.body[i].v = E.body[i].v + dv[i]; E.body[i].w = E.body[i].w + dw[i]; }
      }
      if (LambdaRec* lr = lambda_rec()) {
        float* o = lr->out + ((size_t)s * lr->iterations + it) * lr->rows;
        for (int k = 0; k < E.J; ++k)
          for (int q = 0; q < sv.cons[k].count; ++q) o[8 * k + q] = (float)val(sv.rows[sv.cons[k].first + q].lam);
        for (size_t m = 0; m < det.manifolds.size(); ++m) {
          const Con& cn = sv.cons[E.J + m];
          for (int q = 0; q < cn.count; ++q)
            o[8 * lr->jmax + 3 * det.manifolds[m].first + q] = (float)val(sv.rows[cn.first + q].lam);
        }
      }
    }
    // accumulated impulse (normal, t1, t2) of every contact point over the substeps
    if (rp) {
      if (s == 0) lam_sum.assign(det.contacts.size(), v3<R>(R(0), R(0), R(0)));
      for (size_t m = 0; m < det.manifolds.size(); ++m) {
        const Con& cn = sv.cons[E.J + m];
        for (int k = 0; k < det.manifolds[m].count; ++k) {
          const int r = cn.first + 3 * k;
          V3<R>& L = lam_sum[det.manifolds[m].first + k];
          L = L + v3<R>(sv.rows[r].lam, sv.rows[r + 1].lam, sv.rows[r + 2].lam);
        }
      }
    }
    // a7: x += h v; q <- normalise(q + h/2 (0,w) q)
    for (int i = 0; i < D; ++i) {
      Body<R>& b = E.body[i];
      b.x = b.x + b.v * h;
      Q4<R> wq; wq.w = R(0); wq.x = b.w.x; wq.y = b.w.y; wq.z = b.w.z;
      Q4<R> dq = qmul(wq, b.q);
      R hh = h * R(0.5);
      Q4<R> q; q.w = b.q.w + dq.w * hh; q.x = b.q.x + dq.x * hh; q.y = b.q.y + dq.y * hh; q.z = b.q.z + dq.z * hh;
      R nrm = sqrt_(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
      b.q.w = q.w / nrm; b.q.x = q.x / nrm; b.q.y = q.y / nrm; b.q.z = q.z / nrm;
    }
  }
  if (rp) {
    if (S == 0) lam_sum.assign(det.contacts.size(), v3<R>(R(0), R(0), R(0)));
    contact_report(E, cfg, det, lam_sum, *rp);
  }
  int st = det.status;
  for (int i = 0; i < D; ++i) {
    const Body<R>& b = E.body[i];
    R vals[13] = {b.x.x, b.x.y, b.x.z, b.q.w, b.q.x, b.q.y, b.q.z, b.v.x, b.v.y, b.v.z, b.w.x, b.w.y, b.w.z};
    for (int k = 0; k < 13; ++k) if (!finite_(vals[k])) st |= ST_NONFINITE;
  }
  if (dbg) *dbg = det;
  return st;
}

// Loads env e of the scene with its state (element type T) into working form.
template <class R, class T> void load_env(const OracleScene& sc, int e, const T* pos, const T* quat,
                                          const T* lv, const T* av, const R* mass_override, EnvState<R>& E) {
  int b0 = sc.body_off[e], b1 = sc.body_off[e + 1];
  int s0 = sc.static_off[e], s1 = sc.static_off[e + 1];
  int j0 = sc.joint_off[e], j1 = sc.joint_off[e + 1];
  E.D = b1 - b0; E.S = s1 - s0; E.J = j1 - j0;
  E.body.resize(E.D);
  for (int i = 0; i < E.D; ++i) {
    int g = b0 + i;
    Body<R>& b = E.body[i];
    b.x = v3<R>(R(pos[3 * g]), R(pos[3 * g + 1]), R(pos[3 * g + 2]));
    b.q.w = R(quat[4 * g]); b.q.x = R(quat[4 * g + 1]); b.q.y = R(quat[4 * g + 2]); b.q.z = R(quat[4 * g + 3]);
    b.v = v3<R>(R(lv[3 * g]), R(lv[3 * g + 1]), R(lv[3 * g + 2]));
    b.w = v3<R>(R(av[3 * g]), R(av[3 * g + 1]), R(av[3 * g + 2]));
    b.shape = sc.body_shape[g];
    for (int k = 0; k < 3; ++k) b.dim[k] = R(sc.body_dims[4 * g + k]);
    b.mass = mass_override ? mass_override[g] : R(sc.body_mass[g]);
    b.invm = R(1) / b.mass;
    b.invI = inv_inertia<R>(b.shape, b.mass, b.dim);
  }
  E.stat.resize(E.S);
  for (int i = 0; i < E.S; ++i) {
    const float* p = sc.static_pose + 7 * (s0 + i);
    const float* hh = sc.static_half + 3 * (s0 + i);
    E.stat[i].x = v3<R>(R(p[0]), R(p[1]), R(p[2]));
    E.stat[i].q.w = R(p[3]); E.stat[i].q.x = R(p[4]); E.stat[i].q.y = R(p[5]); E.stat[i].q.z = R(p[6]);
    E.stat[i].h = v3<R>(R(hh[0]), R(hh[1]), R(hh[2]));
  }
  E.joint.resize(E.J);
  for (int i = 0; i < E.J; ++i) {
    int g = j0 + i;
    Joint<R>& j = E.joint[i];
    j.type = sc.joint_type[g]; j.parent = sc.joint_parent[g]; j.child = sc.joint_child[g]; j.dof = sc.joint_dof[g];
    const float* fa = sc.joint_frame_a + 7 * g;
    const float* fb = sc.joint_frame_b + 7 * g;
    j.pa = v3<R>(R(fa[0]), R(fa[1]), R(fa[2]));
    j.qa.w = R(fa[3]); j.qa.x = R(fa[4]); j.qa.y = R(fa[5]); j.qa.z = R(fa[6]);
    j.pb = v3<R>(R(fb[0]), R(fb[1]), R(fb[2]));
    j.qb.w = R(fb[3]); j.qb.x = R(fb[4]); j.qb.y = R(fb[5]); j.qb.z = R(fb[6]);
    j.k = R(sc.joint_gains[4 * g]); j.d = R(sc.joint_gains[4 * g + 1]); j.fmax = R(sc.joint_gains[4 * g + 2]);
    j.lo = R(sc.joint_limits[2 * g]); j.hi = R(sc.joint_limits[2 * g + 1]);
  }
}

template <class R, class T> void store_env(const OracleScene& sc, int e, const EnvState<R>& E,
                                           T* pos, T* quat, T* lv, T* av) {
  int b0 = sc.body_off[e];
  for (int i = 0; i < E.D; ++i) {
    int g = b0 + i;
    const Body<R>& b = E.body[i];
    pos[3 * g] = T(val(b.x.x)); pos[3 * g + 1] = T(val(b.x.y)); pos[3 * g + 2] = T(val(b.x.z));
    quat[4 * g] = T(val(b.q.w)); quat[4 * g + 1] = T(val(b.q.x)); quat[4 * g + 2] = T(val(b.q.y)); quat[4 * g + 3] = T(val(b.q.z));
    lv[3 * g] = T(val(b.v.x)); lv[3 * g + 1] = T(val(b.v.y)); lv[3 * g + 2] = T(val(b.v.z));
    av[3 * g] = T(val(b.w.x)); av[3 * g + 1] = T(val(b.w.y)); av[3 * g + 2] = T(val(b.w.z));
  }
}

template <class R, class TT = float>
int step_batch(const OracleScene* sc, const OracleCfg* cfg, R* pos, R* quat, R* lv, R* av, const TT* targets,
               int nsteps, int32_t* status, int nthreads, const double* mass64 = nullptr) {
  int E = sc->num_envs;
  int md = sc->max_dof > 0 ? sc->max_dof : 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int e = 0; e < E; ++e) {
    EnvState<R> S;
    std::vector<R> mass;
    if (mass64) {
      mass.resize(sc->body_off[E]);
      for (int g = sc->body_off[e]; g < sc->body_off[e + 1]; ++g) mass[g] = R(mass64[g]);
    }
    load_env<R, R>(*sc, e, pos, quat, lv, av, mass64 ? mass.data() : nullptr, S);
    int st = 0;
    std::vector<R> tg(md);
    for (int t = 0; t < nsteps; ++t) {
      const TT* tt = targets ? targets + ((size_t)t * E + e) * md : nullptr;
      for (int k = 0; k < md; ++k) tg[k] = tt ? R(tt[k]) : R(0);
      st |= step_env(S, *cfg, tg.data(), (Detect<R>*)nullptr);
    }
    store_env<R, R>(*sc, e, S, pos, quat, lv, av);
    if (status) status[e] = st;
  }
  return 0;
}

}  // namespace orc

extern "C" struct OracleReportSpec {
  const int32_t* body_flags;   // [B]: bit 0 robot link, bit 1 end-effector link
  const int32_t* fingers;      // [E][2] env-local ids (-1: none)
  const int32_t* target;       // [E] env-local id (-1: none)
  double grasp_min_force;      // N
  double grasp_max_angle_deg;
};

namespace orc {

// `nsteps` steps with the contact report of the last step written out and the
// robot collision force of every step added to robot_force [E].
template <class R>
int step_report_batch(const OracleScene* sc, const OracleCfg* cfg, R* pos, R* quat, R* lv, R* av, const float* targets,
                      int nsteps, int32_t* status, int nthreads, const OracleReportSpec* spec, R* body_force,
                      R* target_force, R* finger_force, R* robot_force, int32_t* grasped) {
  int E = sc->num_envs;
  int md = sc->max_dof > 0 ? sc->max_dof : 1;
  const double cosmax = std::cos(spec->grasp_max_angle_deg * 3.14159265358979323846 / 180.0);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int e = 0; e < E; ++e) {
    EnvState<R> S;
    load_env<R, R>(*sc, e, pos, quat, lv, av, nullptr, S);
    const int b0 = sc->body_off[e];
    ReportEnv<R> rp;
    rp.flags = spec->body_flags + b0;
    rp.finger[0] = spec->fingers ? spec->fingers[2 * e] : -1;
    rp.finger[1] = spec->fingers ? spec->fingers[2 * e + 1] : -1;
    rp.target = spec->target ? spec->target[e] : -1;
    rp.fmin = spec->grasp_min_force;
    rp.cosmax = cosmax;
    int st = 0;
    std::vector<R> tg(md);
    for (int t = 0; t < nsteps; ++t) {
      const float* tt = targets ? targets + ((size_t)t * E + e) * md : nullptr;
      for (int k = 0; k < md; ++k) tg[k] = tt ? R(tt[k]) : R(0);
      st |= step_env(S, *cfg, tg.data(), (Detect<R>*)nullptr, &rp);
      robot_force[e] = robot_force[e] + rp.robot_inc;
    }
    store_env<R, R>(*sc, e, S, pos, quat, lv, av);
    for (int i = 0; i < S.D; ++i) {
      body_force[3 * (b0 + i)] = rp.body_force[i].x;
      body_force[3 * (b0 + i) + 1] = rp.body_force[i].y;
      body_force[3 * (b0 + i) + 2] = rp.body_force[i].z;
    }
    target_force[3 * e] = rp.target_force.x; target_force[3 * e + 1] = rp.target_force.y;
    target_force[3 * e + 2] = rp.target_force.z;
    for (int f = 0; f < 2; ++f) {
      finger_force[6 * e + 3 * f] = rp.finger_force[f].x;
      finger_force[6 * e + 3 * f + 1] = rp.finger_force[f].y;
      finger_force[6 * e + 3 * f + 2] = rp.finger_force[f].z;
    }
    grasped[e] = rp.grasped;
    if (status) status[e] = st;
  }
  return 0;
}

template <class R> int detect_batch(const OracleScene* sc, const OracleCfg* cfg, const R* pos, const R* quat,
                                    R* aabb_body, R* aabb_static, int32_t* pair_count, int32_t* pairs,
                                    int32_t* contact_count, int32_t* contact_ids, R* contact_geom,
                                    int32_t* manifold_count, int32_t* colours, int32_t* ncolours, int32_t* status) {
  int E = sc->num_envs;
  int J = sc->joint_off[E];
  std::vector<R> zero((size_t)3 * sc->body_off[E], R(0));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int e = 0; e < E; ++e) {
    EnvState<R> S;
    load_env<R, R>(*sc, e, pos, quat, zero.data(), zero.data(), nullptr, S);
    Detect<R> d;
    detect(S, *cfg, d);
    int b0 = sc->body_off[e], s0 = sc->static_off[e], j0 = sc->joint_off[e];
    for (int i = 0; i < S.D + S.S; ++i) {
      R* o = i < S.D ? aabb_body + 6 * (b0 + i) : aabb_static + 6 * (s0 + i - S.D);
      const AABB<R>& a = d.aabb[i];
      o[0] = a.lo.x; o[1] = a.lo.y; o[2] = a.lo.z; o[3] = a.hi.x; o[4] = a.hi.y; o[5] = a.hi.z;
    }
    pair_count[e] = (int)d.pairs.size();
    for (size_t p = 0; p < d.pairs.size(); ++p) {
      pairs[((size_t)e * cfg->max_pairs + p) * 2] = d.pairs[p].first;
      pairs[((size_t)e * cfg->max_pairs + p) * 2 + 1] = d.pairs[p].second;
    }
    contact_count[e] = (int)d.contacts.size();
    for (size_t c = 0; c < d.contacts.size(); ++c) {
      const Contact<R>& ct = d.contacts[c];
      size_t k = (size_t)e * cfg->max_contacts + c;
      contact_ids[2 * k] = ct.a; contact_ids[2 * k + 1] = ct.b;
      R* gq = contact_geom + 10 * k;
      gq[0] = ct.n.x; gq[1] = ct.n.y; gq[2] = ct.n.z;
      gq[3] = ct.ra.x; gq[4] = ct.ra.y; gq[5] = ct.ra.z;
      gq[6] = ct.rb.x; gq[7] = ct.rb.y; gq[8] = ct.rb.z; gq[9] = ct.s0;
    }
    manifold_count[e] = (int)d.manifolds.size();
    for (int k = 0; k < S.J; ++k) colours[j0 + k] = d.colour[k];
    for (size_t k = 0; k < d.manifolds.size(); ++k)
      colours[J + (size_t)e * cfg->max_pairs + k] = d.colour[S.J + k];
    ncolours[e] = d.ncolours;
    status[e] = d.status;
  }
  return 0;
}


// Reference gradients by forward-mode dual numbers: the rollout is run with
// every scalar carrying NDIR tangents seeded on the initial velocities, the
// per-step joint targets and the body masses; the loss of env e is the
// squared distance of its goal body to its goal position after the last step.
// Branch decisions (contact set, clamps) follow the primal values, so the
// result is the derivative of the piecewise-smooth rollout at this point.
constexpr int NDIR = 4;
typedef Dual<NDIR> DR;

int grad_batch(const OracleScene* sc, const OracleCfg* cfg, const double* pos, const double* quat, const double* lv,
               const double* av, const float* targets, int nsteps, const int32_t* goal_body, const double* goal_pos,
               int ndir, const double* dvel, const double* dtg, const double* dmass, double* loss, double* dloss,
               int32_t* status, int nthreads) {
  int E = sc->num_envs;
  int B = sc->body_off[E];
  int md = sc->max_dof > 0 ? sc->max_dof : 1;
  if (ndir < 1 || ndir > NDIR) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int e = 0; e < E; ++e) {
    int b0 = sc->body_off[e], D = sc->body_off[e + 1] - b0;
    std::vector<DR> mass(B);
    for (int i = 0; i < D; ++i) {
      int g = b0 + i;
      mass[g] = DR(sc->body_mass[g]);
      for (int k = 0; k < ndir; ++k) mass[g].d[k] = dmass ? dmass[(size_t)k * B + g] : 0.0;
    }
    EnvState<DR> S;
    load_env<DR, double>(*sc, e, pos, quat, lv, av, mass.data(), S);
    for (int i = 0; i < D; ++i) {
      int g = b0 + i;
      for (int k = 0; k < ndir; ++k) {
        const double* dv = dvel ? dvel + ((size_t)k * B + g) * 6 : nullptr;
        if (!dv) continue;
        S.body[i].v.x.d[k] = dv[0]; S.body[i].v.y.d[k] = dv[1]; S.body[i].v.z.d[k] = dv[2];
        S.body[i].w.x.d[k] = dv[3]; S.body[i].w.y.d[k] = dv[4]; S.body[i].w.z.d[k] = dv[5];
      }
    }
    int st = 0;
    std::vector<DR> tg(md);
    for (int t = 0; t < nsteps; ++t) {
      for (int j = 0; j < md; ++j) {
        size_t idx = ((size_t)t * E + e) * md + j;
        tg[j] = DR(targets ? (double)targets[idx] : 0.0);
        for (int k = 0; k < ndir; ++k)
          tg[j].d[k] = dtg ? dtg[(size_t)k * nsteps * E * md + idx] : 0.0;
      }
      st |= step_env(S, *cfg, tg.data(), (Detect<DR>*)nullptr);
    }
    DR L = DR(0.0);
    int gb = goal_body ? goal_body[e] : -1;
    if (gb >= 0 && gb < D) {
      V3<DR> d = S.body[gb].x - v3<DR>(DR(goal_pos[3 * e]), DR(goal_pos[3 * e + 1]), DR(goal_pos[3 * e + 2]));
      L = dot(d, d);
    }
    loss[e] = L.v;
    for (int k = 0; k < ndir; ++k) dloss[(size_t)k * E + e] = L.d[k];
    if (status) status[e] = st;
  }
  return 0;
}

// Reference vector-Jacobian products of ONE step by reverse mode. For env e
// the step maps (state x, joint targets u, body masses m) to the state x';
// given the adjoint w of x' (seed, double) it returns w^T dx'/dx, w^T dx'/du
// and w^T dx'/dm (each written, not added), along with x' itself. Every
// scalar of the step is a Rev<P>: inputs are tape leaves, the step runs as in
// step_env, the outputs are seeded with w and the tape is swept once. Branch
// decisions (contact set and features, colouring, clamps, bias cases) follow
// the primal values, so the result is the derivative of the piecewise-smooth
// step on the piece that contains this point; with P = float the primal and
// hence every decision is the FP32 oracle's.
}  // namespace orc

// Decision reporting and inversion of a reverse-mode step (see DecisionLog):
// margins, and per env the number of fragile decisions with the first kmax
// of their indices; flip_off [E+1] / flip_idx: per env (CSR) the decision
// indices to take the other way. NULL in the entry points: no log.
extern "C" struct OracleDecisions {
  double delta, len_tol;
  int32_t kmax;
  int32_t* nfragile;        // [E]
  int32_t* fragile;         // [E][kmax] decision indices
  int32_t* fragile_site;    // [E][kmax] solver row of each (-1: joint limit or contact bias), may be NULL
  int32_t* fragile_choice;  // [E][kmax] its natural outcome (1: the clamp is active), may be NULL
  double* fragile_margin;   // [E][kmax] margin of each, may be NULL
  const int32_t* flip_off;  // [E+1] or NULL
  const int32_t* flip_idx;
};

namespace orc {

template <class P, class T>
int vjp_batch(const OracleScene* sc, const OracleCfg* cfg, const T* pos, const T* quat, const T* lv, const T* av,
              const T* targets, const double* wpos, const double* wquat, const double* wlv, const double* wav,
              T* opos, T* oquat, T* olv, T* oav, double* gpos, double* gquat, double* glv, double* gav,
              double* gtg, double* gmass, int32_t* status, int nthreads, const OracleDecisions* dec) {
  typedef Rev<P> RV;
  const int E = sc->num_envs;
  const int B = sc->body_off[E];
  const int md = sc->max_dof > 0 ? sc->max_dof : 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int e = 0; e < E; ++e) {
    static thread_local RevTape tape;   // reused by the thread's envs (keeps its capacity)
    tape.clear();
    rev_tape() = &tape;
    DecisionLog log;
    if (dec) {
      log.delta = dec->delta;
      log.len_tol = dec->len_tol;
      if (dec->flip_off) {
        log.flip = dec->flip_idx + dec->flip_off[e];
        log.nflip = dec->flip_off[e + 1] - dec->flip_off[e];
      }
      dec_log() = &log;
    }
    const int b0 = sc->body_off[e], D = sc->body_off[e + 1] - b0;
    std::vector<RV> mass(B);
    for (int i = 0; i < D; ++i) mass[b0 + i] = RV::leaf(P(sc->body_mass[b0 + i]));
    EnvState<RV> S;
    load_env<RV, T>(*sc, e, pos, quat, lv, av, mass.data(), S);
    std::vector<int> in_id(13 * D);   // tape ids of the state leaves
    for (int i = 0; i < D; ++i) {
      Body<RV>& b = S.body[i];
      RV* xs[13] = {&b.x.x, &b.x.y, &b.x.z, &b.q.w, &b.q.x, &b.q.y, &b.q.z, &b.v.x, &b.v.y, &b.v.z,
                    &b.w.x, &b.w.y, &b.w.z};
      for (int k = 0; k < 13; ++k) {
        *xs[k] = RV::leaf(xs[k]->v);
        in_id[13 * i + k] = xs[k]->id;
      }
    }
    std::vector<RV> tg(md);
    for (int k = 0; k < md; ++k)
      tg[k] = RV::leaf(P(targets && sc->max_dof > 0 ? (double)targets[(size_t)e * sc->max_dof + k] : 0.0));
    const int st = step_env(S, *cfg, tg.data(), (Detect<RV>*)nullptr);
    for (int i = 0; i < D; ++i) {
      const int g = b0 + i;
      const Body<RV>& b = S.body[i];
      const RV* ys[13] = {&b.x.x, &b.x.y, &b.x.z, &b.q.w, &b.q.x, &b.q.y, &b.q.z, &b.v.x, &b.v.y, &b.v.z,
                          &b.w.x, &b.w.y, &b.w.z};
      const double w[13] = {wpos[3 * g], wpos[3 * g + 1], wpos[3 * g + 2], wquat[4 * g], wquat[4 * g + 1],
                            wquat[4 * g + 2], wquat[4 * g + 3], wlv[3 * g], wlv[3 * g + 1], wlv[3 * g + 2],
                            wav[3 * g], wav[3 * g + 1], wav[3 * g + 2]};
      for (int k = 0; k < 13; ++k) tape.seed(ys[k]->id, w[k]);
      if (opos) {
        opos[3 * g] = T(ys[0]->v); opos[3 * g + 1] = T(ys[1]->v); opos[3 * g + 2] = T(ys[2]->v);
        for (int k = 0; k < 4; ++k) oquat[4 * g + k] = T(ys[3 + k]->v);
        for (int k = 0; k < 3; ++k) { olv[3 * g + k] = T(ys[7 + k]->v); oav[3 * g + k] = T(ys[10 + k]->v); }
      }
    }
    tape.sweep();
    for (int i = 0; i < D; ++i) {
      const int g = b0 + i;
      gmass[g] = tape.get(mass[g].id);
      const int* id = &in_id[13 * i];
      for (int k = 0; k < 3; ++k) gpos[3 * g + k] = tape.get(id[k]);
      for (int k = 0; k < 4; ++k) gquat[4 * g + k] = tape.get(id[3 + k]);
      for (int k = 0; k < 3; ++k) { glv[3 * g + k] = tape.get(id[7 + k]); gav[3 * g + k] = tape.get(id[10 + k]); }
    }
    if (gtg && sc->max_dof > 0)
      for (int k = 0; k < sc->max_dof; ++k) gtg[(size_t)e * sc->max_dof + k] = tape.get(tg[k].id);
    if (status) status[e] = st;
    rev_tape() = nullptr;
    if (dec) {
      dec_log() = nullptr;
      dec->nfragile[e] = (int32_t)log.fragile.size();
      for (int k = 0; k < dec->kmax && k < (int)log.fragile.size(); ++k) {
        const size_t o = (size_t)e * dec->kmax + k;
        dec->fragile[o] = log.fragile[k];
        if (dec->fragile_site) dec->fragile_site[o] = log.fragile_site[k];
        if (dec->fragile_choice) dec->fragile_choice[o] = log.fragile_choice[k];
        if (dec->fragile_margin) dec->fragile_margin[o] = log.fragile_margin[k];
      }
    }
  }
  return 0;
}

}  // namespace orc

extern "C" {

// One step's vector-Jacobian products by reverse mode (see vjp_batch): the
// FP32 form (primal arithmetic and decisions of the FP32 oracle, adjoints in
// double) and the FP64 form. State arrays [B][3|4], targets [E][max_dof];
// seeds w* and outputs g* are double; gtg [E][max_dof] and gmass [B] are
// written; o* receive the stepped state (may be NULL together); dec (may be
// NULL) reports fragile decisions and inverts chosen ones.
int oracle_vjp_f32(const OracleScene* sc, const OracleCfg* cfg, const float* pos, const float* quat, const float* lv,
                   const float* av, const float* targets, const double* wpos, const double* wquat, const double* wlv,
                   const double* wav, float* opos, float* oquat, float* olv, float* oav, double* gpos, double* gquat,
                   double* glv, double* gav, double* gtg, double* gmass, int32_t* status, int nthreads,
                   const OracleDecisions* dec) {
  return orc::vjp_batch<float, float>(sc, cfg, pos, quat, lv, av, targets, wpos, wquat, wlv, wav, opos, oquat, olv,
                                      oav, gpos, gquat, glv, gav, gtg, gmass, status, nthreads, dec);
}
int oracle_vjp_f64(const OracleScene* sc, const OracleCfg* cfg, const double* pos, const double* quat,
                   const double* lv, const double* av, const double* targets, const double* wpos, const double* wquat,
                   const double* wlv, const double* wav, double* opos, double* oquat, double* olv, double* oav,
                   double* gpos, double* gquat, double* glv, double* gav, double* gtg, double* gmass, int32_t* status,
                   int nthreads, const OracleDecisions* dec) {
  return orc::vjp_batch<double, double>(sc, cfg, pos, quat, lv, av, targets, wpos, wquat, wlv, wav, opos, oquat, olv,
                                        oav, gpos, gquat, glv, gav, gtg, gmass, status, nthreads, dec);
}

int oracle_step_f32(const OracleScene* sc, const OracleCfg* cfg, float* pos, float* quat, float* lv,
                    float* av, const float* targets, int nsteps, int32_t* status, int nthreads) {
  return orc::step_batch<float>(sc, cfg, pos, quat, lv, av, targets, nsteps, status, nthreads);
}
int oracle_step_f64(const OracleScene* sc, const OracleCfg* cfg, double* pos, double* quat, double* lv,
                    double* av, const float* targets, int nsteps, int32_t* status, int nthreads) {
  return orc::step_batch<double>(sc, cfg, pos, quat, lv, av, targets, nsteps, status, nthreads);
}
// FP64 rollout whose joint targets [nsteps][E][max_dof] and body masses [B]
// are given in double (so finite differences can use exact perturbations).
int oracle_step_f64x(const OracleScene* sc, const OracleCfg* cfg, double* pos, double* quat, double* lv,
                     double* av, const double* targets, const double* mass, int nsteps, int32_t* status,
                     int nthreads) {
  return orc::step_batch<double, double>(sc, cfg, pos, quat, lv, av, targets, nsteps, status, nthreads, mass);
}
int oracle_detect_f32(const OracleScene* sc, const OracleCfg* cfg, const float* pos, const float* quat,
                      float* aabb_body, float* aabb_static, int32_t* pair_count, int32_t* pairs,
                      int32_t* contact_count, int32_t* contact_ids, float* contact_geom,
                      int32_t* manifold_count, int32_t* colours, int32_t* ncolours, int32_t* status) {
  return orc::detect_batch<float>(sc, cfg, pos, quat, aabb_body, aabb_static, pair_count, pairs, contact_count,
                                  contact_ids, contact_geom, manifold_count, colours, ncolours, status);
}
int oracle_detect_f64(const OracleScene* sc, const OracleCfg* cfg, const double* pos, const double* quat,
                      double* aabb_body, double* aabb_static, int32_t* pair_count, int32_t* pairs,
                      int32_t* contact_count, int32_t* contact_ids, double* contact_geom,
                      int32_t* manifold_count, int32_t* colours, int32_t* ncolours, int32_t* status) {
  return orc::detect_batch<double>(sc, cfg, pos, quat, aabb_body, aabb_static, pair_count, pairs, contact_count,
                                   contact_ids, contact_geom, manifold_count, colours, ncolours, status);
}
// Loss and NDIR (<= 4) directional derivatives of the rollout (see grad_batch).
// dvel [ndir][B][6] (linear, angular), dtg [ndir][nsteps][E][max_dof],
// dmass [ndir][B]; any may be NULL. Outputs loss [E], dloss [ndir][E].
int oracle_grad_f64(const OracleScene* sc, const OracleCfg* cfg, const double* pos, const double* quat,
                    const double* lv, const double* av, const float* targets, int nsteps, const int32_t* goal_body,
                    const double* goal_pos, int ndir, const double* dvel, const double* dtg, const double* dmass,
                    double* loss, double* dloss, int32_t* status, int nthreads) {
  return orc::grad_batch(sc, cfg, pos, quat, lv, av, targets, nsteps, goal_body, goal_pos, ndir, dvel, dtg, dmass,
                         loss, dloss, status, nthreads);
}
// `nsteps` steps with the contact report (see contact_report): body_force [B][3],
// target_force [E][3] and finger_force [E][2][3] of the last step, grasped [E];
// robot_force [E] accumulates every step's robot collision force.
int oracle_step_report_f32(const OracleScene* sc, const OracleCfg* cfg, float* pos, float* quat, float* lv, float* av,
                           const float* targets, int nsteps, int32_t* status, int nthreads,
                           const OracleReportSpec* spec, float* body_force, float* target_force, float* finger_force,
                           float* robot_force, int32_t* grasped) {
  return orc::step_report_batch<float>(sc, cfg, pos, quat, lv, av, targets, nsteps, status, nthreads, spec,
                                       body_force, target_force, finger_force, robot_force, grasped);
}
int oracle_step_report_f64(const OracleScene* sc, const OracleCfg* cfg, double* pos, double* quat, double* lv,
                           double* av, const float* targets, int nsteps, int32_t* status, int nthreads,
                           const OracleReportSpec* spec, double* body_force, double* target_force,
                           double* finger_force, double* robot_force, int32_t* grasped) {
  return orc::step_report_batch<double>(sc, cfg, pos, quat, lv, av, targets, nsteps, status, nthreads, spec,
                                        body_force, target_force, finger_force, robot_force, grasped);
}
// One FP32 step of every env with the impulses after every sweep written to
// lam [E][substeps][iterations][8 * jmax + 3 * max_contacts] (see LambdaRec).
int oracle_step_lambdas_f32(const OracleScene* sc, const OracleCfg* cfg, float* pos, float* quat, float* lv,
                            float* av, const float* targets, int jmax, float* lam, int nthreads) {
  const int E = sc->num_envs;
  const int md = sc->max_dof > 0 ? sc->max_dof : 1;
  const int rows = 8 * jmax + 3 * cfg->max_contacts;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int e = 0; e < E; ++e) {
    orc::EnvState<float> S;
    orc::load_env<float, float>(*sc, e, pos, quat, lv, av, nullptr, S);
    std::vector<float> tg(md);
    for (int k = 0; k < md; ++k) tg[k] = targets ? targets[(size_t)e * md + k] : 0.f;
    orc::LambdaRec rec;
    rec.out = lam + (size_t)e * cfg->substeps * cfg->iterations * rows;
    rec.jmax = jmax; rec.rows = rows; rec.iterations = cfg->iterations;
    orc::lambda_rec() = &rec;
    orc::step_env(S, *cfg, tg.data(), (orc::Detect<float>*)nullptr);
    orc::lambda_rec() = nullptr;
    orc::store_env<float, float>(*sc, e, S, pos, quat, lv, av);
  }
  return 0;
}

// Clip outputs dropped by the box-box clipper's 8-vertex cap since the
// library was loaded (a convex quad clipped by four half-planes has at most
// 8 vertices in exact arithmetic; this counts any rounding case beyond it).
long long oracle_clip_cap_drops(void) { return orc::clip_cap_drops(); }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
