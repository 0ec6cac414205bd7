// Collision stages of the step: world AABBs (a2) and primitive narrowphase
// to contact manifolds (a4). Templated on the scalar; the step instantiates
// them with `nf` (no FMA contraction) so that pair lists and contact counts
// are reproducible bit for bit from identical poses.
//
// Manifold routines follow the methods named in the library header:
// closed-form sphere and plane contacts; segment-segment closest points for
// capsules (Ericson, Real-Time Collision Detection, 5.1.9), two points when
// the segments are near-parallel; capsule-box as sphere-box tests at the two
// endpoints and at the exact minimiser of the segment-box distance; box-box by
// the separating-axis test over 15 axes, Sutherland-Hodgman clipping of the
// incident face and reduction to 4 points, or one edge-edge point.
// Every routine returns points whose normal points from its first shape to
// its second, with pa on the first, pb on the second, s = n.(pb - pa).
// The four large routines (sphere-box, capsule-capsule, capsule-box,
// box-box) are kept out of line: the persistent step kernel runs every stage
// in one body, and with them inlined its code crowds the solver loop out of
// the instruction caches (measured on the 4096-env apartment batch: 1.98 ms
// per step inlined, 1.89 ms out of line; making the small routines or the
// stage functions out of line as well was slower).
#pragma once
#include "msh_math.cuh"

namespace msh {

enum { SH_SPHERE = 0, SH_CAPSULE = 1, SH_BOX = 2, SH_PLANE = 3 };

template <class T> struct Pt { V3<T> n, pa, pb; T s; };
template <class T> struct Shape { int type; V3<T> c; M3<T> M; T d0, d1, d2; };

template <class T> struct AABBt { V3<T> lo, hi; };

template <class T> __device__ __forceinline__ AABBt<T> shape_aabb(const Shape<T>& s, T off) {
  V3<T> e;
  if (s.type == SH_SPHERE) {
    e = v3<T>(s.d0, s.d0, s.d0);
  } else if (s.type == SH_CAPSULE) {
    V3<T> a = col(s.M, 0);
    e = v3<T>(abs_(a.x) * s.d1 + s.d0, abs_(a.y) * s.d1 + s.d0, abs_(a.z) * s.d1 + s.d0);
  } else {
    e.x = abs_(s.M.m[0][0]) * s.d0 + abs_(s.M.m[0][1]) * s.d1 + abs_(s.M.m[0][2]) * s.d2;
    e.y = abs_(s.M.m[1][0]) * s.d0 + abs_(s.M.m[1][1]) * s.d1 + abs_(s.M.m[1][2]) * s.d2;
    e.z = abs_(s.M.m[2][0]) * s.d0 + abs_(s.M.m[2][1]) * s.d1 + abs_(s.M.m[2][2]) * s.d2;
  }
  AABBt<T> b;
  b.lo = v3<T>((s.c.x - e.x) - off, (s.c.y - e.y) - off, (s.c.z - e.z) - off);
  b.hi = v3<T>((s.c.x + e.x) + off, (s.c.y + e.y) + off, (s.c.z + e.z) + off);
  return b;
}

template <class T> __device__ int sphere_sphere(V3<T> c1, T r1, V3<T> c2, T r2, Pt<T>* out) {
  V3<T> d = c2 - c1;
  T dist = sqrt_(dot(d, d));
  V3<T> n;
  if (dist > T(1e-6f)) n = v3<T>(d.x / dist, d.y / dist, d.z / dist);
  else n = v3<T>(T(0.f), T(0.f), T(1.f));
  out[0].n = n;
  out[0].s = (dist - r1) - r2;
  out[0].pa = c1 + n * r1;
  out[0].pb = c2 - n * r2;
  return 1;
}

template <class T> __device__ int sphere_plane(V3<T> c, T r, Pt<T>* out) {
  out[0].n = v3<T>(T(0.f), T(0.f), T(-1.f));
  out[0].s = c.z - r;
  out[0].pa = v3<T>(c.x, c.y, c.z - r);
  out[0].pb = v3<T>(c.x, c.y, T(0.f));
  return 1;
}

template <class T> __device__ int sphere_capsule(V3<T> c, T r, const Shape<T>& cap, Pt<T>* out) {
  V3<T> a = col(cap.M, 0);
  T t = clampv(dot(c - cap.c, a), -cap.d1, cap.d1);
  V3<T> q = cap.c + a * t;
  return sphere_sphere(c, r, q, cap.d0, out);
}

template <class T> __device__ __noinline__ int sphere_box(V3<T> c, T r, const Shape<T>& box, Pt<T>* out) {
  V3<T> l = mulT(box.M, c - box.c);
  T h[3] = {box.d0, box.d1, box.d2};
  bool inside = abs_(l.x) <= h[0] && abs_(l.y) <= h[1] && abs_(l.z) <= h[2];
  V3<T> nl, pl;
  T s;
  if (!inside) {
    V3<T> q = v3<T>(clampv(l.x, -h[0], h[0]), clampv(l.y, -h[1], h[1]), clampv(l.z, -h[2], h[2]));
    V3<T> df = l - q;
    T dist = sqrt_(dot(df, df));
    nl = v3<T>(df.x / dist, df.y / dist, df.z / dist);
    s = dist - r;
    pl = q;
  } else {
    T dx = h[0] - abs_(l.x), dy = h[1] - abs_(l.y), dz = h[2] - abs_(l.z);
    int k = 0;
    T best = dx;
    if (dy < best) { k = 1; best = dy; }
    if (dz < best) { k = 2; best = dz; }
    T lk = comp(l, k);
    T sg = lk >= T(0.f) ? T(1.f) : T(-1.f);
    nl = unit<T>(k) * sg;
    s = -best - r;
    pl = l;
    setc(pl, k, sg * h[k]);
  }
  V3<T> nw = mul(box.M, nl);
  out[0].n = -nw;
  out[0].s = s;
  out[0].pa = c + out[0].n * r;
  out[0].pb = box.c + mul(box.M, pl);
  return 1;
}

template <class T> __device__ int capsule_plane(const Shape<T>& cap, T off, Pt<T>* out) {
  V3<T> a = col(cap.M, 0);
  int n = 0;
  for (int e = 0; e < 2; ++e) {
    T t = e == 0 ? -cap.d1 : cap.d1;
    V3<T> p = cap.c + a * t;
    T s = p.z - cap.d0;
    if (s < off) {
      out[n].n = v3<T>(T(0.f), T(0.f), T(-1.f));
      out[n].s = s;
      out[n].pa = v3<T>(p.x, p.y, p.z - cap.d0);
      out[n].pb = v3<T>(p.x, p.y, T(0.f));
      ++n;
    }
  }
  return n;
}

template <class T> __device__ __noinline__ int capsule_capsule(const Shape<T>& c1, const Shape<T>& c2, Pt<T>* out) {
  V3<T> a1 = col(c1.M, 0), a2 = col(c2.M, 0);
  T L1 = c1.d1, L2 = c2.d1;
  V3<T> rr = c1.c - c2.c;
  T b = dot(a1, a2), cc = dot(a1, rr), f = dot(a2, rr);
  V3<T> cr = cross(a1, a2);
  if (dot(cr, cr) < T(1e-6f)) {
    T ta = -cc - b * L2, tb = -cc + b * L2;
    T lo = minv(ta, tb), hi = maxv(ta, tb);
    lo = maxv(lo, -L1);
    hi = minv(hi, L1);
    if (lo <= hi) {
      int n = 0;
      for (int e = 0; e < 2; ++e) {
        if (e == 1 && hi == lo) break;
        T t = e == 0 ? lo : hi;
        V3<T> p1 = c1.c + a1 * t;
        T u = clampv(dot(p1 - c2.c, a2), -L2, L2);
        V3<T> p2 = c2.c + a2 * u;
        n += sphere_sphere(p1, c1.d0, p2, c2.d0, out + n);
      }
      return n;
    }
  }
  T denom = T(1.f) - b * b;
  T s = denom > T(1e-6f) ? clampv((b * f - cc) / denom, -L1, L1) : T(0.f);
  T t = b * s + f;
  if (t < -L2) { t = -L2; s = clampv(b * t - cc, -L1, L1); }
  else if (t > L2) { t = L2; s = clampv(b * t - cc, -L1, L1); }
  V3<T> p1 = c1.c + a1 * s, p2 = c2.c + a2 * t;
  return sphere_sphere(p1, c1.d0, p2, c2.d0, out);
}

template <class T> __device__ __forceinline__ T seg_box_d2(const V3<T>& p0, const V3<T>& d, const T* h, T t) {
  T acc = T(0.f);
  for (int k = 0; k < 3; ++k) {
    T x = comp(p0, k) + comp(d, k) * t;
    T q = clampv(x, -h[k], h[k]);
    T e = x - q;
    acc = acc + e * e;
  }
  return acc;
}

template <class T> __device__ __noinline__ int capsule_box(const Shape<T>& cap, const Shape<T>& box, T off, Pt<T>* out) {
  V3<T> a = col(cap.M, 0);
  T L = cap.d1;
  T h[3] = {box.d0, box.d1, box.d2};
  V3<T> p0 = mulT(box.M, cap.c - box.c);
  V3<T> d = mulT(box.M, a);
  T brk[8];
  int nb = 0;
  brk[nb++] = -L;
  for (int k = 0; k < 3; ++k) {
    T dk = comp(d, k);
    if (abs_(dk) > T(1e-6f)) {
      for (int e = 0; e < 2; ++e) {
        T bound = e == 0 ? -h[k] : h[k];
        T t = (bound - comp(p0, k)) / dk;
        if (t > -L && t < L) brk[nb++] = t;
      }
    }
  }
  brk[nb++] = L;
  for (int i = 1; i < nb; ++i) {
    T key = brk[i];
    int j = i - 1;
    while (j >= 0 && brk[j] > key) { brk[j + 1] = brk[j]; --j; }
    brk[j + 1] = key;
  }
  T best_t = -L;
  T best_f = seg_box_d2(p0, d, h, best_t);
  for (int i = 0; i + 1 < nb; ++i) {
    T t0 = brk[i], t1 = brk[i + 1];
    if (!(t1 > t0)) continue;
    T tm = (t0 + t1) * T(0.5f);
    T A = T(0.f), B = T(0.f);
    for (int k = 0; k < 3; ++k) {
      T x = comp(p0, k) + comp(d, k) * tm;
      T bound;
      if (x > h[k]) bound = h[k];
      else if (x < -h[k]) bound = -h[k];
      else continue;
      T e = comp(p0, k) - bound;
      A = A + comp(d, k) * comp(d, k);
      B = B + comp(d, k) * e;
    }
    T topt = A > T(0.f) ? clampv(-B / A, t0, t1) : t0;
    T fo = seg_box_d2(p0, d, h, topt);
    if (fo < best_f) { best_f = fo; best_t = topt; }
  }
  T cand[3];
  int nc = 0;
  cand[nc++] = -L;
  cand[nc++] = L;
  if ((best_t + L) > T(1e-3f) && (L - best_t) > T(1e-3f)) cand[nc++] = best_t;
  int n = 0;
  for (int i = 0; i < nc; ++i) {
    V3<T> q = cap.c + a * cand[i];
    Pt<T> p;
    sphere_box(q, cap.d0, box, &p);
    if (p.s < off) out[n++] = p;
  }
  return n;
}

template <class T> __device__ int box_plane(const Shape<T>& box, T off, Pt<T>* out) {
  V3<T> v[8];
  T s[8];
  for (int i = 0; i < 8; ++i) {
    V3<T> l = v3<T>((i & 1) ? box.d0 : -box.d0, (i & 2) ? box.d1 : -box.d1, (i & 4) ? box.d2 : -box.d2);
    v[i] = box.c + mul(box.M, l);
    s[i] = v[i].z;
  }
  unsigned used = 0u;
  int n = 0;
  while (n < 4) {
    int k = -1;
    for (int i = 0; i < 8; ++i) {
      if ((used >> i) & 1u) continue;
      if (!(s[i] < off)) continue;
      if (k < 0 || s[i] < s[k]) k = i;
    }
    if (k < 0) break;
    used |= 1u << k;
    out[n].n = v3<T>(T(0.f), T(0.f), T(-1.f));
    out[n].s = s[k];
    out[n].pa = v[k];
    out[n].pb = v3<T>(v[k].x, v[k].y, T(0.f));
    ++n;
  }
  return n;
}

template <class T> __device__ int clip_poly(const T (*in)[3], int n, T (*out)[3], int axis, T sg, T bound) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const T* P = in[i];
    const T* Q = in[(i + 1) % n];
    T dp = sg * P[axis] - bound;
    T dq = sg * Q[axis] - bound;
    if (dp <= T(0.f) && m < 8) { out[m][0] = P[0]; out[m][1] = P[1]; out[m][2] = P[2]; ++m; }
    if (((dp < T(0.f) && dq > T(0.f)) || (dp > T(0.f) && dq < T(0.f))) && m < 8) {
      T t = dp / (dp - dq);
      for (int k = 0; k < 3; ++k) out[m][k] = P[k] + (Q[k] - P[k]) * t;
      ++m;
    }
  }
  return m;
}

template <class T> __device__ __noinline__ int box_box(const Shape<T>& A, const Shape<T>& B, T off, Pt<T>* out) {
  V3<T> d = B.c - A.c;
  V3<T> axA[3] = {col(A.M, 0), col(A.M, 1), col(A.M, 2)};
  V3<T> axB[3] = {col(B.M, 0), col(B.M, 1), col(B.M, 2)};
  T hA[3] = {A.d0, A.d1, A.d2}, hB[3] = {B.d0, B.d1, B.d2};
  T C[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = abs_(dot(axA[i], axB[j]));
  T dA[3], dB[3];
  for (int i = 0; i < 3; ++i) { dA[i] = dot(d, axA[i]); dB[i] = dot(d, axB[i]); }
  T best_face_sep = T(0.f);
  int best_face = -1;
  for (int i = 0; i < 3; ++i) {
    T pB = hB[0] * C[i][0] + hB[1] * C[i][1] + hB[2] * C[i][2];
    T sep = abs_(dA[i]) - (hA[i] + pB);
    if (sep > off) return 0;
    if (best_face < 0 || sep > best_face_sep) { best_face_sep = sep; best_face = i; }
  }
  for (int j = 0; j < 3; ++j) {
    T pA = hA[0] * C[0][j] + hA[1] * C[1][j] + hA[2] * C[2][j];
    T sep = abs_(dB[j]) - (pA + hB[j]);
    if (sep > off) return 0;
    if (sep > best_face_sep) { best_face_sep = sep; best_face = 3 + j; }
  }
  T best_edge_sep = T(0.f);
  int best_edge = -1;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      V3<T> Lx = cross(axA[i], axB[j]);
      T len = sqrt_(dot(Lx, Lx));
      if (len < T(1e-5f)) continue;
      V3<T> L = v3<T>(Lx.x / len, Lx.y / len, Lx.z / len);
      T pA = hA[0] * abs_(dot(L, axA[0])) + hA[1] * abs_(dot(L, axA[1])) + hA[2] * abs_(dot(L, axA[2]));
      T pB = hB[0] * abs_(dot(L, axB[0])) + hB[1] * abs_(dot(L, axB[1])) + hB[2] * abs_(dot(L, axB[2]));
      T sep = abs_(dot(d, L)) - (pA + pB);
      if (sep > off) return 0;
      if (best_edge < 0 || sep > best_edge_sep) { best_edge_sep = sep; best_edge = 3 * i + j; }
    }
  }
  bool use_edge = best_edge >= 0 &&
                  best_edge_sep > best_face_sep + T(1e-4f) * (T(1.f) + abs_(best_face_sep));
  if (use_edge) {
    int i = best_edge / 3, j = best_edge % 3;
    V3<T> Lx = cross(axA[i], axB[j]);
    T len = sqrt_(dot(Lx, Lx));
    V3<T> L = v3<T>(Lx.x / len, Lx.y / len, Lx.z / len);
    V3<T> n = dot(d, L) >= T(0.f) ? L : -L;
    V3<T> pa = A.c;
    for (int m = 0; m < 3; ++m) {
      if (m == i) continue;
      T sg = dot(n, axA[m]) > T(0.f) ? T(1.f) : T(-1.f);
      pa = pa + axA[m] * (hA[m] * sg);
    }
    V3<T> pb = B.c;
    for (int m = 0; m < 3; ++m) {
      if (m == j) continue;
      T sg = dot(n, axB[m]) > T(0.f) ? T(-1.f) : T(1.f);
      pb = pb + axB[m] * (hB[m] * sg);
    }
    V3<T> rr = pa - pb;
    T b = dot(axA[i], axB[j]), cc = dot(axA[i], rr), f = dot(axB[j], rr);
    T denom = T(1.f) - b * b;
    T s = denom > T(1e-6f) ? (b * f - cc) / denom : T(0.f);
    s = clampv(s, -hA[i], hA[i]);
    T t = clampv(b * s + f, -hB[j], hB[j]);
    V3<T> qa = pa + axA[i] * s, qb = pb + axB[j] * t;
    T sep = dot(n, qb - qa);
    if (!(sep < off)) return 0;
    out[0].n = n; out[0].pa = qa; out[0].pb = qb; out[0].s = sep;
    return 1;
  }
  bool refA = best_face < 3;
  int k = refA ? best_face : best_face - 3;
  const V3<T>* axR = refA ? axA : axB;
  const V3<T>* axI = refA ? axB : axA;
  const T* hR = refA ? hA : hB;
  const T* hI = refA ? hB : hA;
  V3<T> cR = refA ? A.c : B.c, cI = refA ? B.c : A.c;
  T dist = refA ? dA[k] : dB[k];
  T sgn = refA ? (dist >= T(0.f) ? T(1.f) : T(-1.f)) : (dist >= T(0.f) ? T(-1.f) : T(1.f));
  V3<T> nR = axR[k] * sgn;
  V3<T> fc = cR + nR * hR[k];
  int ku = (k + 1) % 3, kv = (k + 2) % 3;
  V3<T> u = axR[ku], v = axR[kv];
  T hu = hR[ku], hv = hR[kv];
  int m = 0;
  T bestd = abs_(dot(nR, axI[0]));
  T dm = dot(nR, axI[0]);
  for (int q = 1; q < 3; ++q) {
    T dq = dot(nR, axI[q]);
    if (abs_(dq) > bestd) { bestd = abs_(dq); m = q; dm = dq; }
  }
  T sgI = dm > T(0.f) ? T(-1.f) : T(1.f);
  V3<T> ic = cI + axI[m] * (hI[m] * sgI);
  int m1 = (m + 1) % 3, m2 = (m + 2) % 3;
  V3<T> e1 = axI[m1] * hI[m1], e2 = axI[m2] * hI[m2];
  V3<T> vert[4] = {(ic + e1) + e2, (ic - e1) + e2, (ic - e1) - e2, (ic + e1) - e2};
  T P0[8][3], P1[8][3];
  for (int i = 0; i < 4; ++i) {
    V3<T> rel = vert[i] - fc;
    P0[i][0] = dot(rel, u); P0[i][1] = dot(rel, v); P0[i][2] = dot(rel, nR);
  }
  int np = 4;
  np = clip_poly<T>(P0, np, P1, 0, T(1.f), hu);
  np = clip_poly<T>(P1, np, P0, 0, T(-1.f), hu);
  np = clip_poly<T>(P0, np, P1, 1, T(1.f), hv);
  np = clip_poly<T>(P1, np, P0, 1, T(-1.f), hv);
  int keep[8];
  int nk = 0;
  for (int i = 0; i < np; ++i) if (P0[i][2] < off) keep[nk++] = i;
  int sel[4];
  int ns = 0;
  if (nk <= 4) {
    for (int i = 0; i < nk; ++i) sel[ns++] = keep[i];
  } else {
    int i0 = keep[0];
    for (int i = 1; i < nk; ++i) if (P0[keep[i]][2] < P0[i0][2]) i0 = keep[i];
    int i1 = -1; T bd = T(0.f);
    for (int i = 0; i < nk; ++i) {
      int c = keep[i]; if (c == i0) continue;
      T dx = P0[c][0] - P0[i0][0], dy = P0[c][1] - P0[i0][1];
      T dd = dx * dx + dy * dy;
      if (i1 < 0 || dd > bd) { bd = dd; i1 = c; }
    }
    T ex = P0[i1][0] - P0[i0][0], ey = P0[i1][1] - P0[i0][1];
    int i2 = -1; T ba = T(0.f), a2 = T(0.f);
    for (int i = 0; i < nk; ++i) {
      int c = keep[i]; if (c == i0 || c == i1) continue;
      T ar = ex * (P0[c][1] - P0[i0][1]) - ey * (P0[c][0] - P0[i0][0]);
      if (i2 < 0 || abs_(ar) > ba) { ba = abs_(ar); i2 = c; a2 = ar; }
    }
    T flip = a2 >= T(0.f) ? T(-1.f) : T(1.f);
    int i3 = -1; T bv = T(0.f);
    for (int i = 0; i < nk; ++i) {
      int c = keep[i]; if (c == i0 || c == i1 || c == i2) continue;
      T ar = (ex * (P0[c][1] - P0[i0][1]) - ey * (P0[c][0] - P0[i0][0])) * flip;
      if (i3 < 0 || ar > bv) { bv = ar; i3 = c; }
    }
    sel[0] = i0; sel[1] = i1; sel[2] = i2; sel[3] = i3; ns = 4;
  }
  for (int i = 0; i < ns; ++i) {
    const T* P = P0[sel[i]];
    V3<T> pR = (fc + u * P[0]) + v * P[1];
    V3<T> pI = pR + nR * P[2];
    if (refA) { out[i].n = nR; out[i].pa = pR; out[i].pb = pI; }
    else { out[i].n = -nR; out[i].pa = pI; out[i].pb = pR; }
    out[i].s = P[2];
  }
  return ns;
}

// Pair dispatch; S1 is the dynamic body of lower index, S2 a body, a static
// box or the plane. Returns at most 4 points with s < off.
template <class T> __device__ int collide(const Shape<T>& S1, const Shape<T>& S2, T off, Pt<T>* out) {
  int n = 0;
  if (S2.type == SH_PLANE) {
    if (S1.type == SH_SPHERE) n = sphere_plane(S1.c, S1.d0, out);
    else if (S1.type == SH_CAPSULE) n = capsule_plane(S1, off, out);
    else n = box_plane(S1, off, out);
  } else {
    bool swp = S1.type > S2.type;
    const Shape<T>& P = swp ? S2 : S1;
    const Shape<T>& Q = swp ? S1 : S2;
    if (P.type == SH_SPHERE) {
      if (Q.type == SH_SPHERE) n = sphere_sphere(P.c, P.d0, Q.c, Q.d0, out);
      else if (Q.type == SH_CAPSULE) n = sphere_capsule(P.c, P.d0, Q, out);
      else n = sphere_box(P.c, P.d0, Q, out);
    } else if (P.type == SH_CAPSULE) {
      if (Q.type == SH_CAPSULE) n = capsule_capsule(P, Q, out);
      else n = capsule_box(P, Q, off, out);
    } else {
      n = box_box(P, Q, off, out);
    }
    if (swp) {
      for (int i = 0; i < n; ++i) {
        out[i].n = -out[i].n;
        V3<T> t = out[i].pa; out[i].pa = out[i].pb; out[i].pb = t;
      }
    }
  }
  int m = 0;
  for (int i = 0; i < n; ++i) if (out[i].s < off) out[m++] = out[i];
  return m;
}

}  // namespace msh
