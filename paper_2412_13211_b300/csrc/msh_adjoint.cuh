// Adjoint of one recorded step (reverse mode), per env.
//
// Given the adjoint of the state after a recorded step, computes the adjoint
// of the state before it, of that step's joint targets and (accumulated) of
// the body masses. The step is differentiated as the forward computes it,
// with its discrete decisions frozen: the contact set and features found by
// the narrowphase, the colouring, and every clamp of the projected
// Gauss-Seidel sweeps.
//   * integration: hand-written reverse of x += h v and of the normalised
//     quaternion update;
//   * mass-split Jacobi: per sweep, the iteration-start velocities from the
//     recorded lambdas, every constraint's rows reversed on its local copies,
//     and the copies' adjoints summed per body in constraint order;
//   * coloured PGS: the sweeps run backwards (iterations, then colours in
//     reverse order, rows of a constraint in reverse order); velocities before
//     each update are rebuilt from the velocities after it and the recorded
//     lambdas (v_before = v_after - M^-1 J^T (lambda_after - lambda_before));
//     clamp states come from the recorded lambdas. Joint rows are stored whole
//     (Jacobians, inertia products, mass, bias, softness). A contact point
//     keeps its normal, world lever arms, bias, three effective masses, the
//     tangent-basis scale and the three couplings of its rows, and is reversed
//     as the forward updates it: its impulse once, then the scalar chain of
//     its three rows through the couplings; its adjoint accumulators are those
//     of the normal, tangents, arms, masses, bias, carried lambdas and
//     couplings, with the inverse-inertia and inverse-mass adjoints kept per
//     manifold;
//   * row set-up (lever arms, Jacobians, biases, drives): hand-written
//     reverses of the joint and contact row geometry; the narrowphase: local
//     Jacobians by single-tangent dual numbers, one input direction at a
//     time, contracted with the contact adjoints;
//   * effective masses, couplings and world inverse inertias: hand-written
//     reverse.
// Per-body sums are gathered in constraint order, so results are
// deterministic (checkpointed and plain backward passes agree bitwise).
#pragma once
#include "msh_stages.cuh"

namespace msh {

#define CLAMP_FRIC (-3.f)

// Per-env adjoint workspace (HBM), byte offsets.
struct AdjLayout {
  int Rm, Km;
  int bx, bq, bv, bw, bI0, bI1, bm;   // per body: x, q, v, w adjoints; Iw adjoint (6) + 1/m adjoint; mass accum
  int rows, radj;                     // per joint row: 5 float4 params, 5 float4 adjoints
  int cpar, cadj;                     // per contact point: CPAR_F4 float4 params, CADJ_F4 float4 adjoints
  int madj;                           // per manifold: 4 float4 (gIw_a, gIw_b, g(1/m_a), g(1/m_b))
  int cpose;                          // per contact point: 16 floats, its pose adjoints in gather-slot order
  int moff;                           // per manifold + 1: first dual-pass item of the narrowphase reverse
  int mord;                           // per manifold: the manifolds sorted by narrowphase routine
  int gat;                            // per constraint: 8 float4 (xa, qa, xb, qb, Iwa0, Iwa1|ima, Iwb0, Iwb1|imb)
  int cg;                             // per contact point: 3 float4 (n, ra, rb adjoints)
  int inc_off, inc, tg, bytes;
};

struct AdjParams {
  AdjLayout A;
  char* aws;             // per-env adjoint workspace slabs
  long long aws_stride;
  int slot;              // tape slot being reversed
  const float* ax; const float* aq; const float* av; const float* aw;   // adjoint of the state after the step
  float* ox; float* oq; float* ov; float* ow;                           // adjoint of the state before the step
  float* otg;            // [E, max_dof] adjoint of this step's targets
  float* omass;          // [B] accumulated mass adjoint
};

// float4s per contact point: parameters (n|m_n, ra|bias, rb|m_t1, m_t2|onb
// scale|K(t1,n)|K(t2,n), K(t2,t1)) and adjoint accumulators (d|m x3, ra|bias,
// rb|lambda_n, lambda_t1|lambda_t2|K(t1,n)|K(t2,n), K(t2,t1)).
enum { CPAR_F4 = 5, CADJ_F4 = 7 };

struct AWs {
  float4 *bx, *bq, *bv, *bw, *bI0, *bI1, *bm;
  float4 *rows, *radj;
  float4 *cpar, *cadj, *madj;
  float* cpose;
  int* moff;
  int* mord;
  float4* gat;
  float4* cg;
  int *inc_off, *inc;
  float* tg;
};

__device__ __forceinline__ AWs make_aws(char* b, const AdjLayout& A) {
  AWs a;
  a.bx = (float4*)(b + A.bx); a.bq = (float4*)(b + A.bq); a.bv = (float4*)(b + A.bv); a.bw = (float4*)(b + A.bw);
  a.bI0 = (float4*)(b + A.bI0); a.bI1 = (float4*)(b + A.bI1); a.bm = (float4*)(b + A.bm);
  a.rows = (float4*)(b + A.rows); a.radj = (float4*)(b + A.radj);
  a.cpar = (float4*)(b + A.cpar); a.cadj = (float4*)(b + A.cadj); a.madj = (float4*)(b + A.madj);
  a.cpose = (float*)(b + A.cpose);
  a.moff = (int*)(b + A.moff); a.mord = (int*)(b + A.mord);
  a.gat = (float4*)(b + A.gat); a.cg = (float4*)(b + A.cg);
  a.inc_off = (int*)(b + A.inc_off); a.inc = (int*)(b + A.inc); a.tg = (float*)(b + A.tg);
  return a;
}

__device__ __forceinline__ void add4(float4& a, const V3<float>& v) { a.x += v.x; a.y += v.y; a.z += v.z; }
__device__ __forceinline__ V3<float> sym_outer_diag(const V3<float>& g, const V3<float>& a) { return v3<float>(g.x * a.x, g.y * a.y, g.z * a.z); }

// Row index of joint k row r, or of contact point c row i (the recorded
// lambdas of a step use this numbering).
__device__ __forceinline__ int jrow(int k, int r) { return k * ROWS_PER_JOINT + r; }
__device__ __forceinline__ int crow(const Layout& L, int c, int i) { return ROWS_PER_JOINT * L.Jm + 4 * c + i; }

// Adds the symmetric outer product g a^T + a g^T (diagonal once) of an
// inverse-inertia adjoint, in the entry order xx xy xz yy yz zz.
__device__ __forceinline__ void add_sym(float* G, const V3<float>& g, const V3<float>& a) {
  G[0] += g.x * a.x; G[1] += g.x * a.y + g.y * a.x; G[2] += g.x * a.z + g.z * a.x;
  G[3] += g.y * a.y; G[4] += g.y * a.z + g.z * a.y; G[5] += g.z * a.z;
}

// ---------------------------------------------------------------------------
// replay helpers
// ---------------------------------------------------------------------------
// Loads the recorded step-start state into the workspace (as stage_load does
// from the state arrays) and the joints' row information.
static __device__ void load_from_tape(const Params& p, const EnvInfo& e, const Ws& w, const float* tape) {
  for (int i = e.lane; i < e.D; i += e.nthr) {
    const float* t = tape + 13 * i;
    float4 inv = p.binv[e.b0 + i];
    w.bx[i] = make_float4(t[0], t[1], t[2], inv.x);
    w.bq[i] = make_float4(t[3], t[4], t[5], t[6]);
    w.bv[i] = make_float4(t[7], t[8], t[9], 0.f);
    w.bw[i] = make_float4(t[10], t[11], t[12], 0.f);
    w.bIw1[i] = make_float4(0.f, 0.f, 1.f, 0.f);
  }
  load_jinfo(p, e, w);
}

// World inverse inertia from an orientation and principal inverse inertia.
template <class T> __device__ __forceinline__ void world_inv_inertia(const Q4<T>& q, const T* d, T* W6) {
  M3<T> R = qmat(q);
  T W[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      W[a][b] = R.m[a][0] * d[0] * R.m[b][0] + R.m[a][1] * d[1] * R.m[b][1] + R.m[a][2] * d[2] * R.m[b][2];
  W6[0] = W[0][0]; W6[1] = W[0][1]; W6[2] = W[0][2]; W6[3] = W[1][1]; W6[4] = W[1][2]; W6[5] = W[2][2];
}

// Constraint -> body incidence lists in constraint order (for deterministic gathers).
static __device__ void build_incidence(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a) {
  if (e.lane == 0) {
    const int K = e.J + w.misc[MC_MANIFOLDS];
    for (int i = 0; i <= e.D; ++i) a.inc_off[i] = 0;
    for (int k = 0; k < K; ++k) {
      int x, y;
      con_bodies(p, e, w, k, e.J, x, y);
      if (x >= 0) a.inc_off[x + 1]++;
      if (y >= 0) a.inc_off[y + 1]++;
    }
    for (int i = 0; i < e.D; ++i) a.inc_off[i + 1] += a.inc_off[i];
    for (int i = 0; i < e.D; ++i) w.masks[i] = (unsigned long long)a.inc_off[i];
    for (int k = 0; k < K; ++k) {
      int x, y;
      con_bodies(p, e, w, k, e.J, x, y);
      if (x >= 0) a.inc[w.masks[x]++] = 2 * k;
      if (y >= 0) a.inc[w.masks[y]++] = 2 * k + 1;
    }
  }
  gsync(e);
}

// One contact point's parameters for the reverse sweeps (BK: the kind of b;
// a static b's terms drop out at compile time, the same values).
template <int BK>
__device__ __forceinline__ void contact_rev_rows(const Params& p, const Ws& w, const AWs& a, int ci, int ia, int ibd) {
  const int ib = BK == BK_STATIC ? -1 : ibd;
  const bool bdyn = b_dyn<BK>(ib >= 0);
  RowCtx ctx = row_ctx(w, ia, ib);
  V3<float> n = f3(w.cn[ci]);
  V3<float> ra, rb;
  float bias;
  V3<float> xb = bdyn ? f3(w.bx[ib]) : v3<float>(0.f, 0.f, 0.f);
  Q4<float> qb = bdyn ? ldq4(w.bq[ib]) : ldq4(make_float4(1.f, 0.f, 0.f, 0.f));
  contact_geom<float>(f3(w.bx[ia]), ldq4(w.bq[ia]), xb, qb, bdyn, n, f3(w.cra[ci]), f3(w.crb[ci]), p.h, p.beta,
                      p.slop, ra, rb, bias);
  V3<float> t1, t2;
  const float sc = onb_scale(n);
  onb_with(n, sc, t1, t2);
  V3<float> dirs[3] = {n, t1, t2};
  float m[3];
  for (int r = 0; r < 3; ++r) {
    JRow x = blank_row();
    x.la = -dirs[r]; x.lb = dirs[r]; x.aa = -cross(ra, dirs[r]); x.ab = cross(rb, dirs[r]);
    finish_row(x, ctx, false);
    m[r] = x.m;
  }
  float K[6];
  point_K(ctx, dirs, ra, rb, K);   // the couplings the forward sweeps use
  float4* P = a.cpar + CPAR_F4 * ci;
  P[0] = f4(n, m[0]); P[1] = f4(ra, bias); P[2] = f4(rb, m[1]); P[3] = make_float4(m[2], sc, K[3], K[4]);
  P[4] = make_float4(K[5], 0.f, 0.f, 0.f);
  float4* G = a.cadj + CADJ_F4 * ci;
  for (int q = 0; q < CADJ_F4; ++q) G[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Generic rows of every constraint at the workspace poses (for the reverse
// sweeps): la|m, aa|bias, ab|gamma, Ia|0, Ib|clamp, plus a kind code.
static __device__ void build_rows(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a, const float* tg) {
  const int nc = w.misc[MC_CONTACTS];
  for (int t = e.lane; t < e.J + nc; t += e.nthr) {
    if (t < e.J) {
      const JointDesc& j = p.joints[e.j0 + t];
      const int A = j.parent, B = j.child;
      RowCtx ctx = row_ctx(w, A, B);
      float tgl[3] = {0.f, 0.f, 0.f};
      if (j.k > 0.f || j.d > 0.f)
        for (int c = 0; c < joint_ndof(j.type); ++c) tgl[c] = tg[j.dof + c];
      V3<float> xa = A >= 0 ? f3(w.bx[A]) : v3<float>(0.f, 0.f, 0.f);
      Q4<float> qa = A >= 0 ? ldq4(w.bq[A]) : ldq4(make_float4(1.f, 0.f, 0.f, 0.f));
      GRow<float> g[ROWS_PER_JOINT];
      int n = joint_geom<float>(j, A >= 0, xa, qa, f3(w.bx[B]), ldq4(w.bq[B]), tgl, p.h, p.jbeta, g);
      for (int r = 0; r < n; ++r) {
        JRow x = blank_row();
        x.la = g[r].la; x.lb = -g[r].la; x.aa = g[r].aa; x.ab = g[r].ab;
        x.bias = g[r].bias; x.gamma = g[r].gamma;
        const bool soft = g[r].clamp >= 0.f;
        finish_row(x, ctx, soft);
        float4* R = a.rows + ROW_F4 * jrow(t, r);
        R[0] = f4(x.la, x.m); R[1] = f4(x.aa, x.bias); R[2] = f4(x.ab, x.gamma);
        R[3] = f4(x.Ia, 0.f); R[4] = f4(x.Ib, g[r].clamp);
        float4* G = a.radj + ROW_F4 * jrow(t, r);
        for (int q = 0; q < ROW_F4; ++q) G[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
      const int ci = t - e.J;
      const int ids = w.cid[ci];
      const int ia = ids & 0xffff, bc = ids >> 16;
      const int ib = bc < e.D ? bc : -1;
      by_b_kind(ib >= 0, [&](auto k) { contact_rev_rows<decltype(k)::v>(p, w, a, ci, ia, ib); });
    }
  }
  const int M = w.misc[MC_MANIFOLDS];
  for (int m = e.lane; m < 4 * M; m += e.nthr) a.madj[m] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// reverse of the projected Gauss-Seidel sweeps
// ---------------------------------------------------------------------------
struct BodyAdj { V3<float> va, wa, vb, wb; };

// The loaded state of one row for its reverse update: parameters, adjoint
// accumulators and its recorded lambdas.
struct RevRow {
  float4 r0, r1, r2, r3, r4;   // la|m, aa|bias, ab|gamma, Ia|-, Ib|clamp
  float4 g0, g1, g2, g3, g4;   // adjoints (gla|gm, gaa|gbias, gab|glam, gIa|g(1/m_a), gIb|g(1/m_b))
  float lam_after, lam_before, lam_n_after;
};

__device__ __forceinline__ void load_rev_row(const AWs& a, int r, const float* lam_it, const float* lam_prev, int nrow,
                                             RevRow& x) {
  const float4* R = a.rows + ROW_F4 * r;
  const float4* G = a.radj + ROW_F4 * r;
  x.r0 = R[0]; x.r1 = R[1]; x.r2 = R[2]; x.r3 = R[3]; x.r4 = R[4];
  x.g0 = G[0]; x.g1 = G[1]; x.g2 = G[2]; x.g3 = G[3]; x.g4 = G[4];
  x.lam_after = lam_it[r];
  x.lam_before = lam_prev ? lam_prev[r] : 0.f;
  x.lam_n_after = nrow >= 0 ? lam_it[nrow] : 0.f;
}

// Reverse of one row update on the loaded row `x` (writes its adjoints back
// to row r). `gfric` receives the adjoint this row (a friction row at its
// limit) sends to its normal row's lambda; the caller adds it when it
// reaches that row. JAC (mass-split Jacobi): the update moves the
// constraint's local velocity copies through the split inverse masses (sa,
// sb times the true ones) and adds the true-mass change to the bodies'
// iteration sums, whose adjoint is G; v and g are the local copies and
// their adjoints.
template <bool JAC>
__device__ __forceinline__ void reverse_row(const AWs& a, int r, int A, int B, float ima, float imb, BodyVel& v,
                                            BodyAdj& g, const RevRow& x, float mu, float& gfric, float sa = 1.f,
                                            float sb = 1.f, const BodyAdj* GS = nullptr) {
  V3<float> la = f3(x.r0), aa = f3(x.r1), ab = f3(x.r2), Ia = f3(x.r3), Ib = f3(x.r4);
  const float m = x.r0.w, bias = x.r1.w, gamma = x.r2.w, clamp = x.r4.w;
  const float lam_after = x.lam_after, lam_before = x.lam_before;
  const float D = lam_after - lam_before;
  // velocities before the update
  if (JAC) {
    if (A >= 0) { v.va = v.va - la * ((sa * ima) * D); v.wa = v.wa - Ia * (sa * D); }
    if (B >= 0) { v.vb = v.vb + la * ((sb * imb) * D); v.wb = v.wb - Ib * (sb * D); }
  } else {
    if (A >= 0) { v.va = v.va - la * (ima * D); v.wa = v.wa - Ia * D; }
    if (B >= 0) { v.vb = v.vb + la * (imb * D); v.wb = v.wb - Ib * D; }
  }
  V3<float> gla = f3(x.g0), gaa = f3(x.g1), gab = f3(x.g2), gIa = f3(x.g3), gIb = f3(x.g4);
  float gm = x.g0.w, gbias = x.g1.w, glam = x.g2.w, gima = x.g3.w, gimb = x.g4.w;
  // adjoint of D through the velocity update
  float gD = 0.f;
  if (JAC) {
    if (A >= 0) {
      const float lva = dot(la, g.va), LVa = dot(la, GS->va);
      gD += (sa * ima) * lva + sa * dot(Ia, g.wa) + ima * LVa + dot(Ia, GS->wa);
      gla = gla + (g.va * (sa * ima) + GS->va * ima) * D;
      gIa = gIa + (g.wa * sa + GS->wa) * D;
      gima += (sa * lva + LVa) * D;
    }
    if (B >= 0) {
      const float lvb = dot(la, g.vb), LVb = dot(la, GS->vb);
      gD += -(sb * imb) * lvb + sb * dot(Ib, g.wb) - imb * LVb + dot(Ib, GS->wb);
      gla = gla - (g.vb * (sb * imb) + GS->vb * imb) * D;
      gIb = gIb + (g.wb * sb + GS->wb) * D;
      gimb += -(sb * lvb + LVb) * D;
    }
  } else {
    if (A >= 0) {
      gD += ima * dot(la, g.va) + dot(Ia, g.wa);
      gla = gla + g.va * (ima * D);
      gIa = gIa + g.wa * D;
      gima += dot(la, g.va) * D;        // adjoint of 1/m_a (kept in the row, moved to the body later)
    }
    if (B >= 0) {
      gD += -imb * dot(la, g.vb) + dot(Ib, g.wb);
      gla = gla - g.vb * (imb * D);
      gIb = gIb + g.wb * D;
      gimb += -dot(la, g.vb) * D;       // adjoint of 1/m_b
    }
  }
  const float a_after = glam + gD;
  float glam_before = -gD;
  // pre-clamp value
  float jv = 0.f;
  if (B >= 0) jv = dotf(ab, v.wb) - dotf(la, v.vb);
  if (A >= 0) jv = jv + dotf(la, v.va) + dotf(aa, v.wa);
  const float u = jv + bias + gamma * lam_before;
  // the clamp state as selects (the lanes of a warp reverse rows of
  // different clamp kinds at the same time)
  const float lim = clamp >= 0.f ? clamp : (clamp == CLAMP_FRIC ? mu * x.lam_n_after : 0.f);
  const bool bounded = clamp >= 0.f || clamp == CLAMP_FRIC || clamp == CLAMP_UNI;
  const bool clamped = bounded && (lam_after == lim || lam_after == -lim);
  const float fric_sign = lam_after == lim ? 1.f : -1.f;
  float gpre = clamped ? 0.f : a_after;
  gfric = clamped && clamp == CLAMP_FRIC ? fric_sign * mu * a_after : 0.f;
  glam_before += gpre;
  const float gu = -m * gpre;
  gm += -u * gpre;
  if (A >= 0) { g.va = g.va + la * gu; g.wa = g.wa + aa * gu; gaa = gaa + v.wa * gu; }
  if (B >= 0) { g.vb = g.vb - la * gu; g.wb = g.wb + ab * gu; gab = gab + v.wb * gu; }
  gla = gla + (v.va - v.vb) * gu;
  gbias += gu;
  glam_before += gamma * gu;
  float4* G = a.radj + ROW_F4 * r;
  G[0] = f4(gla, gm); G[1] = f4(gaa, gbias); G[2] = f4(gab, glam_before); G[3] = f4(gIa, gima); G[4] = f4(gIb, gimb);
}

// Reverse of contact point ci's update in a sweep. The forward forms the
// velocity of b relative to a at the point, vr = (vb + wb x rb) - (va + wa x
// ra), its components u = d.vr along d in (n, t1, t2), updates lambda_n, then
// lambda_t1, lambda_t2, each later row's u moved by the earlier rows' impulse
// changes D through the couplings K(t1,n), K(t2,n), K(t2,t1), and applies the
// point's impulse P = sum_d d D once (-P on a, +P on b, through 1/m and the
// world inverse inertias). This undoes it: the velocities before the point,
// then the adjoints of the velocities, of lambda before the update, of d, ra,
// rb, the masses, the bias and the couplings (accumulated per point for the
// set-up reverse), and of the manifold's inverse inertias and inverse masses
// `mi` (gIw_a[6], gIw_b[6], g(1/m_a), g(1/m_b)). A friction row at its limit
// mu * lambda_n sends its adjoint to lambda_n.
// JAC: as in reverse_row, the local velocity copies move through the split
// inverse masses and the bodies' iteration sums (adjoint G) through the true
// ones. BK: the kind of b (`bd`: b is dynamic, read with BK_EITHER; a static
// b's terms drop out at compile time; the same values).
template <bool JAC, int BK>
__device__ __forceinline__ void reverse_point(const AWs& a, int ci, int rn, bool bd, float ima, float imb,
                                              const Sym3& Iwa, const Sym3& Iwb, BodyVel& v, BodyAdj& g,
                                              const float* lam_it, const float* lam_prev, float mu, float* mi,
                                              float sa = 1.f, float sb = 1.f, const BodyAdj* GS = nullptr) {
  const bool bdyn = b_dyn<BK>(bd);
  const float4* P = a.cpar + CPAR_F4 * ci;
  float4* Q = a.cadj + CADJ_F4 * ci;
  const float4 P0 = P[0], P1 = P[1], P2 = P[2], P3 = P[3], P4 = P[4];
  const float4 Q0 = Q[0], Q1 = Q[1], Q2 = Q[2], Q3 = Q[3], Q4 = Q[4], Q5 = Q[5], Q6 = Q[6];
  const V3<float> n = f3(P0), ra = f3(P1), rb = f3(P2);
  const float m0 = P0.w, m1 = P2.w, m2 = P3.x, bias = P1.w;
  const float K10 = P3.z, K20 = P3.w, K21 = P4.x;
  V3<float> t1, t2;
  onb_with(n, P3.y, t1, t2);
  V3<float> gd0 = f3(Q0), gd1 = f3(Q1), gd2 = f3(Q2);
  float gm0 = Q0.w, gm1 = Q1.w, gm2 = Q2.w;
  V3<float> gra = f3(Q3), grb = f3(Q4);
  float gbias = Q3.w;
  float gl0 = Q4.w, gl1 = Q5.x, gl2 = Q5.y;
  float gK10 = Q5.z, gK20 = Q5.w, gK21 = Q6.x;
  // a point's three lambdas start a 16-byte slot of the sweep's record
  const float4 LA = *reinterpret_cast<const float4*>(lam_it + rn);
  const float4 LB = lam_prev ? *reinterpret_cast<const float4*>(lam_prev + rn) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float la0 = LA.x, la1 = LA.y, la2 = LA.z;
  const float lb0 = LB.x, lb1 = LB.y, lb2 = LB.z;
  const float D0 = la0 - lb0, D1 = la1 - lb1, D2 = la2 - lb2;
  // the point's impulse and the velocities before the point
  const V3<float> Pi = (n * D0 + t1 * D1) + t2 * D2;
  const V3<float> ta = cross(ra, Pi);
  V3<float> tb = v3<float>(0.f, 0.f, 0.f);
  V3<float> gP;
  if (JAC) {
    v.va = v.va + Pi * (sa * ima);
    v.wa = v.wa + smul(Iwa, ta) * sa;
    if (bdyn) {
      tb = cross(rb, Pi);
      v.vb = v.vb - Pi * (sb * imb);
      v.wb = v.wb - smul(Iwb, tb) * sb;
    }
    // adjoint of the impulse's application to the local copies and the sums
    const V3<float> ewa = g.wa * sa + GS->wa;
    const V3<float> sI = smul(Iwa, ewa);
    gP = (g.va * (sa * ima) + GS->va * ima) * (-1.f) + cross(ra, sI);
    gra = gra + cross(sI, Pi);
    add_sym(mi, ewa, -ta);
    mi[12] -= dot(Pi, g.va * sa + GS->va);
    if (bdyn) {
      const V3<float> ewb = g.wb * sb + GS->wb;
      const V3<float> sJ = smul(Iwb, ewb);
      gP = gP + (g.vb * (sb * imb) + GS->vb * imb) + cross(sJ, rb);
      grb = grb + cross(Pi, sJ);
      add_sym(mi + 6, ewb, tb);
      mi[13] += dot(Pi, g.vb * sb + GS->vb);
    }
  } else {
    v.va = v.va + Pi * ima;
    v.wa = v.wa + smul(Iwa, ta);
    if (bdyn) {
      tb = cross(rb, Pi);
      v.vb = v.vb - Pi * imb;
      v.wb = v.wb - smul(Iwb, tb);
    }
    // adjoint of the impulse's application
    const V3<float> sI = smul(Iwa, g.wa);
    gP = g.va * (-ima) + cross(ra, sI);
    gra = gra + cross(sI, Pi);
    add_sym(mi, g.wa, -ta);
    mi[12] -= dot(Pi, g.va);
    if (bdyn) {
      const V3<float> sJ = smul(Iwb, g.wb);
      gP = gP + g.vb * imb + cross(sJ, rb);
      grb = grb + cross(Pi, sJ);
      add_sym(mi + 6, g.wb, tb);
      mi[13] += dot(Pi, g.vb);
    }
  }
  float gD0 = dot(n, gP), gD1 = dot(t1, gP), gD2 = dot(t2, gP);
  gd0 = gd0 + gP * D0; gd1 = gd1 + gP * D1; gd2 = gd2 + gP * D2;
  // the rows' inputs as the forward formed them
  V3<float> vr = v3<float>(0.f, 0.f, 0.f) - (v.va + cross(v.wa, ra));
  if (bdyn) vr = vr + (v.vb + cross(v.wb, rb));
  const float u0 = dot(n, vr);
  const float u1 = dot(t1, vr) + K10 * D0;
  const float u2 = (dot(t2, vr) + K20 * D0) + K21 * D1;
  const float lim = mu * la0;
  float pend = 0.f;
  // friction t2
  const float a2 = gl2 + gD2;
  const bool c2 = la2 == lim || la2 == -lim;
  if (c2) pend += (la2 == lim ? 1.f : -1.f) * mu * a2;
  const float gp2 = c2 ? 0.f : a2;
  gl2 = gp2 - gD2;
  gm2 += -u2 * gp2;
  const float gu2 = -m2 * gp2;
  gK21 += D1 * gu2;
  gD1 += K21 * gu2;
  // friction t1
  const float a1 = gl1 + gD1;
  const bool c1 = la1 == lim || la1 == -lim;
  if (c1) pend += (la1 == lim ? 1.f : -1.f) * mu * a1;
  const float gp1 = c1 ? 0.f : a1;
  gl1 = gp1 - gD1;
  gm1 += -u1 * gp1;
  const float gu1 = -m1 * gp1;
  gK10 += D0 * gu1;
  gK20 += D0 * gu2;
  gD0 += K10 * gu1 + K20 * gu2;
  // normal
  gl0 += pend;
  const float a0 = gl0 + gD0;
  const float gp0 = la0 == 0.f ? 0.f : a0;
  gl0 = gp0 - gD0;
  gm0 += -(u0 + bias) * gp0;
  const float gu0 = -m0 * gp0;
  gbias += gu0;
  // u = d.vr
  const V3<float> gvr = (n * gu0 + t1 * gu1) + t2 * gu2;
  gd0 = gd0 + vr * gu0; gd1 = gd1 + vr * gu1; gd2 = gd2 + vr * gu2;
  g.va = g.va - gvr;
  g.wa = g.wa - cross(ra, gvr);
  gra = gra - cross(gvr, v.wa);
  if (bdyn) {
    g.vb = g.vb + gvr;
    g.wb = g.wb + cross(rb, gvr);
    grb = grb + cross(gvr, v.wb);
  }
  Q[0] = f4(gd0, gm0); Q[1] = f4(gd1, gm1); Q[2] = f4(gd2, gm2);
  Q[3] = f4(gra, gbias); Q[4] = f4(grb, gl0); Q[5] = make_float4(gl1, gl2, gK10, gK20);
  Q[6] = make_float4(gK21, 0.f, 0.f, 0.f);
}

// Reverse of one joint's update in a sweep: its rows in reverse order.
__device__ __forceinline__ void reverse_joint(const Params& p, const Ws& w, const AWs& a, int k,
                                              const float* lam_it, const float* lam_prev) {
  const int4 ji = w.jinfo[k];
  const int A = ji.x, B = ji.y;
  BodyVel v = load_vel(w, A, B);
  BodyAdj g;
  V3<float> z = v3<float>(0.f, 0.f, 0.f);
  g.va = A >= 0 ? f3(a.bv[A]) : z; g.wa = A >= 0 ? f3(a.bw[A]) : z;
  g.vb = f3(a.bv[B]); g.wb = f3(a.bw[B]);
  const float ima = A >= 0 ? w.bx[A].w : 0.f, imb = w.bx[B].w;
  const int jnr = ji.w;
  // software pipelining: the next row's parameters, adjoints and lambdas
  // load while this row runs (rows of a constraint never alias)
  int r_cur = jrow(k, jnr - 1);
  RevRow cur, nxt;
  load_rev_row(a, r_cur, lam_it, lam_prev, -1, cur);
  for (int i = 0; i < jnr; ++i) {
    const int r_nxt = jrow(k, jnr - 2 - i);
    if (i + 1 < jnr) load_rev_row(a, r_nxt, lam_it, lam_prev, -1, nxt);
    float gfric;
    reverse_row<false>(a, r_cur, A, B, ima, imb, v, g, cur, 0.f, gfric);
    if (i + 1 < jnr) { cur = nxt; r_cur = r_nxt; }
  }
  if (A >= 0) { w.bv[A] = f4(v.va, 0.f); w.bw[A] = f4(v.wa, 0.f); a.bv[A] = f4(g.va, 0.f); a.bw[A] = f4(g.wa, 0.f); }
  w.bv[B] = f4(v.vb, 0.f); w.bw[B] = f4(v.wb, 0.f); a.bv[B] = f4(g.vb, 0.f); a.bw[B] = f4(g.wb, 0.f);
}

// Reverse of manifold m's update in a sweep: its points in reverse order.
// BK: the kind of b; a static b (nearly every manifold of the apartment
// batch) has no velocity or adjoint to load or store, and with BK_STATIC its
// terms drop out of the point reverse at compile time (the same values).
template <int BK>
__device__ __forceinline__ void reverse_manifold(const Params& p, const Ws& w, const AWs& a, int m, int4 mf,
                                                 const float* lam_it, const float* lam_prev) {
  const int A = mf.x, B = BK == BK_STATIC ? -1 : mf.y;
  const bool bdyn = b_dyn<BK>(B >= 0);
  const V3<float> z = v3<float>(0.f, 0.f, 0.f);
  BodyVel v;
  v.va = f3(w.bv[A]); v.wa = f3(w.bw[A]);
  v.vb = bdyn ? f3(w.bv[B]) : z; v.wb = bdyn ? f3(w.bw[B]) : z;
  BodyAdj g;
  g.va = f3(a.bv[A]); g.wa = f3(a.bw[A]);
  g.vb = bdyn ? f3(a.bv[B]) : z; g.wb = bdyn ? f3(a.bw[B]) : z;
  const float ima = w.bx[A].w, imb = bdyn ? w.bx[B].w : 0.f;
  const Sym3 Iwa = load_Iw(w, A);
  const Sym3 Iwb = bdyn ? load_Iw(w, B) : Iwa;
  float4* MA = a.madj + 4 * m;
  float4 m0 = MA[0], m1 = MA[1], m2 = MA[2], m3 = MA[3];
  float mi[14] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x, m2.y, m2.z, m2.w, m3.x, m3.y};
  for (int c = mf.z + mf.w - 1; c >= mf.z; --c)
    reverse_point<false, BK>(a, c, crow(p.L, c, 0), bdyn, ima, imb, Iwa, Iwb, v, g, lam_it, lam_prev, p.mu, mi);
  MA[0] = make_float4(mi[0], mi[1], mi[2], mi[3]); MA[1] = make_float4(mi[4], mi[5], mi[6], mi[7]);
  MA[2] = make_float4(mi[8], mi[9], mi[10], mi[11]); MA[3] = make_float4(mi[12], mi[13], 0.f, 0.f);
  w.bv[A] = f4(v.va, 0.f); w.bw[A] = f4(v.wa, 0.f); a.bv[A] = f4(g.va, 0.f); a.bw[A] = f4(g.wa, 0.f);
  if (bdyn) { w.bv[B] = f4(v.vb, 0.f); w.bw[B] = f4(v.wb, 0.f); a.bv[B] = f4(g.vb, 0.f); a.bw[B] = f4(g.wb, 0.f); }
}

// Reverse of one sweep: colours in reverse order; within a colour (its
// constraints share no dynamic body) the joints, then the manifolds.
static __device__ void reverse_sweep(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a, const float* lam_it,
                              const float* lam_prev) {
  const int J = e.J;
  const int ncol = w.misc[MC_COLOURS];
  for (int c = ncol - 1; c >= 0; --c) {
    const int v = w.coff[c], c0 = v & 0xffff, cm = c0 + (v >> 16), c1 = w.coff[c + 1] & 0xffff;
    for (int idx = c0 + e.lane; idx < cm; idx += e.nthr)
      reverse_joint(p, w, a, w.corder[idx], lam_it, lam_prev);
    for (int idx = cm + e.lane; idx < c1; idx += e.nthr) {
      const int m = w.corder[idx] - J;
      const int4 mf = man_get(w, m);
      by_b_kind(mf.y >= 0, [&](auto k) { reverse_manifold<decltype(k)::v>(p, w, a, m, mf, lam_it, lam_prev); });
    }
    gsync(e);
  }
}

// ---------------------------------------------------------------------------
// reverse of the mass-split Jacobi sweeps
// ---------------------------------------------------------------------------
// A Jacobi sweep: every constraint k copies the iteration-start velocities V
// of its bodies, updates its rows on the copies through the split inverse
// masses (the body's constraint count times the true ones), and adds its
// true-mass velocity change dV_k to the bodies' sums; then every body takes
// V + sum_k dV_k (constraint order). Reversed in three phases: dV_k from the
// recorded lambda changes and V = V' - sum_k dV_k; each constraint's rows in
// reverse on its copies (ending at V + split * dV_k) with the bodies'
// after-sweep adjoint G as the adjoint of the sums, leaving the adjoint of
// its copies at the start in the constraint's slot; then G + sum of the slots.
// The slots are the forward's per-constraint velocity-change array.

// True-mass velocity change of constraint k from its recorded lambda changes.
static __device__ void jacobi_dv(const Params& p, const Ws& w, const AWs& a, int k, int J, const float* lam_it,
                          const float* lam_prev) {
  V3<float> z = v3<float>(0.f, 0.f, 0.f);
  BodyVel d;
  d.va = z; d.wa = z; d.vb = z; d.wb = z;
  if (k < J) {
    const int4 ji = w.jinfo[k];
    const int A = ji.x;
    const float ima = A >= 0 ? w.bx[A].w : 0.f, imb = w.bx[ji.y].w;
    for (int r = 0; r < ji.w; ++r) {
      const int row = jrow(k, r);
      const float4* R = a.rows + ROW_F4 * row;
      const float D = lam_it[row] - (lam_prev ? lam_prev[row] : 0.f);
      const V3<float> la = f3(R[0]);
      if (A >= 0) { d.va = d.va + la * (ima * D); d.wa = d.wa + f3(R[3]) * D; }
      d.vb = d.vb - la * (imb * D);
      d.wb = d.wb + f3(R[4]) * D;
    }
  } else {
    const int4 mf = man_get(w, k - J);
    const int A = mf.x, B = mf.y;
    const float ima = w.bx[A].w, imb = B >= 0 ? w.bx[B].w : 0.f;
    const Sym3 Iwa = load_Iw(w, A);
    Sym3 Iwb = Iwa;
    if (B >= 0) Iwb = load_Iw(w, B);
    for (int c = mf.z; c < mf.z + mf.w; ++c) {
      const float4* P = a.cpar + CPAR_F4 * c;
      const V3<float> n = f3(P[0]), ra = f3(P[1]), rb = f3(P[2]);
      V3<float> t1, t2;
      onb_with(n, P[3].y, t1, t2);
      const int rn = crow(p.L, c, 0);
      const float D0 = lam_it[rn] - (lam_prev ? lam_prev[rn] : 0.f);
      const float D1 = lam_it[rn + 1] - (lam_prev ? lam_prev[rn + 1] : 0.f);
      const float D2 = lam_it[rn + 2] - (lam_prev ? lam_prev[rn + 2] : 0.f);
      const V3<float> Pi = (n * D0 + t1 * D1) + t2 * D2;
      d.va = d.va - Pi * ima;
      d.wa = d.wa - smul(Iwa, cross(ra, Pi));
      if (B >= 0) { d.vb = d.vb + Pi * imb; d.wb = d.wb + smul(Iwb, cross(rb, Pi)); }
    }
  }
  w.jdv[4 * k + 0] = f4(d.va, 0.f); w.jdv[4 * k + 1] = f4(d.wa, 0.f);
  w.jdv[4 * k + 2] = f4(d.vb, 0.f); w.jdv[4 * k + 3] = f4(d.wb, 0.f);
}

// Phase 2 for constraint k: its reversed rows on its local copies.
template <bool JOINT>
static __device__ void reverse_constraint_jacobi(const Params& p, const Ws& w, const AWs& a, int k, int J,
                                          const float* lam_it, const float* lam_prev) {
  int A, B;
  if (JOINT) { const int4 ji = w.jinfo[k]; A = ji.x; B = ji.y; }
  else { const int4 mf = man_get(w, k - J); A = mf.x; B = mf.y; }
  const float sa = A >= 0 ? w.bIw1[A].z : 1.f, sb = B >= 0 ? w.bIw1[B].z : 1.f;
  // the copies after the constraint's rows: V + split * dV_k
  BodyVel v = load_vel(w, A, B);
  const V3<float> z = v3<float>(0.f, 0.f, 0.f);
  if (A >= 0) { v.va = v.va + f3(w.jdv[4 * k]) * sa; v.wa = v.wa + f3(w.jdv[4 * k + 1]) * sa; }
  if (B >= 0) { v.vb = v.vb + f3(w.jdv[4 * k + 2]) * sb; v.wb = v.wb + f3(w.jdv[4 * k + 3]) * sb; }
  BodyAdj G, g;
  G.va = A >= 0 ? f3(a.bv[A]) : z; G.wa = A >= 0 ? f3(a.bw[A]) : z;
  G.vb = B >= 0 ? f3(a.bv[B]) : z; G.wb = B >= 0 ? f3(a.bw[B]) : z;
  g.va = z; g.wa = z; g.vb = z; g.wb = z;
  const float ima = A >= 0 ? w.bx[A].w : 0.f, imb = B >= 0 ? w.bx[B].w : 0.f;
  if (JOINT) {
    const int jnr = w.jinfo[k].w;
    for (int i = jnr - 1; i >= 0; --i) {
      RevRow x;
      load_rev_row(a, jrow(k, i), lam_it, lam_prev, -1, x);
      float gfric;
      reverse_row<true>(a, jrow(k, i), A, B, ima, imb, v, g, x, 0.f, gfric, sa, sb, &G);
    }
  } else {
    const int4 mf = man_get(w, k - J);
    const Sym3 Iwa = load_Iw(w, A);
    Sym3 Iwb = Iwa;
    if (B >= 0) Iwb = load_Iw(w, B);
    float4* MA = a.madj + 4 * (k - J);
    float4 m0 = MA[0], m1 = MA[1], m2 = MA[2], m3 = MA[3];
    float mi[14] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x, m2.y, m2.z, m2.w, m3.x, m3.y};
    by_b_kind(B >= 0, [&](auto kb) {
      for (int c = mf.z + mf.w - 1; c >= mf.z; --c)
        reverse_point<true, decltype(kb)::v>(a, c, crow(p.L, c, 0), B >= 0, ima, imb, Iwa, Iwb, v, g, lam_it,
                                             lam_prev, p.mu, mi, sa, sb, &G);
    });
    MA[0] = make_float4(mi[0], mi[1], mi[2], mi[3]); MA[1] = make_float4(mi[4], mi[5], mi[6], mi[7]);
    MA[2] = make_float4(mi[8], mi[9], mi[10], mi[11]); MA[3] = make_float4(mi[12], mi[13], 0.f, 0.f);
  }
  w.jdv[4 * k + 0] = f4(g.va, 0.f); w.jdv[4 * k + 1] = f4(g.wa, 0.f);
  w.jdv[4 * k + 2] = f4(g.vb, 0.f); w.jdv[4 * k + 3] = f4(g.wb, 0.f);
}

static __device__ void reverse_sweep_jacobi(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a,
                                     const float* lam_it, const float* lam_prev) {
  const int J = e.J, K = J + w.misc[MC_MANIFOLDS];
  for (int k = e.lane; k < K; k += e.nthr) jacobi_dv(p, w, a, k, J, lam_it, lam_prev);
  gsync(e);
  // iteration-start velocities
  for (int i = e.lane; i < e.D; i += e.nthr) {
    V3<float> dv = v3<float>(0.f, 0.f, 0.f), dw = dv;
    for (int q = a.inc_off[i]; q < a.inc_off[i + 1]; ++q) {
      const int t = a.inc[q], k = t >> 1, side = t & 1;
      dv = dv + f3(w.jdv[4 * k + 2 * side]);
      dw = dw + f3(w.jdv[4 * k + 2 * side + 1]);
    }
    w.bv[i] = f4(f3(w.bv[i]) - dv, 0.f);
    w.bw[i] = f4(f3(w.bw[i]) - dw, 0.f);
  }
  gsync(e);
  for (int k = e.lane; k < K; k += e.nthr) {
    if (k < J) reverse_constraint_jacobi<true>(p, w, a, k, J, lam_it, lam_prev);
    else reverse_constraint_jacobi<false>(p, w, a, k, J, lam_it, lam_prev);
  }
  gsync(e);
  for (int i = e.lane; i < e.D; i += e.nthr) {
    V3<float> gv = f3(a.bv[i]), gw = f3(a.bw[i]);
    for (int q = a.inc_off[i]; q < a.inc_off[i + 1]; ++q) {
      const int t = a.inc[q], k = t >> 1, side = t & 1;
      gv = gv + f3(w.jdv[4 * k + 2 * side]);
      gw = gw + f3(w.jdv[4 * k + 2 * side + 1]);
    }
    a.bv[i] = f4(gv, 0.f);
    a.bw[i] = f4(gw, 0.f);
  }
  gsync(e);
}

// ---------------------------------------------------------------------------
// reverse of the row set-up
// ---------------------------------------------------------------------------
// Effective-mass and inertia terms of one row (K = ima la.la + aa.Ia + imb
// la.la + ab.Ib, Ia = Iw_a aa, Ib = Iw_b ab, m = 1/(K + gamma)): moves the
// adjoints of m, Ia, Ib and the row's 1/m adjoints onto la, aa, ab, the world
// inverse inertias (gIwa/gIwb, unique entries xx xy xz yy yz zz) and 1/m.
__device__ __forceinline__ void reverse_mass_part(const AWs& a, int r, int A, int B, float ima, float imb,
                                                  const Sym3& Iwa, const Sym3& Iwb, float* gIwa, float* gIwb,
                                                  float& gima, float& gimb, float sa, float sb) {
  float4* R = a.rows + ROW_F4 * r;
  float4* G = a.radj + ROW_F4 * r;
  V3<float> la = f3(R[0]), aa = f3(R[1]), ab = f3(R[2]), Ia = f3(R[3]), Ib = f3(R[4]);
  const float m = R[0].w;
  V3<float> gla = f3(G[0]), gaa = f3(G[1]), gab = f3(G[2]), gIa = f3(G[3]), gIb = f3(G[4]);
  const float gm = G[0].w;
  gima += G[3].w;
  gimb += G[4].w;
  const float gK = m > 0.f ? -m * m * gm : 0.f;
  const float ll = dot(la, la);
  // K = sa (ima la.la + aa.Ia) + sb (imb la.la + ab.Ib): sa, sb the Jacobi
  // mass splits (1 for coloured PGS)
  if (A >= 0) {
    const float gKa = gK * sa;
    gla = gla + la * (2.f * gKa * ima);
    gima += gKa * ll;
    gaa = gaa + Ia * gKa;
    gIa = gIa + aa * gKa;
    gaa = gaa + smul(Iwa, gIa);
    gIwa[0] += gIa.x * aa.x; gIwa[1] += gIa.x * aa.y + gIa.y * aa.x; gIwa[2] += gIa.x * aa.z + gIa.z * aa.x;
    gIwa[3] += gIa.y * aa.y; gIwa[4] += gIa.y * aa.z + gIa.z * aa.y; gIwa[5] += gIa.z * aa.z;
  }
  if (B >= 0) {
    const float gKb = gK * sb;
    gla = gla + la * (2.f * gKb * imb);
    gimb += gKb * ll;
    gab = gab + Ib * gKb;
    gIb = gIb + ab * gKb;
    gab = gab + smul(Iwb, gIb);
    gIwb[0] += gIb.x * ab.x; gIwb[1] += gIb.x * ab.y + gIb.y * ab.x; gIwb[2] += gIb.x * ab.z + gIb.z * ab.x;
    gIwb[3] += gIb.y * ab.y; gIwb[4] += gIb.y * ab.z + gIb.z * ab.y; gIwb[5] += gIb.z * ab.z;
  }
  G[0] = f4(gla, 0.f); G[1] = f4(gaa, G[1].w); G[2] = f4(gab, G[2].w);
}

// The mass part of a contact point's rows: K(x, y) = J_x M^-1 J_y^T = ima
// x.y + (ra x x).Iw_a (ra x y) [+ imb x.y + (rb x x).Iw_b (rb x y)] over x, y
// in (n, t1, t2). The diagonal enters through the effective masses m = 1/K,
// the off-diagonal (t1,n), (t2,n), (t2,t1) through the couplings of the
// sweeps; their adjoints move onto the directions, the arms, the inverse
// inertias and the inverse masses.
template <int BK>
__device__ __forceinline__ void contact_mass_adjoint(const AWs& a, int ci, bool bd, float ima, float imb,
                                                     const Sym3& Iwa, const Sym3& Iwb, float* gIwa, float* gIwb,
                                                     float& gima, float& gimb, float sa, float sb) {
  const bool bdyn = b_dyn<BK>(bd);
  const float4* P = a.cpar + CPAR_F4 * ci;
  float4* Q = a.cadj + CADJ_F4 * ci;
  const V3<float> n = f3(P[0]), ra = f3(P[1]), rb = f3(P[2]);
  const float ms[3] = {P[0].w, P[2].w, P[3].x};
  V3<float> t1, t2;
  onb_with(n, P[3].y, t1, t2);
  const V3<float> dirs[3] = {n, t1, t2};
  V3<float> gra = f3(Q[3]), grb = f3(Q[4]);
  V3<float> gd[3] = {f3(Q[0]), f3(Q[1]), f3(Q[2])};
  const float gKo[3] = {Q[5].z, Q[5].w, Q[6].x};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int i = q < 3 ? q : (q == 5 ? 2 : q - 2), j = q < 3 ? q : (q == 5 ? 1 : 0);
    float gK;
    if (q < 3) { const float m = ms[q]; gK = m > 0.f ? -m * m * Q[q].w : 0.f; }
    else gK = gKo[q - 3];
    const V3<float> x = dirs[i], y = dirs[j];
    const float xy = dot(x, y);
    // body a (its terms scaled by the Jacobi mass split sa; 1 for coloured PGS)
    {
      const float gKa = gK * sa;
      const V3<float> cx = cross(ra, x), cy = cross(ra, y);
      const V3<float> gcx = smul(Iwa, cy) * gKa, gcy = smul(Iwa, cx) * gKa;
      gd[i] = gd[i] + y * (gKa * ima) + cross(gcx, ra);
      gd[j] = gd[j] + x * (gKa * ima) + cross(gcy, ra);
      gima += gKa * xy;
      add_sym(gIwa, cx * gKa, cy);
      gra = gra + cross(x, gcx) + cross(y, gcy);
    }
    if (bdyn) {
      const float gKb = gK * sb;
      const V3<float> cx = cross(rb, x), cy = cross(rb, y);
      const V3<float> gcx = smul(Iwb, cy) * gKb, gcy = smul(Iwb, cx) * gKb;
      gd[i] = gd[i] + y * (gKb * imb) + cross(gcx, rb);
      gd[j] = gd[j] + x * (gKb * imb) + cross(gcy, rb);
      gimb += gKb * xy;
      add_sym(gIwb, cx * gKb, cy);
      grb = grb + cross(x, gcx) + cross(y, gcy);
    }
  }
  for (int q = 0; q < 3; ++q) Q[q] = f4(gd[q], 0.f);
  Q[3] = f4(gra, Q[3].w);
  Q[4] = f4(grb, Q[4].w);
}

__device__ __forceinline__ d1 tan_of(int idx, int k, float v) { return d1(v, idx == k ? 1.f : 0.f); }

// Adjoint of r = R(q) v (R the rotation matrix of the quaternion q = (w, u),
// as qmat forms it, R v = v + 2w (u x v) + 2 u x (u x v)) for the adjoint g of
// r: adds R^T g to gv and dr/dq^T g to gq (w, x, y, z).
__device__ __forceinline__ void rotate_adjoint(const float4& q4, const V3<float>& v, const V3<float>& g,
                                               V3<float>& gv, float* gq) {
  const V3<float> u = v3<float>(q4.y, q4.z, q4.w);
  const float w = q4.x;
  const M3<float> R = qmat(ldq4(q4));
  gv = gv + mulT(R, g);
  gq[0] += 2.f * dot(g, cross(u, v));
  const V3<float> gu = cross(v, g) * (2.f * w) + g * (2.f * dot(u, v)) + v * (2.f * dot(u, g)) - u * (4.f * dot(v, g));
  gq[1] += gu.x; gq[2] += gu.y; gq[3] += gu.z;
}

// Hand-written reverse of a joint's row geometry (joint_geom): from the
// adjoints of its rows' Jacobians and biases (the accumulators the reversed
// sweeps and the mass-part reverse left in radj) to the adjoints of the poses
// x_a (out 0-2), q_a (3-6), x_b (7-9), q_b (10-13) and of the joint's targets
// (14-16). Each step follows the branch its forward evaluation takes (the
// sign of q_r.w, the side of a limit's speculative bias). The forward, for
// reference: r_a = R(q_a) p_a, r_b = R(q_b) p_b, the world anchors x + r,
// dp = x_b + r_b - x_a - r_a, the frames q_FA = q_a q_jA and q_FB = q_b q_jB
// with axes u_x, u_y, u_z = the columns of R(q_FA), q_r = conj(q_FA) q_FB
// (negated when q_r.w < 0); a linear row along u has J = (-u, -(r1 x u),
// r_b x u), an angular row (0, -u, u).
static __device__ void joint_geom_adjoint(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a, int k,
                                          float* out) {
  for (int i = 0; i < 17; ++i) out[i] = 0.f;
  const JointDesc& j = p.joints[e.j0 + k];
  const int A = j.parent, B = j.child;
  const bool hasA = A >= 0, drive = j.k > 0.f || j.d > 0.f;
  const float h = p.h, tb = p.jbeta / h;
  const V3<float> z3 = v3<float>(0.f, 0.f, 0.f);
  // the forward's values
  const float4 xa4 = hasA ? w.bx[A] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 qa4 = hasA ? w.bq[A] : make_float4(1.f, 0.f, 0.f, 0.f);
  const float4 xb4 = w.bx[B], qb4 = w.bq[B];
  const V3<float> pa_l = tv<float>(j.pa), pb_l = tv<float>(j.pb);
  const Q4<float> qjA = tq<float>(j.qa), qjB = tq<float>(j.qb);
  V3<float> ra = z3, pa_w = pa_l, xA = pa_l;
  Q4<float> qFA = qjA;
  if (hasA) {
    xA = f3(xa4);
    ra = mul(qmat(ldq4(qa4)), pa_l);
    pa_w = xA + ra;
    qFA = qmul(ldq4(qa4), qjA);
  }
  const V3<float> rb = mul(qmat(ldq4(qb4)), pb_l), pb_w = f3(xb4) + rb;
  const Q4<float> qFB = qmul(ldq4(qb4), qjB);
  const M3<float> MF = qmat(qFA), MB = qmat(qFB);
  const V3<float> ux = col(MF, 0), uy = col(MF, 1), uz = col(MF, 2);
  const V3<float> dp = pb_w - pa_w;
  Q4<float> qr = qmul(qconj(qFA), qFB);
  const float sgn = qr.w < 0.f ? -1.f : 1.f;
  if (sgn < 0.f) { qr.w = -qr.w; qr.x = -qr.x; qr.y = -qr.y; qr.z = -qr.z; }
  const V3<float> raB = hasA ? pb_w - xA : z3;
  // adjoints
  V3<float> gux = z3, guy = z3, guz = z3, gra = z3, grb = z3, graB = z3, gdp = z3, gcr = z3;
  float gq[4] = {0.f, 0.f, 0.f, 0.f};   // of q_r (w, x, y, z)
  float gth = 0.f;                        // of the drive/limit angle
  const float4* G0 = a.radj + ROW_F4 * jrow(k, 0);
  int r = 0;
  // a linear row along u with arms (r1, r_b); returns the bias adjoint
  auto rev_lin = [&](const V3<float>& u, const V3<float>& r1, V3<float>* gu, V3<float>& gr1) {
    const float4* G = G0 + ROW_F4 * r++;
    const V3<float> gla = f3(G[0]), gaa = f3(G[1]), gab = f3(G[2]);
    if (gu) *gu = ((*gu - gla) - cross(gaa, r1)) + cross(gab, rb);
    gr1 = gr1 - cross(u, gaa);
    grb = grb + cross(u, gab);
    return G[1].w;
  };
  // an angular row about u
  auto rev_ang = [&](V3<float>& gu) {
    const float4* G = G0 + ROW_F4 * r++;
    gu = (gu + f3(G[2])) - f3(G[1]);
    return G[1].w;
  };
  // the soft drive's bias factor (Catto 2011), as g_soft forms it
  const float soft = (h * j.k / (j.d + h * j.k)) / h;
  int fbc = -1;   // column of R(q_FB) in the angular rows' error (revolute 0, planar 2)
  if (j.type == JT_REVOLUTE) {
    for (int c = 0; c < 3; ++c) {
      const float gb = rev_lin(unit<float>(c), ra, nullptr, gra);
      setc(gdp, c, comp(gdp, c) + tb * gb);
    }
    fbc = 0;
    const V3<float> fb = col(MB, 0), cr = cross(ux, fb);
    { const float gb = tb * rev_ang(guy); gcr = gcr + uy * gb; guy = guy + cr * gb; }
    { const float gb = tb * rev_ang(guz); gcr = gcr + uz * gb; guz = guz + cr * gb; }
    if (drive) { const float gC = soft * rev_ang(gux); gth += gC; out[14] -= gC; }
    if (j.lo < j.hi) {
      const float theta = 2.f * atan2f(qr.x, qr.w);
      for (int c = 0; c < 2; ++c) {
        V3<float> gu = z3;
        const float gb = rev_ang(gu);
        gux = c == 0 ? gux + gu : gux - gu;   // about u_x, then -u_x
        const float C = c == 0 ? theta - j.lo : j.hi - theta;
        const float gC = C > 0.f ? gb / h : tb * gb;
        gth += c == 0 ? gC : -gC;
      }
    }
    gux = gux + cross(fb, gcr);
    gcr = cross(gcr, ux);   // now the adjoint of R(q_FB)'s column
    const float den = qr.w * qr.w + qr.x * qr.x;
    if (den > 0.f) { gq[1] += gth * (2.f * qr.w) / den; gq[0] -= gth * (2.f * qr.x) / den; }
  } else if (j.type == JT_PRISMATIC) {
    { const float gb = tb * rev_lin(uy, raB, &guy, graB); gdp = gdp + uy * gb; guy = guy + dp * gb; }
    { const float gb = tb * rev_lin(uz, raB, &guz, graB); gdp = gdp + uz * gb; guz = guz + dp * gb; }
    gq[1] += 2.f * tb * rev_ang(gux);
    gq[2] += 2.f * tb * rev_ang(guy);
    gq[3] += 2.f * tb * rev_ang(guz);
    const float dd = dot(dp, ux);
    float gdd = 0.f;
    if (drive) { const float gC = soft * rev_lin(ux, raB, &gux, graB); gdd += gC; out[14] -= gC; }
    for (int c = 0; c < 2; ++c) {
      V3<float> gu = z3;
      const float gb = rev_lin(c == 0 ? ux : -ux, raB, &gu, graB);
      gux = c == 0 ? gux + gu : gux - gu;
      const float C = c == 0 ? dd - j.lo : j.hi - dd;
      const float gC = C > 0.f ? gb / h : tb * gb;
      gdd += c == 0 ? gC : -gC;
    }
    gdp = gdp + ux * gdd;
    gux = gux + dp * gdd;
  } else {
    { const float gb = tb * rev_lin(uz, raB, &guz, graB); gdp = gdp + uz * gb; guz = guz + dp * gb; }
    fbc = 2;
    const V3<float> fb = col(MB, 2), cr = cross(uz, fb);
    { const float gb = tb * rev_ang(gux); gcr = gcr + ux * gb; gux = gux + cr * gb; }
    { const float gb = tb * rev_ang(guy); gcr = gcr + uy * gb; guy = guy + cr * gb; }
    if (drive) {
      { const float gC = soft * rev_lin(ux, raB, &gux, graB); gdp = gdp + ux * gC; gux = gux + dp * gC; out[14] -= gC; }
      { const float gC = soft * rev_lin(uy, raB, &guy, graB); gdp = gdp + uy * gC; guy = guy + dp * gC; out[15] -= gC; }
      { const float gC = soft * rev_ang(guz); gth += gC; out[16] -= gC; }
    }
    guz = guz + cross(fb, gcr);
    gcr = cross(gcr, uz);
    const float den = qr.w * qr.w + qr.z * qr.z;
    if (den > 0.f) { gq[3] += gth * (2.f * qr.w) / den; gq[0] -= gth * (2.f * qr.z) / den; }
  }
  // q_r = sgn conj(q_FA) q_FB
  Q4<float> g0;
  g0.w = sgn * gq[0]; g0.x = sgn * gq[1]; g0.y = sgn * gq[2]; g0.z = sgn * gq[3];
  const Q4<float> gFAq = qconj(qmul(g0, qconj(qFB))), gFBq = qmul(qFA, g0);
  float gFA[4] = {gFAq.w, gFAq.x, gFAq.y, gFAq.z}, gFB[4] = {gFBq.w, gFBq.x, gFBq.y, gFBq.z};
  V3<float> unused = z3;
  const float4 fa4 = make_float4(qFA.w, qFA.x, qFA.y, qFA.z), fb4 = make_float4(qFB.w, qFB.x, qFB.y, qFB.z);
  rotate_adjoint(fa4, unit<float>(0), gux, unused, gFA);
  rotate_adjoint(fa4, unit<float>(1), guy, unused, gFA);
  rotate_adjoint(fa4, unit<float>(2), guz, unused, gFA);
  if (fbc >= 0) rotate_adjoint(fb4, unit<float>(fbc), gcr, unused, gFB);
  // q_FB = q_b q_jB, q_FA = q_a q_jA
  Q4<float> t;
  t.w = gFB[0]; t.x = gFB[1]; t.y = gFB[2]; t.z = gFB[3];
  const Q4<float> gqb = qmul(t, qconj(qjB));
  out[10] = gqb.w; out[11] = gqb.x; out[12] = gqb.y; out[13] = gqb.z;
  // positions: dp = p_b - p_a, raB = p_b - x_a, p = x + r
  const V3<float> gpb = gdp + graB;
  out[7] = gpb.x; out[8] = gpb.y; out[9] = gpb.z;
  grb = grb + gpb;
  rotate_adjoint(qb4, pb_l, grb, unused, out + 10);
  if (hasA) {
    t.w = gFA[0]; t.x = gFA[1]; t.y = gFA[2]; t.z = gFA[3];
    const Q4<float> gqa = qmul(t, qconj(qjA));
    out[3] = gqa.w; out[4] = gqa.x; out[5] = gqa.y; out[6] = gqa.z;
    const V3<float> gxa = (z3 - gdp) - graB;
    out[0] = gxa.x; out[1] = gxa.y; out[2] = gxa.z;
    gra = gra - gdp;
    rotate_adjoint(qa4, pa_l, gra, unused, out + 3);
  }
}

// Adjoint of one contact point's row geometry (contact_geom, then the
// tangent basis of the normal) for the adjoints of its normal, tangents,
// world arms and bias: out = adjoints of x_a 0-2, q_a 3-6, x_b 7-9, q_b
// 10-13, n 14-16, ra_l 17-19, rb_l 20-22 (a static b's anchor is in world).
template <int BK>
static __device__ void contact_geom_adjoint(const Params& p, const Ws& w, const AWs& a, int ci, int ia, int ibd,
                                     float* out) {
  const int ib = BK == BK_STATIC ? -1 : ibd;   // a static b's terms drop out at compile time
  for (int k = 0; k < 23; ++k) out[k] = 0.f;
  const float4* Q = a.cadj + CADJ_F4 * ci;
  const float4 xa4 = w.bx[ia], qa4 = w.bq[ia];
  const V3<float> n = f3(w.cn[ci]), ral = f3(w.cra[ci]), rbl = f3(w.crb[ci]);
  V3<float> gn = f3(Q[0]);
  const V3<float> gt1 = f3(Q[1]), gt2 = f3(Q[2]);
  // the tangent basis (Duff et al.): t1, t2 from n
  {
    const float sg = n.z >= 0.f ? 1.f : -1.f;
    const float al = -1.f / (sg + n.z);
    const float gb = gt1.y * sg + gt2.x;
    const float gal = gt1.x * sg * n.x * n.x + gt2.y * n.y * n.y + gb * n.x * n.y;
    gn.x += gt1.x * 2.f * sg * n.x * al + gb * n.y * al - gt1.z * sg;
    gn.y += gb * n.x * al + gt2.y * 2.f * n.y * al - gt2.z;
    gn.z += gal * al * al;
  }
  // arms and separation
  const V3<float> ra = mul(qmat(ldq4(qa4)), ral);
  const V3<float> pa = f3(xa4) + ra;
  V3<float> pb;
  float4 xb4 = make_float4(0.f, 0.f, 0.f, 0.f), qb4 = make_float4(1.f, 0.f, 0.f, 0.f);
  if (ib >= 0) {
    xb4 = w.bx[ib]; qb4 = w.bq[ib];
    pb = f3(xb4) + mul(qmat(ldq4(qb4)), rbl);
  } else pb = rbl;
  const float sep = dot(n, pb - pa);
  const float gbias = Q[3].w;
  const float gs = sep > 0.f ? gbias / p.h : (-sep - p.slop > 0.f ? gbias * (p.beta / p.h) : 0.f);
  gn = gn + (pb - pa) * gs;
  const V3<float> gpa = n * (-gs), gpb = n * gs;
  // a: pa = xa + R(qa) ra_l
  out[0] = gpa.x; out[1] = gpa.y; out[2] = gpa.z;
  V3<float> gral = v3<float>(0.f, 0.f, 0.f);
  rotate_adjoint(qa4, ral, f3(Q[3]) + gpa, gral, out + 3);
  // b: pb = xb + R(qb) rb_l, or the world anchor rb_l
  V3<float> grbl = v3<float>(0.f, 0.f, 0.f);
  if (ib >= 0) {
    out[7] = gpb.x; out[8] = gpb.y; out[9] = gpb.z;
    rotate_adjoint(qb4, rbl, f3(Q[4]) + gpb, grbl, out + 10);
  } else grbl = gpb;
  out[14] = gn.x; out[15] = gn.y; out[16] = gn.z;
  out[17] = gral.x; out[18] = gral.y; out[19] = gral.z;
  out[20] = grbl.x; out[21] = grbl.y; out[22] = grbl.z;
}

// Component `idx` (0-13) of a gather slot's pose part: x_a in 0-2, q_a in
// 4-7, x_b in 8-10, q_b in 12-15 of the slot's first four float4.
__device__ __forceinline__ int pose_slot(int idx) { return idx < 3 ? idx : idx < 7 ? idx + 1 : idx < 10 ? idx + 1 : idx + 2; }

// The reverse of the row set-up: per constraint the effective-mass part
// (onto Jacobians, arms, inverse inertias and inverse masses, written to the
// constraint's gather slot); then one item per joint and per contact point
// (the hand-written reverses of their row geometry); a contact point's pose
// adjoints are summed per manifold in point order, its normal and arm
// adjoints added to the point, a joint's target adjoints to its DoFs.
static __device__ void reverse_setup(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a) {
  const int J = e.J, M = w.misc[MC_MANIFOLDS], K = J + M, nc = w.misc[MC_CONTACTS];
  for (int k = e.lane; k < K; k += e.nthr) {
    int A, B;
    con_bodies(p, e, w, k, J, A, B);
    const float ima = A >= 0 ? w.bx[A].w : 0.f, imb = B >= 0 ? w.bx[B].w : 0.f;
    Sym3 Iwa, Iwb;
    if (A >= 0) Iwa = load_Iw(w, A);
    if (B >= 0) Iwb = load_Iw(w, B);
    float gIwa[6] = {0, 0, 0, 0, 0, 0}, gIwb[6] = {0, 0, 0, 0, 0, 0};
    float gima = 0.f, gimb = 0.f;
    const float sa = A >= 0 ? w.bIw1[A].z : 1.f, sb = B >= 0 ? w.bIw1[B].z : 1.f;   // Jacobi mass splits
    if (k < J) {
      const JointDesc& j = p.joints[e.j0 + k];
      const int nr = joint_row_count(j);
      for (int r = 0; r < nr; ++r)
        reverse_mass_part(a, jrow(k, r), A, B, ima, imb, Iwa, Iwb, gIwa, gIwb, gima, gimb, sa, sb);
    } else {
      int4 mf = man_get(w, k - J);
      const float4* MA = a.madj + 4 * (k - J);
      gIwa[0] = MA[0].x; gIwa[1] = MA[0].y; gIwa[2] = MA[0].z; gIwa[3] = MA[0].w; gIwa[4] = MA[1].x; gIwa[5] = MA[1].y;
      gIwb[0] = MA[1].z; gIwb[1] = MA[1].w; gIwb[2] = MA[2].x; gIwb[3] = MA[2].y; gIwb[4] = MA[2].z; gIwb[5] = MA[2].w;
      gima = MA[3].x; gimb = MA[3].y;
      by_b_kind(B >= 0, [&](auto kb) {
        for (int ci = mf.z; ci < mf.z + mf.w; ++ci)
          contact_mass_adjoint<decltype(kb)::v>(a, ci, B >= 0, ima, imb, Iwa, Iwb, gIwa, gIwb, gima, gimb, sa, sb);
      });
    }
    float4* S = a.gat + 8 * k;
    S[4] = make_float4(gIwa[0], gIwa[1], gIwa[2], gIwa[3]);
    S[5] = make_float4(gIwa[4], gIwa[5], gima, 0.f);
    S[6] = make_float4(gIwb[0], gIwb[1], gIwb[2], gIwb[3]);
    S[7] = make_float4(gIwb[4], gIwb[5], gimb, 0.f);
  }
  gsync(e);
  for (int t = e.lane; t < J + nc; t += e.nthr) {
    if (t < J) {
      float out[17];
      joint_geom_adjoint(p, e, w, a, t, out);
      float* S = (float*)(a.gat + 8 * t);
      for (int idx = 0; idx < 14; ++idx) S[pose_slot(idx)] = out[idx];
      S[pose_slot(2) + 1] = 0.f;
      S[pose_slot(9) + 1] = 0.f;
      const JointDesc& j = p.joints[e.j0 + t];
      const int nd = (j.k > 0.f || j.d > 0.f) ? joint_ndof(j.type) : 0;
      for (int c = 0; c < nd; ++c) a.tg[j.dof + c] += out[14 + c];
    } else {
      const int ci = t - J;
      const int ids = w.cid[ci];
      const int ia = ids & 0xffff, bc = ids >> 16;
      float out[23];
      const int ib = bc < e.D ? bc : -1;
      by_b_kind(ib >= 0, [&](auto k) { contact_geom_adjoint<decltype(k)::v>(p, w, a, ci, ia, ib, out); });
      float* cp = a.cpose + 16 * ci;
      for (int idx = 0; idx < 14; ++idx) cp[pose_slot(idx)] = out[idx];
      add4(a.cg[3 * ci + 0], v3<float>(out[14], out[15], out[16]));
      add4(a.cg[3 * ci + 1], v3<float>(out[17], out[18], out[19]));
      add4(a.cg[3 * ci + 2], v3<float>(out[20], out[21], out[22]));
    }
  }
  gsync(e);
  for (int m = e.lane; m < M; m += e.nthr) {
    const int4 mf = man_get(w, m);
    float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
    for (int ci = mf.z; ci < mf.z + mf.w; ++ci) {
      const float4* c = (const float4*)(a.cpose + 16 * ci);
      const float4 c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
      s0.x += c0.x; s0.y += c0.y; s0.z += c0.z;
      s1.x += c1.x; s1.y += c1.y; s1.z += c1.z; s1.w += c1.w;
      s2.x += c2.x; s2.y += c2.y; s2.z += c2.z;
      s3.x += c3.x; s3.y += c3.y; s3.z += c3.z; s3.w += c3.w;
    }
    float4* S = a.gat + 8 * (J + m);
    S[0] = s0; S[1] = s1; S[2] = s2; S[3] = s3;
  }
}

// Per body: sums the constraint gather slots in constraint order into the
// pose adjoints (and, when `inertia`, the world-inverse-inertia and 1/m
// adjoints into bI0/bI1).
static __device__ void gather_bodies(const EnvInfo& e, const AWs& a, bool inertia) {
  for (int i = e.lane; i < e.D; i += e.nthr) {
    float4 gx = a.bx[i], gq = a.bq[i];
    float4 I0 = make_float4(0.f, 0.f, 0.f, 0.f), I1 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = a.inc_off[i]; q < a.inc_off[i + 1]; ++q) {
      const int t = a.inc[q], k = t >> 1, side = t & 1;
      const float4* S = a.gat + 8 * k;
      float4 px = S[2 * side], pq = S[2 * side + 1];
      gx.x += px.x; gx.y += px.y; gx.z += px.z;
      gq.x += pq.x; gq.y += pq.y; gq.z += pq.z; gq.w += pq.w;
      if (inertia) {
        float4 s0 = S[4 + 2 * side], s1 = S[5 + 2 * side];
        I0.x += s0.x; I0.y += s0.y; I0.z += s0.z; I0.w += s0.w;
        I1.x += s1.x; I1.y += s1.y; I1.z += s1.z;
      }
    }
    a.bx[i] = gx;
    a.bq[i] = gq;
    if (inertia) { a.bI0[i] = I0; a.bI1[i] = I1; }
  }
}

// World inverse inertia adjoints -> orientation adjoint and principal inverse
// inertia adjoint; 1/m adjoint into the mass accumulator. W = sum_k d_k r_k
// r_k^T over the columns r_k of R(q) (world_inv_inertia), so with G the
// symmetric matrix of the six entries' adjoints (off-diagonal ones split
// between the two places) g(d_k) = r_k . G r_k and g(r_k) = 2 d_k G r_k,
// which the column's rotation adjoint takes to q.
static __device__ void reverse_inertia(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a) {
  for (int i = e.lane; i < e.D; i += e.nthr) {
    const float4 I0 = a.bI0[i], I1 = a.bI1[i];
    const float4 q4 = w.bq[i], inv = p.binv[e.b0 + i];
    const float hxy = 0.5f * I0.y, hxz = 0.5f * I0.z, hyz = 0.5f * I1.x;
    const M3<float> R = qmat(ldq4(q4));
    const float d[3] = {inv.y, inv.z, inv.w};
    float gq[4] = {0.f, 0.f, 0.f, 0.f}, gd[3];
    V3<float> unused = v3<float>(0.f, 0.f, 0.f);
    for (int k = 0; k < 3; ++k) {
      const V3<float> r = col(R, k);
      const V3<float> Gr = v3<float>(I0.x * r.x + hxy * r.y + hxz * r.z, hxy * r.x + I0.w * r.y + hyz * r.z,
                                     hxz * r.x + hyz * r.y + I1.y * r.z);
      gd[k] = dot(r, Gr);
      rotate_adjoint(q4, unit<float>(k), Gr * (2.f * d[k]), unused, gq);
    }
    float4 g = a.bq[i];
    g.x += gq[0]; g.y += gq[1]; g.z += gq[2]; g.w += gq[3];
    a.bq[i] = g;
    float4 m = a.bm[i];
    m.x += I1.z; m.y += gd[0]; m.z += gd[1]; m.w += gd[2];
    a.bm[i] = m;
  }
}

// Reverse of x += h v and q <- normalise(q + h/2 (0,w) q) for one substep,
// with x_s, q_s the substep-start pose and v_e, w_e the velocities it used.
static __device__ void reverse_integrate(const Params& p, const EnvInfo& e, const AWs& a, const float* sub_tape) {
  for (int i = e.lane; i < e.D; i += e.nthr) {
    const float* t = sub_tape + 19 * i;
    const float qw = t[3], qx = t[4], qy = t[5], qz = t[6];
    const float wx = t[16], wy = t[17], wz = t[18];
    float4 gx = a.bx[i], gq = a.bq[i], gv = a.bv[i], gw = a.bw[i];
    const float h = p.h, hh = h * 0.5f;
    // x' = x + h v
    gv.x += h * gx.x; gv.y += h * gx.y; gv.z += h * gx.z;
    // p = q + hh (0,w) q ; q' = p / |p|
    const float dqw = -(wx * qx + wy * qy + wz * qz);
    const float dqx = qw * wx + (wy * qz - wz * qy);
    const float dqy = qw * wy + (wz * qx - wx * qz);
    const float dqz = qw * wz + (wx * qy - wy * qx);
    const float pw = qw + hh * dqw, px = qx + hh * dqx, py = qy + hh * dqy, pz = qz + hh * dqz;
    const float nrm = sqrtf(pw * pw + px * px + py * py + pz * pz);
    const float ow = pw / nrm, ox = px / nrm, oy = py / nrm, oz = pz / nrm;
    const float s = ow * gq.x + ox * gq.y + oy * gq.z + oz * gq.w;
    const float gpw = (gq.x - ow * s) / nrm, gpx = (gq.y - ox * s) / nrm, gpy = (gq.z - oy * s) / nrm,
                gpz = (gq.w - oz * s) / nrm;
    float4 nq;
    nq.x = gpw + hh * (gpx * wx + gpy * wy + gpz * wz);
    nq.y = gpx + hh * (-gpw * wx + gpy * wz - gpz * wy);
    nq.z = gpy + hh * (-gpw * wy - gpx * wz + gpz * wx);
    nq.w = gpz + hh * (-gpw * wz + gpx * wy - gpy * wx);
    gw.x += hh * (-gpw * qx + gpx * qw - gpy * qz + gpz * qy);
    gw.y += hh * (-gpw * qy + gpx * qz + gpy * qw - gpz * qx);
    gw.z += hh * (-gpw * qz - gpx * qy + gpy * qx + gpz * qw);
    a.bq[i] = nq;
    a.bv[i] = gv;
    a.bw[i] = gw;
  }
}

// One dual pass of the narrowphase of manifold m's pair along pose input
// `idx` (x_a 0-2, q_a 3-6, x_b 7-9, q_b 10-13), contracted with the contact
// points' normal and anchor adjoints.
__device__ __forceinline__ float detect_pass(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a, int m,
                                             int idx) {
  const int4 mf = man_get(w, m);
  const int ia = mf.x, ib = mf.y;
  const int pj = w.cid[mf.z] >> 16;
  const float4 xa4 = w.bx[ia], qa4 = w.bq[ia];
  Shape<d1> Si, Sj;
  {
    float4 d = p.bdims[e.b0 + ia];
    Q4<d1> q; q.w = tan_of(idx, 3, qa4.x); q.x = tan_of(idx, 4, qa4.y); q.y = tan_of(idx, 5, qa4.z); q.z = tan_of(idx, 6, qa4.w);
    Si.type = __float_as_int(d.w);
    Si.c = v3<d1>(tan_of(idx, 0, xa4.x), tan_of(idx, 1, xa4.y), tan_of(idx, 2, xa4.z));
    Si.M = qmat(q);
    Si.d0 = d1(d.x); Si.d1 = d1(d.y); Si.d2 = d1(d.z);
  }
  if (ib >= 0) {
    const float4 xb4 = w.bx[ib], qb4 = w.bq[ib];
    float4 d = p.bdims[e.b0 + ib];
    Q4<d1> q; q.w = tan_of(idx, 10, qb4.x); q.x = tan_of(idx, 11, qb4.y); q.y = tan_of(idx, 12, qb4.z); q.z = tan_of(idx, 13, qb4.w);
    Sj.type = __float_as_int(d.w);
    Sj.c = v3<d1>(tan_of(idx, 7, xb4.x), tan_of(idx, 8, xb4.y), tan_of(idx, 9, xb4.z));
    Sj.M = qmat(q);
    Sj.d0 = d1(d.x); Sj.d1 = d1(d.y); Sj.d2 = d1(d.z);
  } else if (pj < e.D + e.S) {
    Sj = static_shape<d1>(p.sworld + (size_t)SW_N * (e.s0 + pj - e.D));   // the scene's static record
  } else {
    Sj.type = SH_PLANE;
    Sj.c = v3<d1>(d1(0.f), d1(0.f), d1(0.f));
    Sj.d0 = Sj.d1 = Sj.d2 = d1(0.f);
  }
  Pt<d1> pts[4];
  int n = collide(Si, Sj, d1(p.off), pts);
  float acc = 0.f;
  for (int k = 0; k < n && k < mf.w; ++k) {
    const int ci = mf.z + k;
    V3<d1> ral = mulT(Si.M, pts[k].pa - Si.c);
    V3<d1> rbl = ib >= 0 ? mulT(Sj.M, pts[k].pb - Sj.c) : pts[k].pb;
    float4 gn = a.cg[3 * ci], gra = a.cg[3 * ci + 1], grb = a.cg[3 * ci + 2];
    acc += gn.x * pts[k].n.x.d + gn.y * pts[k].n.y.d + gn.z * pts[k].n.z.d;
    acc += gra.x * ral.x.d + gra.y * ral.y.d + gra.z * ral.z.d;
    acc += grb.x * rbl.x.d + grb.y * rbl.y.d + grb.z * rbl.z.d;
  }
  return acc;
}

// Narrowphase routine class of manifold m's pair (collide's dispatch): the
// plane against each shape, then each unordered pair of shape types.
__device__ __forceinline__ int routine_class(const Params& p, const EnvInfo& e, const Ws& w, int m) {
  const int4 mf = man_get(w, m);
  const int ta = __float_as_int(p.bdims[e.b0 + mf.x].w);
  int tb;
  if (mf.y >= 0) tb = __float_as_int(p.bdims[e.b0 + mf.y].w);
  else tb = (w.cid[mf.z] >> 16) < e.D + e.S ? SH_BOX : SH_PLANE;
  if (tb == SH_PLANE) return ta;
  return 3 + 3 * min(ta, tb) + max(ta, tb);
}

// Adjoints of the step-start poses from the contact-geometry adjoints: dual
// passes of the narrowphase of each manifold's pair over its pose inputs (7
// against a static box or the plane, else 14), one (manifold, input) item per
// lane. The manifolds are taken sorted by routine class, a manifold's items
// on consecutive lanes, so that the lanes of a warp mostly run the same
// routine: its code is fetched once for all of them.
static __device__ void reverse_detection(const Params& p, const EnvInfo& e, const Ws& w, const AWs& a) {
  const int J = e.J, M = w.misc[MC_MANIFOLDS];
  enum { NCLS = 12 };
  if (e.lane == 0) {
    int start[NCLS];
    for (int c = 0; c < NCLS; ++c) start[c] = 0;
    for (int m = 0; m < M; ++m) start[routine_class(p, e, w, m)]++;
    int acc = 0;
    for (int c = 0; c < NCLS; ++c) { const int n = start[c]; start[c] = acc; acc += n; }
    for (int m = 0; m < M; ++m) a.mord[start[routine_class(p, e, w, m)]++] = m;
    acc = 0;
    for (int i = 0; i < M; ++i) { a.moff[i] = acc; acc += man_get(w, a.mord[i]).y >= 0 ? 14 : 7; }
    a.moff[M] = acc;
  }
  gsync(e);
  const int total = a.moff[M];
  for (int t = e.lane; t < total; t += e.nthr) {
    int lo = 0, hi = M - 1;   // the sorted position whose items hold t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.moff[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int m = a.mord[lo], idx = t - a.moff[lo];
    float* S = (float*)(a.gat + 8 * (J + m));
    if (idx == 2) S[3] = 0.f;
    if (idx == 6 && man_get(w, m).y < 0)
      for (int q = 8; q < 16; ++q) S[q] = 0.f;
    if (idx == 9) S[11] = 0.f;
    S[pose_slot(idx)] = detect_pass(p, e, w, a, m, idx);
  }
  // joints have no narrowphase inputs
  for (int k = e.lane; k < J; k += e.nthr)
    for (int q = 0; q < 4; ++q) a.gat[8 * k + q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace msh
