// Stages of the batched rigid-body step, written as block-cooperative device
// functions over one environment's workspace. The fused persistent kernel
// keeps the workspace in shared memory and calls every stage in sequence;
// the plain form launches one kernel per stage with the workspace in HBM.
// Both run the same functions with the same thread mapping, so their results
// are bitwise identical.
#pragma once
#include "msh_collide.cuh"

namespace msh {

enum { ST_PAIR_OVERFLOW = 1, ST_CONTACT_OVERFLOW = 2, ST_COLOUR_OVERFLOW = 4, ST_NONFINITE = 8 };
enum { JT_REVOLUTE = 0, JT_PRISMATIC = 1, JT_PLANAR = 2 };
enum { MODE_COLOURED = 0, MODE_JACOBI = 1 };
enum { MAX_COLOURS = 64, ROWS_PER_JOINT = 8 };
// misc counters in the workspace
enum { MC_PAIRS = 0, MC_CONTACTS = 1, MC_MANIFOLDS = 2, MC_COLOURS = 3, MC_STATUS = 4, MC_N = 8 };

struct JointDesc {     // 96 bytes
  int type, parent, child, dof;
  float pa[3], qa[4], pb[3], qb[4];
  float k, d, fmax, lo, hi;
  int roff;            // first solver row of this joint within its env's joint rows
};

// Solver rows of a joint: revolute 3 linear + 2 angular (+ drive) (+ 2 angle
// limits when lo < hi), prismatic 2 linear + 3 angular (+ drive) + 2 limits,
// planar 3 (+ 3 drives).
__host__ __device__ __forceinline__ int joint_row_count(const JointDesc& j) {
  const bool drive = j.k > 0.f || j.d > 0.f;
  if (j.type == JT_REVOLUTE) return 5 + (drive ? 1 : 0) + (j.lo < j.hi ? 2 : 0);
  if (j.type == JT_PRISMATIC) return drive ? 8 : 7;
  return drive ? 6 : 3;
}

// Byte offsets of the per-env workspace arrays (16-byte aligned).
// The collision-only arrays (body AABBs, pairs, colouring masks) and the
// per-substep contact rows are never live at the same time and share one
// region. Static boxes never move: their world frames and AABBs are computed
// once per scene (StaticWorld) and the collision stage reads them from that table.
struct Layout {
  int Dm, Sm, Jm, P, C, K, R;   // R: joint solver rows of the largest env
  int Ch;                       // contacts of an env whose solver data fit the hot part (fused form)
  int bx, bq, bv, bw, bIw0, bIw1;
  int alo, ahi, salo, sahi;
  int pairs, cn, cra, crb, cid, crep;
  int kra, krb, klam;
  int cnc, krac, krbc, klamc;   // full-capacity contact arrays in the cold part
  int kxc;                      // per contact point: coupling terms of its rows (cold part)
  int man, jr, jinfo, ccol, corder, coff, masks;
  int jdv, inc_off, inc, misc;
  int hot_bytes;    // shared memory in the fused form
  int cold_bytes;   // contact anchors and ids, body poses (read once per substep), always in HBM
  int bytes;        // hot + cold: one HBM slab in the plain form
};

struct Params {
  // scene
  int E, max_dof;
  const int* body_off;
  const int* static_off;
  const int* joint_off;
  const float4* bdims;   // (d0, d1, d2, shape)
  const float4* binv;    // (invm, invIx, invIy, invIz)
  const float* static_pose;
  const float* static_half;
  const float4* sworld;  // per static box: StaticWorld
  const JointDesc* joints;
  const int* env_order;
  int En;                // fused form: envs in this launch's work queue (env_order[0..En))
  // solver
  float dt, h;
  int S, N, mode;
  float gx, gy, gz, mu, rest, off, beta, jbeta, slop;
  int C, P;
  // state
  float* pos;
  float* quat;
  float* lv;
  float* av;
  const float* targets;
  int* status;
  // workspace
  Layout L;
  char* ws;              // HBM workspace base (plain form, or fused without room in SMEM)
  long long ws_stride;   // bytes between per-env (plain) or per-group (fused) slabs
  int G;                 // fused form: threads per env (8 or 16: several envs per warp)
  int* queue;
  // tape (recorded for the adjoint when non-null): slab per env, see TapeLayout
  float* tape;
  long long tape_slab;   // floats per env slab of one recorded step
  int tape_Rm;           // row slots per env and sweep: ROWS_PER_JOINT * Jm + 4 * C (a multiple of 4)
  // contact report (when rep_on; see stage_report)
  int rep_on;
  const int* rep_flags;      // per body: bit 0 robot link, bit 1 end-effector link
  const int* rep_fingers;    // per env: two env-local finger ids (-1: none)
  const int* rep_target;     // per env: env-local target id (-1: none)
  float rep_fmin, rep_cosmax;
  float* rep_body_force;     // [B][3]
  float* rep_target_force;   // [E][3]
  float* rep_finger_force;   // [E][2][3]
  float* rep_robot_force;    // [E], accumulated
  int* rep_grasped;          // [E]
  // plain-form launch indices
  int sub, it;
};

// Tape of one recorded step, per env (floats):
//   state at the step start:       Dm x 13  (x, q, v, w)
//   per substep s:                 Dm x 19  (x_s, q_s, v_s, w_s after gravity; v, w after the solve)
//   lambda after every sweep:      S x N x Rm (joint k row r: k*8 + r; contact c row i: 8*Jm + 4c + i)
//   joint targets of the step:     max_dof
// Tape of one recorded step, floats per env: t0 the start state (13 per
// body), t1 per substep the poses and velocities (19 per body), t2 the
// lambdas after every sweep, t3 the targets, t4 the collision stage's results
// (contact normals, anchors and ids, manifolds, colour order and offsets,
// counts) so that the adjoint need not run it again.
struct TapeLayout { long long t0, t1, t2, t3, t4, slab; };
__host__ __device__ __forceinline__ TapeLayout tape_layout(const Layout& L, int S, int N, int md) {
  TapeLayout t;
  const long long Rm = (long long)ROWS_PER_JOINT * L.Jm + 4LL * L.C;
  t.t0 = 0;
  t.t1 = t.t0 + 13LL * L.Dm;
  t.t2 = (t.t1 + 19LL * L.Dm * S + 3) & ~3LL;   // the sweeps' lambdas start on 16 bytes
  t.t3 = t.t2 + (long long)S * N * Rm;
  t.t4 = (t.t3 + md + 3) & ~3LL;
  t.slab = (t.t4 + ((13LL * L.C + 3) & ~3LL) + 4LL * L.P + L.K + (MAX_COLOURS + 1) + MC_N + 3) & ~3LL;
  return t;
}
// Offsets (floats) inside the t4 record; the float4/int4 arrays start on
// 16-byte boundaries (t4 and the tape slab are multiples of 4 floats).
__host__ __device__ __forceinline__ long long tc_cn(const Layout&) { return 0; }
__host__ __device__ __forceinline__ long long tc_cra(const Layout& L) { return 4LL * L.C; }
__host__ __device__ __forceinline__ long long tc_crb(const Layout& L) { return 8LL * L.C; }
__host__ __device__ __forceinline__ long long tc_cid(const Layout& L) { return 12LL * L.C; }
__host__ __device__ __forceinline__ long long tc_man(const Layout& L) { return (13LL * L.C + 3) & ~3LL; }
__host__ __device__ __forceinline__ long long tc_corder(const Layout& L) { return tc_man(L) + 4LL * L.P; }
__host__ __device__ __forceinline__ long long tc_coff(const Layout& L) { return tc_corder(L) + L.K; }
__host__ __device__ __forceinline__ long long tc_misc(const Layout& L) { return tc_coff(L) + MAX_COLOURS + 1; }
__device__ __forceinline__ float* tape_env(const Params& p, int env) { return p.tape + (long long)env * p.tape_slab; }

// World data of a static box, 6 float4: centre, the three rows of its
// rotation matrix (half extent in .w), AABB low and high corners (widened by
// the contact offset).
enum { SW_C = 0, SW_M = 1, SW_LO = 4, SW_HI = 5, SW_N = 6 };

struct Ws {
  float4 *bx, *bq, *bv, *bw, *bIw0, *bIw1;
  float4 *alo, *ahi;  // body AABBs
  float4 *salo, *sahi;  // the static boxes' AABBs, staged for the broadphase
  int* pairs;
  float4 *cn, *cra, *crb;
  float4* crep;       // contact report: impulse sums over the substeps, then forces
  int* cid;
  float4 *kra, *krb, *klam;
  float4* kx;         // per contact point: K(t1,n), K(t2,n), K(t2,t1)
  int2* man;          // manifolds packed: (a | (b + 1) << 16, first contact | count << 16)
  float4* jr;
  int4* jinfo;      // per joint: parent, child, first solver row, row count
  int *ccol, *corder, *coff;
  unsigned long long* masks;
  float4* jdv;
  int *inc_off, *inc, *misc;
};

// hot: the first L.hot_bytes of a slab or shared memory; cold: HBM.
__device__ __forceinline__ Ws make_ws(char* b, char* cold, const Layout& L) {
  Ws w;
  w.bx = (float4*)(cold + L.bx); w.bq = (float4*)(cold + L.bq);
  w.bv = (float4*)(b + L.bv); w.bw = (float4*)(b + L.bw);
  w.bIw0 = (float4*)(b + L.bIw0); w.bIw1 = (float4*)(b + L.bIw1);
  w.alo = (float4*)(b + L.alo); w.ahi = (float4*)(b + L.ahi);
  w.salo = (float4*)(b + L.salo); w.sahi = (float4*)(b + L.sahi);
  w.pairs = (int*)(b + L.pairs);
  w.cn = (float4*)(b + L.cn);
  w.cra = (float4*)(cold + L.cra); w.crb = (float4*)(cold + L.crb); w.cid = (int*)(cold + L.cid);
  w.crep = (float4*)(cold + L.crep);
  w.kra = (float4*)(b + L.kra); w.krb = (float4*)(b + L.krb); w.klam = (float4*)(b + L.klam);
  w.kx = (float4*)(cold + L.kxc);
  w.man = (int2*)(b + L.man); w.jr = (float4*)(b + L.jr); w.jinfo = (int4*)(b + L.jinfo);
  w.ccol = (int*)(cold + L.ccol); w.corder = (int*)(b + L.corder); w.coff = (int*)(b + L.coff);
  w.masks = (unsigned long long*)(b + L.masks);
  w.jdv = (float4*)(b + L.jdv); w.inc_off = (int*)(b + L.inc_off); w.inc = (int*)(b + L.inc);
  w.misc = (int*)(b + L.misc);
  return w;
}

// Manifold m as (body a, body b or -1, first contact, contact count).
__device__ __forceinline__ int4 man_get(const Ws& w, int m) {
  const int2 v = w.man[m];
  return make_int4(v.x & 0xffff, (int)((unsigned)v.x >> 16) - 1, v.y & 0xffff, (int)((unsigned)v.y >> 16));
}
__device__ __forceinline__ void man_set(const Ws& w, int m, int4 v) {
  w.man[m] = make_int2(v.x | ((v.y + 1) << 16), v.z | (v.w << 16));
}

// One env and the threads that work on it: `nthr` threads with group-local
// index `lane`. A group is a whole CTA (nthr >= 32) or an aligned slice of a
// warp (nthr = 8 or 16, lanes `mask`), so several envs can share one warp.
struct EnvInfo {
  int env, b0, D, s0, S, j0, J;
  int lane, nthr;
  unsigned mask;
};

__device__ __forceinline__ EnvInfo env_info(const Params& p, int env, int lane, int nthr, unsigned mask) {
  EnvInfo e;
  e.env = env;
  e.b0 = p.body_off[env]; e.D = p.body_off[env + 1] - e.b0;
  e.s0 = p.static_off[env]; e.S = p.static_off[env + 1] - e.s0;
  e.j0 = p.joint_off[env]; e.J = p.joint_off[env + 1] - e.j0;
  e.lane = lane; e.nthr = nthr; e.mask = mask;
  return e;
}
// the whole CTA on one env
__device__ __forceinline__ EnvInfo env_info(const Params& p, int env) {
  return env_info(p, env, threadIdx.x, blockDim.x, 0xffffffffu);
}

// Barrier and vote over the env's threads.
__device__ __forceinline__ void gsync(const EnvInfo& e) {
  if (e.nthr < 32) __syncwarp(e.mask);
  else __syncthreads();
}
__device__ __forceinline__ int gany(const EnvInfo& e, int v) {
  return e.nthr < 32 ? __any_sync(e.mask, v) : __syncthreads_or(v);
}

// The kind of a contact's second body b for the code paths specialised on
// it: static (a static box or the plane: no velocity, no impulse, its terms
// drop out at compile time), dynamic, or either (decided per lane at run
// time). A warp takes a specialised path only when all its active lanes
// agree, so lanes whose b differ share one path instead of running the two
// specialised ones after each other. Every path computes the same values.
enum { BK_STATIC = 0, BK_DYNAMIC = 1, BK_EITHER = 2 };
template <int K> struct BKind { static constexpr int v = K; };
template <int BK> __device__ __forceinline__ bool b_dyn(bool dyn) {
  return BK == BK_EITHER ? dyn : BK == BK_DYNAMIC;
}
// Calls f(BKind<kind>()) with the kind the active lanes share (BK_EITHER if
// they differ); all of them take the same branch.
template <class F> __device__ __forceinline__ void by_b_kind(bool dyn, F&& f) {
  const unsigned am = __activemask();
  if (__all_sync(am, !dyn)) f(BKind<BK_STATIC>());
  else if (__all_sync(am, dyn)) f(BKind<BK_DYNAMIC>());
  else f(BKind<BK_EITHER>());
}

// Exclusive block-wide prefix sum; every thread of the block must call it.
// `scr` is 33 ints of shared memory.
__device__ __forceinline__ int block_exscan(int v, int* scr, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scr[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = lane < nw ? scr[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) scr[lane] = s;
  }
  __syncthreads();
  int off = warp > 0 ? scr[warp - 1] : 0;
  *total = scr[nw - 1];
  __syncthreads();
  return off + x - v;
}

// Exclusive count of the set flags over the env's threads (all of them must
// call it): one warp vote within a group of at most 32 threads.
__device__ __forceinline__ int group_flag_exscan(const EnvInfo& e, int flag, int* scr, int* total) {
  if (e.nthr > 32) return block_exscan(flag, scr, total);
  const unsigned b = __ballot_sync(e.mask, flag) & e.mask;
  *total = __popc(b);
  return __popc(b & ((1u << (threadIdx.x & 31)) - 1u));
}

// Exclusive prefix sum of values in 0..7 over the env's threads (all of them
// must call it): one warp vote per bit within a group of at most 32 threads.
__device__ __forceinline__ int group_small_exscan(const EnvInfo& e, int v, int* scr, int* total) {
  if (e.nthr > 32) return block_exscan(v, scr, total);
  const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
  const unsigned b0 = __ballot_sync(e.mask, v & 1) & e.mask;
  const unsigned b1 = __ballot_sync(e.mask, v & 2) & e.mask;
  const unsigned b2 = __ballot_sync(e.mask, v & 4) & e.mask;
  *total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
  return __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
}

// ---------------------------------------------------------------------------
// a0: stage the env's bodies and statics
// ---------------------------------------------------------------------------

// Per-joint solver bookkeeping into the workspace (read by every sweep).
__device__ __forceinline__ void load_jinfo(const Params& p, const EnvInfo& e, const Ws& w) {
  for (int k = e.lane; k < e.J; k += e.nthr) {
    const JointDesc& j = p.joints[e.j0 + k];
    w.jinfo[k] = make_int4(j.parent, j.child, j.roff, joint_row_count(j));
  }
}

static __device__ void stage_load(const Params& p, const EnvInfo& e, const Ws& w) {
  for (int i = e.lane; i < e.D; i += e.nthr) {
    int g = e.b0 + i;
    float4 inv = p.binv[g];
    w.bx[i] = make_float4(p.pos[3 * g], p.pos[3 * g + 1], p.pos[3 * g + 2], inv.x);
    w.bq[i] = make_float4(p.quat[4 * g], p.quat[4 * g + 1], p.quat[4 * g + 2], p.quat[4 * g + 3]);
    w.bv[i] = make_float4(p.lv[3 * g], p.lv[3 * g + 1], p.lv[3 * g + 2], 0.f);
    w.bw[i] = make_float4(p.av[3 * g], p.av[3 * g + 1], p.av[3 * g + 2], 0.f);
    w.bIw1[i] = make_float4(0.f, 0.f, 1.f, 0.f);   // .z: Jacobi split count (1 unless set by the colouring)
    if (p.tape) {
      float* t = tape_env(p, e.env) + 13 * i;
      t[0] = p.pos[3 * g]; t[1] = p.pos[3 * g + 1]; t[2] = p.pos[3 * g + 2];
      t[3] = p.quat[4 * g]; t[4] = p.quat[4 * g + 1]; t[5] = p.quat[4 * g + 2]; t[6] = p.quat[4 * g + 3];
      t[7] = p.lv[3 * g]; t[8] = p.lv[3 * g + 1]; t[9] = p.lv[3 * g + 2];
      t[10] = p.av[3 * g]; t[11] = p.av[3 * g + 1]; t[12] = p.av[3 * g + 2];
    }
  }
  if (p.tape) {
    TapeLayout tl = tape_layout(p.L, p.S, p.N, p.max_dof);
    for (int k = e.lane; k < p.max_dof; k += e.nthr)
      tape_env(p, e.env)[tl.t3 + k] = p.targets ? p.targets[(size_t)e.env * p.max_dof + k] : 0.f;
  }
  load_jinfo(p, e, w);
  if (e.lane < MC_N) w.misc[e.lane] = 0;
}

// Collision shape of a static box from its StaticWorld record.
template <class T> __device__ __forceinline__ Shape<T> static_shape(const float4* sw) {
  float4 c = sw[SW_C], r0 = sw[SW_M], r1 = sw[SW_M + 1], r2 = sw[SW_M + 2];
  Shape<T> s;
  s.type = SH_BOX;
  s.c = v3<T>(T(c.x), T(c.y), T(c.z));
  s.M.m[0][0] = T(r0.x); s.M.m[0][1] = T(r0.y); s.M.m[0][2] = T(r0.z);
  s.M.m[1][0] = T(r1.x); s.M.m[1][1] = T(r1.y); s.M.m[1][2] = T(r1.z);
  s.M.m[2][0] = T(r2.x); s.M.m[2][1] = T(r2.y); s.M.m[2][2] = T(r2.z);
  s.d0 = T(r0.w); s.d1 = T(r1.w); s.d2 = T(r2.w);
  return s;
}

// World frame and AABB of each static box: the same FP32 arithmetic as the
// per-step shapes, done once per scene.
__device__ __forceinline__ void static_world(const float* sp, const float* sh, float off, float4* out) {
  Q4<nf> q; q.w = nf(sp[3]); q.x = nf(sp[4]); q.y = nf(sp[5]); q.z = nf(sp[6]);
  M3<nf> M = qmat(q);
  out[SW_C] = make_float4(sp[0], sp[1], sp[2], 0.f);
  for (int r = 0; r < 3; ++r) out[SW_M + r] = make_float4(M.m[r][0].v, M.m[r][1].v, M.m[r][2].v, sh[r]);
  Shape<nf> s;
  s.type = SH_BOX;
  s.c = v3<nf>(nf(sp[0]), nf(sp[1]), nf(sp[2]));
  s.M = M;
  s.d0 = nf(sh[0]); s.d1 = nf(sh[1]); s.d2 = nf(sh[2]);
  AABBt<nf> b = shape_aabb(s, nf(off));
  out[SW_LO] = make_float4(b.lo.x.v, b.lo.y.v, b.lo.z.v, 0.f);
  out[SW_HI] = make_float4(b.hi.x.v, b.hi.y.v, b.hi.z.v, 0.f);
}

// AABB corners of collision index i < D + S (body or static box).
// (A static box's record is read from the scene's table, through the
// read-only cache.)
__device__ __forceinline__ float4 aabb_lo(const Params& p, const Ws& w, const EnvInfo& e, int i) {
  return i < e.D ? w.alo[i] : w.salo[i - e.D];
}
__device__ __forceinline__ float4 aabb_hi(const Params& p, const Ws& w, const EnvInfo& e, int i) {
  return i < e.D ? w.ahi[i] : w.sahi[i - e.D];
}

// Collision shape of index i: dynamic body, static box or the plane.
__device__ __forceinline__ Shape<nf> coll_shape(const Params& p, const Ws& w, const EnvInfo& e, int i) {
  Shape<nf> s;
  if (i < e.D) {
    float4 x = w.bx[i], q4 = w.bq[i], d = __ldg(&p.bdims[e.b0 + i]);
    Q4<nf> q; q.w = nf(q4.x); q.x = nf(q4.y); q.y = nf(q4.z); q.z = nf(q4.w);
    s.type = __float_as_int(d.w);
    s.c = v3<nf>(nf(x.x), nf(x.y), nf(x.z));
    s.M = qmat(q);
    s.d0 = nf(d.x); s.d1 = nf(d.y); s.d2 = nf(d.z);
  } else if (i < e.D + e.S) {
    s = static_shape<nf>(p.sworld + (size_t)SW_N * (e.s0 + i - e.D));
  } else {
    s.type = SH_PLANE;
    s.c = v3<nf>(nf(0.f), nf(0.f), nf(0.f));
    s.d0 = s.d1 = s.d2 = nf(0.f);
  }
  return s;
}

// ---------------------------------------------------------------------------
// a2: AABBs of the bodies (static boxes: StaticWorld)
// ---------------------------------------------------------------------------
static __device__ void stage_aabb(const Params& p, const EnvInfo& e, const Ws& w) {
  // the static boxes' AABBs (computed once per scene) next to the bodies'
  for (int i = e.lane; i < e.S; i += e.nthr) {
    const float4* r = p.sworld + (size_t)SW_N * (e.s0 + i);
    w.salo[i] = __ldg(r + SW_LO);
    w.sahi[i] = __ldg(r + SW_HI);
  }
  for (int i = e.lane; i < e.D; i += e.nthr) {
    Shape<nf> s = coll_shape(p, w, e, i);
    AABBt<nf> b = shape_aabb(s, nf(p.off));
    w.alo[i] = make_float4(b.lo.x.v, b.lo.y.v, b.lo.z.v, 0.f);
    w.ahi[i] = make_float4(b.hi.x.v, b.hi.y.v, b.hi.z.v, 0.f);
  }
}

// ---------------------------------------------------------------------------
// a3: broadphase over the flattened (i<j) candidate list, order-preserving
// compaction with a block scan
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool jointed(const EnvInfo& e, const Ws& w, int i, int j) {
  for (int k = 0; k < e.J; ++k) {
    const int4 jd = w.jinfo[k];   // parent, child (staged with the bodies)
    if ((jd.x == i && jd.y == j) || (jd.x == j && jd.y == i)) return true;
  }
  return false;
}

static __device__ void stage_broadphase(const Params& p, const EnvInfo& e, const Ws& w, int* scr) {
  const int D = e.D, W = e.D + e.S;   // j in (i, W]; W is the plane
  // The candidates (i, j), i < D, i < j <= W, in row order: row i holds W - i
  // of them. A round tests nthr consecutive candidates; each thread walks its
  // own (i, j) forward by nthr per round (past the end of row i, j restarts
  // at i + 2), and (i, j) with i = D marks the end.
  const long long total = (long long)D * W - (long long)D * (D - 1) / 2;
  int pi = 0, pj = 1 + e.lane;
  while (pj > W && pi < D) { pj -= W - pi - 1; ++pi; }
  int count = 0;
  int status = 0;
  for (long long base = 0; base < total; base += e.nthr) {
    int flag = 0;
    if (pi < D) {
      float4 al = w.alo[pi];
      if (pj == W) {
        flag = al.z <= 0.f;
      } else {
        float4 ah = w.ahi[pi], bl = aabb_lo(p, w, e, pj), bh = aabb_hi(p, w, e, pj);
        flag = al.x <= bh.x && bl.x <= ah.x && al.y <= bh.y && bl.y <= ah.y && al.z <= bh.z && bl.z <= ah.z;
        if (flag && pj < D && jointed(e, w, pi, pj)) flag = 0;
      }
    }
    int tot;
    int pre = group_flag_exscan(e, flag, scr, &tot);
    if (flag) {
      int slot = count + pre;
      if (slot < p.P) w.pairs[slot] = pi | (pj << 16);
    }
    count += tot;
    pj += e.nthr;
    while (pj > W && pi < D) { pj -= W - pi - 1; ++pi; }
  }
  if (count > p.P) { status |= ST_PAIR_OVERFLOW; count = p.P; }
  if (e.lane == 0) {
    w.misc[MC_PAIRS] = count;
    w.misc[MC_STATUS] |= status;
  }
  gsync(e);
}

// ---------------------------------------------------------------------------
// a4: narrowphase, pairs in order, points in routine order, truncated at C
// ---------------------------------------------------------------------------
static __device__ void stage_narrowphase(const Params& p, const EnvInfo& e, const Ws& w, int* scr) {
  const int npairs = w.misc[MC_PAIRS];
  int cbase = 0, mbase = 0;
  bool over = false;
  for (int base = 0; base < npairs; base += e.nthr) {
    int idx = base + e.lane;
    Pt<nf> pts[4];
    Shape<nf> Si, Sj;
    int n = 0, pi = 0, pj = 0;
    if (idx < npairs) {
      int pr = w.pairs[idx];
      pi = pr & 0xffff;
      pj = pr >> 16;
      Si = coll_shape(p, w, e, pi);
      Sj = coll_shape(p, w, e, pj);
      n = collide(Si, Sj, nf(p.off), pts);
    }
    int tot;
    int pre = group_small_exscan(e, n, scr, &tot);   // n <= 4
    int start = cbase + pre;
    int kept = n;
    if (start + kept > p.C) kept = max(0, p.C - start);
    if (idx < npairs && kept > 0) {
      for (int k = 0; k < kept; ++k) {
        int c = start + k;
        V3<nf> ra = mulT(Si.M, pts[k].pa - Si.c);
        V3<nf> rb = pj < e.D ? mulT(Sj.M, pts[k].pb - Sj.c) : pts[k].pb;
        w.cn[c] = make_float4(pts[k].n.x.v, pts[k].n.y.v, pts[k].n.z.v, pts[k].s.v);
        w.cra[c] = make_float4(ra.x.v, ra.y.v, ra.z.v, 0.f);
        w.crb[c] = make_float4(rb.x.v, rb.y.v, rb.z.v, 0.f);
        w.cid[c] = pi | (pj << 16);
      }
    }
    int mt;
    int mpre = group_flag_exscan(e, kept > 0 ? 1 : 0, scr, &mt);
    if (idx < npairs && kept > 0)
      man_set(w, mbase + mpre, make_int4(pi, pj < e.D ? pj : -1, start, kept));
    if (cbase + tot > p.C) over = true;
    cbase = min(cbase + tot, p.C);
    mbase += mt;
  }
  if (e.lane == 0) {
    w.misc[MC_CONTACTS] = cbase;
    w.misc[MC_MANIFOLDS] = mbase;
    if (over) w.misc[MC_STATUS] |= ST_CONTACT_OVERFLOW;
  }
  gsync(e);
}

// ---------------------------------------------------------------------------
// a5 (once per step): greedy colouring of joints then manifolds, colour-sorted
// constraint order; Jacobi split counts and body incidence lists
// ---------------------------------------------------------------------------
static __device__ void stage_colour(const Params& p, const EnvInfo& e, const Ws& w) {
  const int J = e.J, M = w.misc[MC_MANIFOLDS], K = J + M;
  // The constraints of a colour share no dynamic body, so their order does
  // not change the result. A colour lists its joints first, then its
  // manifolds by decreasing point count (classes 0..4: joints, manifolds of
  // 4, 3, 2 and 1 points), so that a sweep runs each colour's joints and its
  // manifolds as two loops of like work: a counting sort on (colour, class)
  // whose keys and bucket counters use the contact-row lambdas as scratch
  // (free until the rows are built). Without room there the constraints keep
  // their index order (joints first too). coff[c] holds the colour's first
  // entry in its low 16 bits and its joint count in the high 16 bits.
  constexpr int NB = 5 * MAX_COLOURS;
  int* key = reinterpret_cast<int*>(w.klam);
  int* bucket = key + K;
  // room for the keys, and no overlap with the colouring masks (the hot
  // contact rows share a region with the collision arrays)
  const char* k0 = reinterpret_cast<const char*>(key);
  const char* m0 = reinterpret_cast<const char*>(w.masks);
  const bool keyed = K + NB <= 4 * min(p.L.Ch, p.L.C) &&
                     (k0 + 4 * (K + NB) <= m0 || k0 >= m0 + 8 * e.D);
  if (keyed)
    for (int i = e.lane; i < NB; i += e.nthr) bucket[i] = 0;
  gsync(e);
  if (e.lane == 0) {
    for (int i = 0; i < e.D; ++i) w.masks[i] = 0ull;
    int ncol = 0, status = 0;
    int cnt[MAX_COLOURS + 1];
    if (!keyed)
      for (int c = 0; c <= MAX_COLOURS; ++c) cnt[c] = 0;
    for (int k = 0; k < K; ++k) {
      int a, b, cls = 0;
      if (k < J) { const int4 jd = w.jinfo[k]; a = jd.x; b = jd.y; }
      else {
        int4 m = man_get(w, k - J); a = m.x; b = m.y;
        cls = 5 - min(m.w, 4);
      }
      unsigned long long msk = 0ull;
      if (a >= 0) msk |= w.masks[a];
      if (b >= 0) msk |= w.masks[b];
      int c;
      if (msk == ~0ull) { c = -1; status |= ST_COLOUR_OVERFLOW; }
      else {
        c = __ffsll((long long)~msk) - 1;
        if (a >= 0) w.masks[a] |= 1ull << c;
        if (b >= 0) w.masks[b] |= 1ull << c;
        if (keyed) bucket[5 * c + cls]++;
        else cnt[c]++;
        if (c + 1 > ncol) ncol = c + 1;
      }
      w.ccol[k] = c;
      if (keyed) key[k] = c < 0 ? -1 : 5 * c + cls;
    }
    int acc = 0;
    if (keyed) {
      for (int c = 0; c < ncol; ++c) {
        w.coff[c] = acc;
        for (int q = 0; q < 5; ++q) { const int n = bucket[5 * c + q]; bucket[5 * c + q] = acc; acc += n; }
      }
      w.coff[ncol] = acc;
      for (int k = 0; k < K; ++k) {
        const int v = key[k];
        if (v >= 0) w.corder[bucket[v]++] = k;
      }
    } else {
      for (int c = 0; c < ncol; ++c) { w.coff[c] = acc; acc += cnt[c]; cnt[c] = w.coff[c]; }
      w.coff[ncol] = acc;
      for (int k = 0; k < K; ++k) {
        const int c = w.ccol[k];
        if (c >= 0) w.corder[cnt[c]++] = k;
      }
    }
    for (int c = 0; c < ncol; ++c) {
      const int c0 = w.coff[c], c1 = w.coff[c + 1];
      int j = c0;
      while (j < c1 && w.corder[j] < J) ++j;
      w.coff[c] = c0 | ((j - c0) << 16);
    }
    w.misc[MC_COLOURS] = ncol;
    w.misc[MC_STATUS] |= status;
    if (p.mode == MODE_JACOBI) {
      for (int i = 0; i <= e.D; ++i) w.inc_off[i] = 0;
      for (int k = 0; k < K; ++k) {
        int a, b;
        if (k < J) { const int4 jd = w.jinfo[k]; a = jd.x; b = jd.y; }
        else { int4 m = man_get(w, k - J); a = m.x; b = m.y; }
        if (a >= 0) w.inc_off[a + 1]++;
        if (b >= 0) w.inc_off[b + 1]++;
      }
      for (int i = 0; i < e.D; ++i) {
        int n = w.inc_off[i + 1];
        w.bIw1[i].z = (float)(n > 0 ? n : 1);
        w.inc_off[i + 1] += w.inc_off[i];
      }
      for (int i = 0; i < e.D; ++i) w.masks[i] = (unsigned long long)w.inc_off[i];   // fill cursor
      for (int k = 0; k < K; ++k) {
        int a, b;
        if (k < J) { const int4 jd = w.jinfo[k]; a = jd.x; b = jd.y; }
        else { int4 m = man_get(w, k - J); a = m.x; b = m.y; }
        if (a >= 0) w.inc[w.masks[a]++] = 2 * k;
        if (b >= 0) w.inc[w.masks[b]++] = 2 * k + 1;
      }
    }
  }
  gsync(e);
}

// Records the collision stage's results of a recorded step (tape record t4).
static __device__ void tape_collision(const Params& p, const EnvInfo& e, const Ws& w) {
  const Layout& L = p.L;
  float* t = tape_env(p, e.env) + tape_layout(L, p.S, p.N, p.max_dof).t4;
  const int nc = w.misc[MC_CONTACTS], nm = w.misc[MC_MANIFOLDS], K = e.J + nm, ncol = w.misc[MC_COLOURS];
  float4* cn = (float4*)(t + tc_cn(L));
  float4* cra = (float4*)(t + tc_cra(L));
  float4* crb = (float4*)(t + tc_crb(L));
  int* cid = (int*)(t + tc_cid(L));
  int4* man = (int4*)(t + tc_man(L));
  int* corder = (int*)(t + tc_corder(L));
  int* coff = (int*)(t + tc_coff(L));
  int* misc = (int*)(t + tc_misc(L));
  for (int i = e.lane; i < nc; i += e.nthr) { cn[i] = w.cn[i]; cra[i] = w.cra[i]; crb[i] = w.crb[i]; cid[i] = w.cid[i]; }
  for (int i = e.lane; i < nm; i += e.nthr) man[i] = man_get(w, i);
  for (int i = e.lane; i < K; i += e.nthr) corder[i] = w.corder[i];
  for (int i = e.lane; i <= ncol; i += e.nthr) coff[i] = w.coff[i];
  for (int i = e.lane; i < MC_N; i += e.nthr) misc[i] = w.misc[i];
}

// The recorded collision stage back into a workspace (the adjoint's replay).
static __device__ void untape_collision(const Params& p, const EnvInfo& e, const Ws& w, const float* tape) {
  const Layout& L = p.L;
  const float* t = tape + tape_layout(L, p.S, p.N, p.max_dof).t4;
  const int* misc = (const int*)(t + tc_misc(L));
  const int nc = misc[MC_CONTACTS], nm = misc[MC_MANIFOLDS], K = e.J + nm, ncol = misc[MC_COLOURS];
  const float4* cn = (const float4*)(t + tc_cn(L));
  const float4* cra = (const float4*)(t + tc_cra(L));
  const float4* crb = (const float4*)(t + tc_crb(L));
  const int* cid = (const int*)(t + tc_cid(L));
  const int4* man = (const int4*)(t + tc_man(L));
  const int* corder = (const int*)(t + tc_corder(L));
  const int* coff = (const int*)(t + tc_coff(L));
  for (int i = e.lane; i < nc; i += e.nthr) { w.cn[i] = cn[i]; w.cra[i] = cra[i]; w.crb[i] = crb[i]; w.cid[i] = cid[i]; }
  for (int i = e.lane; i < nm; i += e.nthr) man_set(w, i, man[i]);
  for (int i = e.lane; i < K; i += e.nthr) w.corder[i] = corder[i];
  for (int i = e.lane; i <= ncol; i += e.nthr) w.coff[i] = coff[i];
  for (int i = e.lane; i < MC_N; i += e.nthr) w.misc[i] = misc[i];
}

// ---------------------------------------------------------------------------
// a1: gravity; world inverse inertia
// ---------------------------------------------------------------------------
static __device__ void stage_integrate_vel(const Params& p, const EnvInfo& e, const Ws& w, int sub) {
  for (int i = e.lane; i < e.D; i += e.nthr) {
    float4 v = w.bv[i];
    v.x = v.x + p.gx * p.h; v.y = v.y + p.gy * p.h; v.z = v.z + p.gz * p.h;
    w.bv[i] = v;
    if (p.tape) {
      TapeLayout tl = tape_layout(p.L, p.S, p.N, p.max_dof);
      float* t = tape_env(p, e.env) + tl.t1 + 19LL * (sub * p.L.Dm + i);
      float4 x = w.bx[i], q = w.bq[i], wv = w.bw[i];
      t[0] = x.x; t[1] = x.y; t[2] = x.z; t[3] = q.x; t[4] = q.y; t[5] = q.z; t[6] = q.w;
      t[7] = v.x; t[8] = v.y; t[9] = v.z; t[10] = wv.x; t[11] = wv.y; t[12] = wv.z;
    }
    float4 q4 = w.bq[i], I = __ldg(&p.binv[e.b0 + i]);
    const float split = w.bIw1[i].z;
    Q4<float> q; q.w = q4.x; q.x = q4.y; q.y = q4.z; q.z = q4.w;
    M3<float> R = qmat(q);
    float d[3] = {I.y, I.z, I.w};
    float W[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        W[a][b] = R.m[a][0] * d[0] * R.m[b][0] + R.m[a][1] * d[1] * R.m[b][1] + R.m[a][2] * d[2] * R.m[b][2];
    w.bIw0[i] = make_float4(W[0][0], W[0][1], W[0][2], W[1][1]);
    w.bIw1[i] = make_float4(W[1][2], W[2][2], split, w.bx[i].w);   // .w: 1/m for the sweeps
  }
}

__device__ __forceinline__ Sym3 load_Iw(const Ws& w, int i) {
  float4 a = w.bIw0[i], b = w.bIw1[i];
  Sym3 S; S.xx = a.x; S.xy = a.y; S.xz = a.z; S.yy = a.w; S.yz = b.x; S.zz = b.y;
  return S;
}

// ---------------------------------------------------------------------------
// a5 (per substep): rows
// ---------------------------------------------------------------------------
// Generic joint row. Every joint row has lb = -la (linear rows: -u, u;
// angular rows: 0, 0), so a row is stored as 5 float4: la|m, aa|bias,
// ab|gamma, Ia|lam, Ib|clamp, where clamp >= 0 means lambda in [-clamp,
// clamp] (soft drive), CLAMP_UNI means lambda >= 0 and CLAMP_FREE no clamp.
enum { ROW_F4 = 5 };
#define CLAMP_UNI (-1.f)
#define CLAMP_FREE (-2.f)
struct JRow { V3<float> la, aa, lb, ab, Ia, Ib; float m, bias, gamma, lam, lo, hi; };

__device__ __forceinline__ void put_row(float4* r, const JRow& x) {
  // only soft rows have a finite upper clamp
  float clamp = x.hi != INFINITY ? x.hi : (x.lo == 0.f ? CLAMP_UNI : CLAMP_FREE);
  r[0] = f4(x.la, x.m); r[1] = f4(x.aa, x.bias); r[2] = f4(x.ab, x.gamma);
  r[3] = f4(x.Ia, x.lam); r[4] = f4(x.Ib, clamp);
}

__device__ __forceinline__ JRow blank_row() {
  JRow r;
  V3<float> z = v3<float>(0.f, 0.f, 0.f);
  r.la = z; r.aa = z; r.lb = z; r.ab = z; r.Ia = z; r.Ib = z;
  r.m = 0.f; r.bias = 0.f; r.gamma = 0.f; r.lam = 0.f; r.lo = -INFINITY; r.hi = INFINITY;
  return r;
}

struct RowCtx { int a, b; float ima, imb, sa, sb; Sym3 Ia, Ib; };

__device__ __forceinline__ void finish_row(JRow& r, const RowCtx& c, bool soft) {
  float K = 0.f;
  if (c.a >= 0) { r.Ia = smulf(c.Ia, r.aa); K = fmaf(c.sa, fmaf(c.ima, dotf(r.la, r.la), dotf(r.aa, r.Ia)), K); }
  if (c.b >= 0) { r.Ib = smulf(c.Ib, r.ab); K = fmaf(c.sb, fmaf(c.imb, dotf(r.lb, r.lb), dotf(r.ab, r.Ib)), K); }
  if (soft) r.m = 1.f / (K + r.gamma);
  else r.m = K > 0.f ? 1.f / K : 0.f;
}

__device__ __forceinline__ Q4<float> ldq4(float4 q) { Q4<float> r; r.w = q.x; r.x = q.y; r.y = q.z; r.z = q.w; return r; }

__device__ __forceinline__ RowCtx row_ctx(const Ws& w, int a, int b) {
  RowCtx c;
  c.a = a; c.b = b;
  c.ima = a >= 0 ? w.bx[a].w : 0.f;
  c.imb = b >= 0 ? w.bx[b].w : 0.f;
  c.sa = a >= 0 ? w.bIw1[a].z : 1.f;
  c.sb = b >= 0 ? w.bIw1[b].z : 1.f;
  if (a >= 0) c.Ia = load_Iw(w, a);
  if (b >= 0) c.Ib = load_Iw(w, b);
  return c;
}

// Row geometry before the mass terms: la (lb = -la), aa, ab, bias, the soft
// constraint's gamma and the clamp code. Templated on the scalar so that the
// adjoint can differentiate it with dual numbers.
template <class T> struct GRow { V3<T> la, aa, ab; T bias; float gamma; float clamp; };

template <class T> __device__ __forceinline__ GRow<T> g_lin(const V3<T>& u, const V3<T>& ra, const V3<T>& rb) {
  GRow<T> r;
  r.la = -u; r.aa = -cross(ra, u); r.ab = cross(rb, u);
  r.bias = T(0.f); r.gamma = 0.f; r.clamp = CLAMP_FREE;
  return r;
}
template <class T> __device__ __forceinline__ GRow<T> g_ang(const V3<T>& u) {
  GRow<T> r;
  r.la = v3<T>(T(0.f), T(0.f), T(0.f)); r.aa = -u; r.ab = u;
  r.bias = T(0.f); r.gamma = 0.f; r.clamp = CLAMP_FREE;
  return r;
}
// Catto (2011) soft constraint: gamma = 1/(h(d + h k)), bias = (h k/(d + h k))/h * C.
template <class T> __device__ __forceinline__ void g_soft(GRow<T>& r, float h, T C, float k, float d, float fmax) {
  float den = d + h * k;
  r.gamma = 1.f / (h * den);
  r.bias = T((h * k / den) / h) * C;
  r.clamp = fmax * h;
}
template <class T> __device__ __forceinline__ Q4<T> tq(const float* q) { Q4<T> r; r.w = T(q[0]); r.x = T(q[1]); r.y = T(q[2]); r.z = T(q[3]); return r; }
template <class T> __device__ __forceinline__ V3<T> tv(const float* v) { return v3<T>(T(v[0]), T(v[1]), T(v[2])); }

// Joint rows from the poses of the parent (when hasA) and the child and the
// joint's targets tgt[0..ndof). Returns the row count.
template <class T>
__device__ int joint_geom(const JointDesc& j, bool hasA, const V3<T>& xa, const Q4<T>& qa, const V3<T>& xb,
                          const Q4<T>& qb, const T* tgt, float h, float jbeta, GRow<T>* rows) {
  const float beta = jbeta / h;
  V3<T> pa_l = tv<T>(j.pa), pb_l = tv<T>(j.pb);
  V3<T> ra, pa_w, xA;
  Q4<T> qFA;
  if (hasA) {
    xA = xa;
    ra = mul(qmat(qa), pa_l);
    pa_w = xa + ra;
    qFA = qmul(qa, tq<T>(j.qa));
  } else {
    xA = pa_l; ra = v3<T>(T(0.f), T(0.f), T(0.f)); pa_w = pa_l; qFA = tq<T>(j.qa);
  }
  V3<T> rb = mul(qmat(qb), pb_l);
  V3<T> pb_w = xb + rb;
  Q4<T> qFB = qmul(qb, tq<T>(j.qb));
  M3<T> MF = qmat(qFA);
  V3<T> ux = col(MF, 0), uy = col(MF, 1), uz = col(MF, 2);
  V3<T> dp = pb_w - pa_w;
  Q4<T> qr = qmul(qconj(qFA), qFB);
  if (qr.w < T(0.f)) { qr.w = -qr.w; qr.x = -qr.x; qr.y = -qr.y; qr.z = -qr.z; }
  V3<T> raB = hasA ? pb_w - xA : v3<T>(T(0.f), T(0.f), T(0.f));
  int n = 0;
  const bool drive = j.k > 0.f || j.d > 0.f;
  const T tb = T(beta);
  if (j.type == JT_REVOLUTE) {
    for (int c = 0; c < 3; ++c) {
      GRow<T> r = g_lin(unit<T>(c), ra, rb);
      r.bias = tb * comp(dp, c);
      rows[n++] = r;
    }
    V3<T> cr = cross(ux, col(qmat(qFB), 0));
    GRow<T> r1 = g_ang(uy); r1.bias = tb * dot(cr, uy); rows[n++] = r1;
    GRow<T> r2 = g_ang(uz); r2.bias = tb * dot(cr, uz); rows[n++] = r2;
    if (drive) {
      GRow<T> r = g_ang(ux);
      T theta = T(2.f) * atan2_(qr.x, qr.w);
      g_soft(r, h, theta - tgt[0], j.k, j.d, j.fmax);
      rows[n++] = r;
    }
    if (j.lo < j.hi) {   // hinge angle limits (unilateral, speculative like the prismatic limits)
      T theta = T(2.f) * atan2_(qr.x, qr.w);
      for (int c = 0; c < 2; ++c) {
        GRow<T> r = g_ang(c == 0 ? ux : -ux);
        T C = c == 0 ? theta - T(j.lo) : T(j.hi) - theta;
        r.bias = C > T(0.f) ? C / T(h) : tb * C;
        r.clamp = CLAMP_UNI;
        rows[n++] = r;
      }
    }
  } else if (j.type == JT_PRISMATIC) {
    V3<T> us[2] = {uy, uz};
    for (int c = 0; c < 2; ++c) {
      GRow<T> r = g_lin(us[c], raB, rb);
      r.bias = tb * dot(dp, us[c]);
      rows[n++] = r;
    }
    V3<T> ua[3] = {ux, uy, uz};
    T qv[3] = {qr.x, qr.y, qr.z};
    for (int c = 0; c < 3; ++c) {
      GRow<T> r = g_ang(ua[c]);
      r.bias = tb * (T(2.f) * qv[c]);
      rows[n++] = r;
    }
    T dd = dot(dp, ux);
    if (drive) {
      GRow<T> r = g_lin(ux, raB, rb);
      g_soft(r, h, dd - tgt[0], j.k, j.d, j.fmax);
      rows[n++] = r;
    }
    for (int c = 0; c < 2; ++c) {
      GRow<T> r = g_lin(c == 0 ? ux : -ux, raB, rb);
      T C = c == 0 ? dd - T(j.lo) : T(j.hi) - dd;
      r.bias = C > T(0.f) ? C / T(h) : tb * C;
      r.clamp = CLAMP_UNI;
      rows[n++] = r;
    }
  } else {
    {
      GRow<T> r = g_lin(uz, raB, rb);
      r.bias = tb * dot(dp, uz);
      rows[n++] = r;
    }
    V3<T> cr = cross(uz, col(qmat(qFB), 2));
    V3<T> us[2] = {ux, uy};
    for (int c = 0; c < 2; ++c) {
      GRow<T> r = g_ang(us[c]);
      r.bias = tb * dot(cr, us[c]);
      rows[n++] = r;
    }
    if (drive) {
      for (int c = 0; c < 2; ++c) {
        GRow<T> r = g_lin(us[c], raB, rb);
        g_soft(r, h, dot(dp, us[c]) - tgt[c], j.k, j.d, j.fmax);
        rows[n++] = r;
      }
      GRow<T> r = g_ang(uz);
      T theta = T(2.f) * atan2_(qr.z, qr.w);
      g_soft(r, h, theta - tgt[2], j.k, j.d, j.fmax);
      rows[n++] = r;
    }
  }
  return n;
}

__device__ __forceinline__ int joint_ndof(int type) { return type == JT_PLANAR ? 3 : 1; }

static __device__ void joint_rows(const Params& p, const EnvInfo& e, const Ws& w, int k) {
  const JointDesc& j = p.joints[e.j0 + k];
  const int A = j.parent, B = j.child;
  RowCtx ctx = row_ctx(w, A, B);
  float tg[3] = {0.f, 0.f, 0.f};
  if (p.targets && (j.k > 0.f || j.d > 0.f))
    for (int c = 0; c < joint_ndof(j.type); ++c) tg[c] = p.targets[(size_t)e.env * p.max_dof + j.dof + c];
  V3<float> xa = A >= 0 ? f3(w.bx[A]) : v3<float>(0.f, 0.f, 0.f);
  Q4<float> qa = A >= 0 ? ldq4(w.bq[A]) : ldq4(make_float4(1.f, 0.f, 0.f, 0.f));
  GRow<float> g[ROWS_PER_JOINT];
  int n = joint_geom<float>(j, A >= 0, xa, qa, f3(w.bx[B]), ldq4(w.bq[B]), tg, p.h, p.jbeta, g);
  float4* rows = w.jr + (size_t)j.roff * ROW_F4;
  for (int r = 0; r < n; ++r) {
    JRow x = blank_row();
    x.la = g[r].la; x.lb = -g[r].la; x.aa = g[r].aa; x.ab = g[r].ab;
    x.bias = g[r].bias; x.gamma = g[r].gamma;
    const bool soft = g[r].clamp >= 0.f;
    if (soft) { x.lo = -g[r].clamp; x.hi = g[r].clamp; }
    else if (g[r].clamp == CLAMP_UNI) { x.lo = 0.f; x.hi = INFINITY; }
    finish_row(x, ctx, soft);
    put_row(rows + ROW_F4 * r, x);
  }
}

// Duff et al. (2017) orthonormal basis from a unit normal: the scale
// a = -1/(sign(n_z) + n_z), then the two tangents from it. The solver keeps a
// per contact point, so its sweeps form the tangents without the division.
template <class T> __device__ __forceinline__ T onb_scale(const V3<T>& n) {
  T sg = n.z >= T(0.f) ? T(1.f) : T(-1.f);
  return T(-1.f) / (sg + n.z);
}
template <class T> __device__ __forceinline__ void onb_with(const V3<T>& n, T a, V3<T>& t1, V3<T>& t2) {
  T sg = n.z >= T(0.f) ? T(1.f) : T(-1.f);
  T b = n.x * n.y * a;
  t1 = v3<T>(T(1.f) + sg * n.x * n.x * a, sg * b, -sg * n.x);
  t2 = v3<T>(b, sg + n.y * n.y * a, -n.y);
}
template <class T> __device__ __forceinline__ void onb(const V3<T>& n, V3<T>& t1, V3<T>& t2) {
  onb_with(n, onb_scale(n), t1, t2);
}

// World lever arms and speculative bias of one contact point from the body
// poses and the point's normal and anchors (rb_l is world space for a static b).
template <class T>
__device__ __forceinline__ void contact_geom(const V3<T>& xa, const Q4<T>& qa, const V3<T>& xb, const Q4<T>& qb,
                                             bool bdyn, const V3<T>& n, const V3<T>& ra_l, const V3<T>& rb_l, float h,
                                             float beta, float slop, V3<T>& ra, V3<T>& rb, T& bias) {
  ra = mul(qmat(qa), ra_l);
  V3<T> pa_w = xa + ra;
  V3<T> pb_w;
  if (bdyn) { rb = mul(qmat(qb), rb_l); pb_w = xb + rb; }
  else { pb_w = rb_l; rb = v3<T>(T(0.f), T(0.f), T(0.f)); }
  T s = dot(n, pb_w - pa_w);
  bias = s > T(0.f) ? s / T(h) : -T(beta / h) * maxv(T(0.f), -s - T(slop));
}

// The 3x3 matrix K(x, y) = J_x M^-1 J_y^T of a contact point over its rows
// x, y in (n, t1, t2) (d[0..2]): K[0..2] its diagonal, K[3..5] = K(t1, n),
// K(t2, n), K(t2, t1). The lever terms r x d and their images under the
// inverse inertias are formed once per row and shared by the entries.
__device__ __forceinline__ void point_K(const RowCtx& ctx, const V3<float>* d, const V3<float>& ra,
                                        const V3<float>& rb, float* K) {
  V3<float> la[3], ma[3], lb[3], mb[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    la[r] = crossf(ra, d[r]); ma[r] = smulf(ctx.Ia, la[r]);
    if (ctx.b >= 0) { lb[r] = crossf(rb, d[r]); mb[r] = smulf(ctx.Ib, lb[r]); }
  }
  const int I[6] = {0, 1, 2, 1, 2, 2}, J[6] = {0, 1, 2, 0, 0, 1};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int i = I[q], j = J[q];
    float k = fmaf(ctx.sa, fmaf(ctx.ima, dotf(d[i], d[j]), dotf(la[i], ma[j])), 0.f);
    if (ctx.b >= 0) k = fmaf(ctx.sb, fmaf(ctx.imb, dotf(d[i], d[j]), dotf(lb[i], mb[j])), k);
    K[q] = k;
  }
}

// BK: the kind of b (BK_STATIC: its pose, velocity and inertia terms drop
// out at compile time).
template <int BK>
__device__ __forceinline__ void contact_rows_t(const Params& p, const Ws& w, int ci, int a, int bd) {
  const int b = BK == BK_STATIC ? -1 : bd;
  const bool bdyn = b_dyn<BK>(b >= 0);
  RowCtx ctx = row_ctx(w, a, b);
  V3<float> n = f3(w.cn[ci]);
  V3<float> ra, rb;
  float bias;
  V3<float> xb = bdyn ? f3(w.bx[b]) : v3<float>(0.f, 0.f, 0.f);
  Q4<float> qb = bdyn ? ldq4(w.bq[b]) : ldq4(make_float4(1.f, 0.f, 0.f, 0.f));
  contact_geom<float>(f3(w.bx[a]), ldq4(w.bq[a]), xb, qb, bdyn, n, f3(w.cra[ci]), f3(w.crb[ci]), p.h, p.beta,
                      p.slop, ra, rb, bias);
  if (p.rest > 0.f) {
    V3<float> va = f3(w.bv[a]), wa = f3(w.bw[a]);
    V3<float> dv = v3<float>(0.f, 0.f, 0.f) - (va + cross(wa, ra));
    if (bdyn) dv = dv + (f3(w.bv[b]) + cross(f3(w.bw[b]), rb));
    float vn = dot(n, dv);
    if (vn < -1.f) bias = fminf(bias, p.rest * vn);
  }
  V3<float> t1, t2;
  const float sc = onb_scale(n);
  onb_with(n, sc, t1, t2);
  const V3<float> d[3] = {n, t1, t2};
  float K[6];
  point_K(ctx, d, ra, rb, K);
  auto inv = [](float k) { return k > 0.f ? 1.f / k : 0.f; };
  w.kra[ci] = f4(ra, inv(K[0]));
  w.krb[ci] = f4(rb, bias);
  w.klam[ci] = make_float4(0.f, 0.f, 0.f, inv(K[1]));
  w.cn[ci].w = inv(K[2]);   // the separation s0 is not needed after the narrowphase
  w.kx[ci] = make_float4(K[3], K[4], K[5], sc);
}

static __device__ void contact_rows(const Params& p, const EnvInfo& e, const Ws& w, int ci) {
  int ids = w.cid[ci];
  int a = ids & 0xffff, bc = ids >> 16;
  const int b = bc < e.D ? bc : -1;
  // two kinds only: a third copy for lanes that differ grew the fused step's
  // stack frame (1008 -> 1072 bytes) and its DRAM writes (12 -> 18 MB per
  // launch at 4096 envs), and the set-up runs once per substep
  if (b >= 0) contact_rows_t<BK_DYNAMIC>(p, w, ci, a, b);
  else contact_rows_t<BK_STATIC>(p, w, ci, a, b);
}

static __device__ void stage_prep(const Params& p, const EnvInfo& e, const Ws& w) {
  const int nc = w.misc[MC_CONTACTS];
  // joints, then contacts: two loops, so that a round of threads takes one kind
  for (int t = e.lane; t < e.J; t += e.nthr) joint_rows(p, e, w, t);
  for (int t = e.lane; t < nc; t += e.nthr) contact_rows(p, e, w, t);
}

// ---------------------------------------------------------------------------
// a6: solver
// ---------------------------------------------------------------------------
struct BodyVel { V3<float> va, wa, vb, wb; };

// Joint rows on velocities (va, wa, vb, wb); `sa`/`sb` scale the inverse
// masses applied to the local copies (Jacobi mass splitting, 1 in PGS); the
// true-mass change is accumulated in `dacc` when non-null. The relative
// velocity along a row is three independent dot products, so the chain from
// one row's impulse to the next row's velocities stays short.
__device__ __forceinline__ void solve_joint(const Params& p, const EnvInfo& e, const Ws& w, int k, BodyVel& bv,
                                            BodyVel* dacc) {
  const int4 ji = w.jinfo[k];   // parent, child, first row, row count
  const int A = ji.x;
  const float ima = A >= 0 ? w.bIw1[A].w : 0.f, imb = w.bIw1[ji.y].w;
  const float sa = A >= 0 ? w.bIw1[A].z : 1.f, sb = w.bIw1[ji.y].z;
  const float ka = sa * ima, kb = sb * imb;
  const int nr = ji.w;
  float4* rows = w.jr + (size_t)ji.z * ROW_F4;
  float4 r0 = rows[0], r1 = rows[1], r2 = rows[2], r3 = rows[3], r4 = rows[4];
  for (int r = 0; r < nr; ++r) {
    float4* R = rows + ROW_F4 * r;
    float4 n0 = r0, n1 = r1, n2 = r2, n3 = r3, n4 = r4;
    if (r + 1 < nr) { n0 = R[5]; n1 = R[6]; n2 = R[7]; n3 = R[8]; n4 = R[9]; }   // next row, loaded early
    V3<float> la = f3(r0), aa = f3(r1), ab = f3(r2), Ia = f3(r3), Ib = f3(r4);
    // J v = la.(va - vb) + aa.wa + ab.wb  (a static parent has va = wa = 0)
    float jv = dotf(la, bv.va - bv.vb) + dotf(ab, bv.wb) + dotf(aa, bv.wa);
    float lam = r3.w;
    float dl = -r0.w * fmaf(r2.w, lam, jv + r1.w);
    float nl = lam + dl;
    // the clamp as selects, not branches: the lanes of a warp run joints
    // whose rows at the same index have different clamp kinds (4096-env
    // apartment batch: 1.73 against 1.77 ms per step)
    const float cl = r4.w;
    const float hi = cl >= 0.f ? cl : INFINITY;
    const float lo = cl >= 0.f ? -cl : (cl == CLAMP_UNI ? 0.f : -INFINITY);
    nl = cl == CLAMP_FREE ? nl : fminf(fmaxf(nl, lo), hi);
    dl = nl - lam;
    R[3].w = nl;
    if (A >= 0) {
      bv.va = axpyf(bv.va, la, ka * dl);
      bv.wa = axpyf(bv.wa, Ia, sa * dl);
      if (dacc) { dacc->va = axpyf(dacc->va, la, ima * dl); dacc->wa = axpyf(dacc->wa, Ia, dl); }
    }
    bv.vb = axpyf(bv.vb, la, -(kb * dl));
    bv.wb = axpyf(bv.wb, Ib, sb * dl);
    if (dacc) { dacc->vb = axpyf(dacc->vb, la, -(imb * dl)); dacc->wb = axpyf(dacc->wb, Ib, dl); }
    r0 = n0; r1 = n1; r2 = n2; r3 = n3; r4 = n4;
  }
}

// One manifold's points in order, each as a normal row then two friction
// rows (Gauss-Seidel). Per point the velocity of b relative to a at the
// point is formed once; each row's impulse moves the later rows' relative
// velocities by the point's coupling terms (J_x M^-1 J_y^T, fixed within a
// substep), and the point's total impulse is applied to the bodies once.
// This is the row-by-row sequential-impulse update, regrouped. BK: the kind
// of b; a static b (or the plane) has no velocity and takes no impulse, so
// with BK_STATIC its terms drop out of the loop (the same values: with a
// static b the relative velocity is the negated velocity of a, as in the
// general form). Nearly every manifold of the apartment and manipulator
// batches has a static b, so their warps mostly run the shorter loop
// (4096-env apartment batch: 1.72 -> 1.69 ms per step; 1024-env manipulator
// batch: 0.648 -> 0.606 ms).
template <int BK>
__device__ __forceinline__ void manifold_points(const Params& p, const Ws& w, int4 mf, BodyVel& bv, BodyVel* dacc,
                                                float4* tq, float ima, float imb, float sa, float sb, float ka,
                                                float kb, const Sym3& Ia, const Sym3& Ib) {
  const bool bdyn = b_dyn<BK>(mf.y >= 0);
  const int c1 = mf.z + mf.w;
  // software pipelining: the next point's data is loaded while this point's rows run
  float4 cn = w.cn[mf.z], kra = w.kra[mf.z], krb = w.krb[mf.z], lam = w.klam[mf.z], kx = w.kx[mf.z];
  for (int c = mf.z; c < c1; ++c) {
    float4 ncn = cn, nkra = kra, nkrb = krb, nlam = lam, nkx = kx;
    if (c + 1 < c1) {
      ncn = w.cn[c + 1]; nkra = w.kra[c + 1]; nkrb = w.krb[c + 1]; nlam = w.klam[c + 1]; nkx = w.kx[c + 1];
    }
    const V3<float> n = f3(cn), ra = f3(kra), rb = f3(krb);
    V3<float> t1, t2;
    onb_with(n, kx.w, t1, t2);
    // velocity of b relative to a at the point (static b: vb = wb = 0)
    V3<float> vr = bv.va + crossf(bv.wa, ra);
    vr = bdyn ? (bv.vb + crossf(bv.wb, rb)) - vr : -vr;
    float u0 = dotf(n, vr), u1 = dotf(t1, vr), u2 = dotf(t2, vr);
    const float l0 = lam.x, l1 = lam.y, l2 = lam.z;
    const float nl0 = fmaxf(l0 + -kra.w * (u0 + krb.w), 0.f);
    const float d0 = nl0 - l0;
    u1 = fmaf(kx.x, d0, u1);
    u2 = fmaf(kx.y, d0, u2);
    const float lim = p.mu * nl0;
    const float nl1 = fminf(fmaxf(l1 + -lam.w * u1, -lim), lim);
    const float d1 = nl1 - l1;
    u2 = fmaf(kx.z, d1, u2);
    const float nl2 = fminf(fmaxf(l2 + -cn.w * u2, -lim), lim);
    const float d2 = nl2 - l2;
    w.klam[c] = make_float4(nl0, nl1, nl2, lam.w);
    if (tq) tq[c] = make_float4(nl0, nl1, nl2, 0.f);   // the recorded sweep's slot of this point
    // the point's impulse on b (its negative on a)
    const V3<float> P = axpyf(axpyf(n * d0, t1, d1), t2, d2);
    const V3<float> ia = smulf(Ia, crossf(ra, P));
    bv.va = axpyf(bv.va, P, -ka);
    bv.wa = axpyf(bv.wa, ia, -sa);
    if (dacc) { dacc->va = axpyf(dacc->va, P, -ima); dacc->wa = dacc->wa - ia; }
    if (bdyn) {
      const V3<float> ib = smulf(Ib, crossf(rb, P));
      bv.vb = axpyf(bv.vb, P, kb);
      bv.wb = axpyf(bv.wb, ib, sb);
      if (dacc) { dacc->vb = axpyf(dacc->vb, P, imb); dacc->wb = dacc->wb + ib; }
    }
    cn = ncn; kra = nkra; krb = nkrb; lam = nlam; kx = nkx;
  }
}

__device__ __forceinline__ void solve_manifold(const Params& p, const EnvInfo& e, const Ws& w, int m, BodyVel& bv,
                                               BodyVel* dacc, float4* tq = nullptr) {
  int4 mf = man_get(w, m);
  const int a = mf.x, b = mf.y;
  const float ima = w.bIw1[a].w, imb = b >= 0 ? w.bIw1[b].w : 0.f;
  const float sa = w.bIw1[a].z, sb = b >= 0 ? w.bIw1[b].z : 1.f;
  const float ka = sa * ima, kb = sb * imb;
  const Sym3 Ia = load_Iw(w, a);
  const Sym3 Ib = b >= 0 ? load_Iw(w, b) : Ia;
  by_b_kind(b >= 0, [&](auto k) {
    manifold_points<decltype(k)::v>(p, w, mf, bv, dacc, tq, ima, imb, sa, sb, ka, kb, Ia, Ib);
  });
}

// One manifold in a coloured sweep: its bodies' velocities, its points, the
// velocities back (BK as in manifold_points; a static b has none).
template <int BK>
__device__ __forceinline__ void sweep_manifold(const Params& p, const Ws& w, int4 mf, float4* tq) {
  const int a = mf.x, b = mf.y;
  const bool bdyn = b_dyn<BK>(b >= 0);
  const V3<float> z = v3<float>(0.f, 0.f, 0.f);
  BodyVel bv;
  bv.va = f3(w.bv[a]); bv.wa = f3(w.bw[a]);
  bv.vb = bdyn ? f3(w.bv[b]) : z; bv.wb = bdyn ? f3(w.bw[b]) : z;
  const float4 xa = w.bIw1[a];
  const float4 xb = bdyn ? w.bIw1[b] : make_float4(0.f, 0.f, 1.f, 0.f);
  const float ima = xa.w, imb = xb.w, sa = xa.z, sb = xb.z;
  const Sym3 Ia = load_Iw(w, a);
  manifold_points<BK>(p, w, mf, bv, nullptr, tq, ima, imb, sa, sb, sa * ima, sb * imb, Ia,
                      bdyn ? load_Iw(w, b) : Ia);
  w.bv[a] = f4(bv.va, 0.f); w.bw[a] = f4(bv.wa, 0.f);
  if (bdyn) { w.bv[b] = f4(bv.vb, 0.f); w.bw[b] = f4(bv.wb, 0.f); }
}

__device__ __forceinline__ void con_bodies(const Params& p, const EnvInfo& e, const Ws& w, int k, int J, int& a, int& b) {
  if (k < J) { int4 ji = w.jinfo[k]; a = ji.x; b = ji.y; }
  else { int4 m = man_get(w, k - J); a = m.x; b = m.y; }
}

__device__ __forceinline__ BodyVel load_vel(const Ws& w, int a, int b) {
  BodyVel v;
  V3<float> z = v3<float>(0.f, 0.f, 0.f);
  v.va = a >= 0 ? f3(w.bv[a]) : z; v.wa = a >= 0 ? f3(w.bw[a]) : z;
  v.vb = b >= 0 ? f3(w.bv[b]) : z; v.wb = b >= 0 ? f3(w.bw[b]) : z;
  return v;
}

// Records the lambdas of constraint k after its update in sweep `it`: a
// joint's 8 row slots as two 16-byte stores (unused slots 0), a contact
// point's three rows as one (4 slots per point, the last 0). The sweep's
// record starts on 16 bytes (tape slab, t2 and tape_Rm are multiples of 4
// floats), so these are aligned vector stores rather than scattered words.
__device__ __forceinline__ void tape_lambdas(const Params& p, const EnvInfo& e, const Ws& w, int k, int sub, int it) {
  TapeLayout tl = tape_layout(p.L, p.S, p.N, p.max_dof);
  float* t = tape_env(p, e.env) + tl.t2 + (long long)(sub * p.N + it) * p.tape_Rm;
  if (k < e.J) {
    const int4 ji = w.jinfo[k];   // first row, row count
    const float4* rows = w.jr + (size_t)ji.z * ROW_F4;
    float v[ROWS_PER_JOINT];
#pragma unroll
    for (int r = 0; r < ROWS_PER_JOINT; ++r) v[r] = r < ji.w ? rows[ROW_F4 * r + 3].w : 0.f;
    float4* q = reinterpret_cast<float4*>(t + k * ROWS_PER_JOINT);
    q[0] = make_float4(v[0], v[1], v[2], v[3]);
    q[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else {
    int4 mf = man_get(w, k - e.J);
    float4* q = reinterpret_cast<float4*>(t + ROWS_PER_JOINT * p.L.Jm);
    for (int c = mf.z; c < mf.z + mf.w; ++c) {
      const float4 l = w.klam[c];
      q[c] = make_float4(l.x, l.y, l.z, 0.f);
    }
  }
}

// One solver iteration over every constraint of the env.
static __device__ void stage_solve_iter(const Params& p, const EnvInfo& e, const Ws& w, int sub, int it) {
  const int J = e.J;
  if (p.mode == MODE_COLOURED) {
    const int ncol = w.misc[MC_COLOURS];
    // a recorded step: this sweep's contact-point slots (4 per point, on 16
    // bytes), written by the point update from its registers
    float4* tq = nullptr;
    if (p.tape) {
      const TapeLayout tl = tape_layout(p.L, p.S, p.N, p.max_dof);
      tq = reinterpret_cast<float4*>(tape_env(p, e.env) + tl.t2 + (long long)(sub * p.N + it) * p.tape_Rm +
                                     ROWS_PER_JOINT * p.L.Jm);
    }
    for (int c = 0; c < ncol; ++c) {
      // the colour's joints, then its manifolds (no barrier between: a
      // colour's constraints share no dynamic body)
      const int v = w.coff[c], c0 = v & 0xffff, cm = c0 + (v >> 16), c1 = w.coff[c + 1] & 0xffff;
      for (int idx = c0 + e.lane; idx < cm; idx += e.nthr) {
        const int k = w.corder[idx];
        const int4 ji = w.jinfo[k];
        BodyVel bv = load_vel(w, ji.x, ji.y);
        solve_joint(p, e, w, k, bv, nullptr);
        if (ji.x >= 0) { w.bv[ji.x] = f4(bv.va, 0.f); w.bw[ji.x] = f4(bv.wa, 0.f); }
        w.bv[ji.y] = f4(bv.vb, 0.f); w.bw[ji.y] = f4(bv.wb, 0.f);
        if (p.tape) tape_lambdas(p, e, w, k, sub, it);
      }
      for (int idx = cm + e.lane; idx < c1; idx += e.nthr) {
        const int4 mf = man_get(w, w.corder[idx] - J);
        by_b_kind(mf.y >= 0, [&](auto k) { sweep_manifold<decltype(k)::v>(p, w, mf, tq); });
      }
      gsync(e);
    }
  } else {
    const int K = J + w.misc[MC_MANIFOLDS];
    for (int k = e.lane; k < K; k += e.nthr) {
      int a, b;
      con_bodies(p, e, w, k, J, a, b);
      BodyVel bv = load_vel(w, a, b);
      BodyVel d;
      V3<float> z = v3<float>(0.f, 0.f, 0.f);
      d.va = z; d.wa = z; d.vb = z; d.wb = z;
      if (k < J) solve_joint(p, e, w, k, bv, &d);
      else solve_manifold(p, e, w, k - J, bv, &d);
      w.jdv[4 * k + 0] = f4(d.va, 0.f); w.jdv[4 * k + 1] = f4(d.wa, 0.f);
      w.jdv[4 * k + 2] = f4(d.vb, 0.f); w.jdv[4 * k + 3] = f4(d.wb, 0.f);
      if (p.tape) tape_lambdas(p, e, w, k, sub, it);
    }
    gsync(e);
    for (int i = e.lane; i < e.D; i += e.nthr) {
      V3<float> dv = v3<float>(0.f, 0.f, 0.f), dw = dv;
      for (int q = w.inc_off[i]; q < w.inc_off[i + 1]; ++q) {
        int t = w.inc[q];
        int k = t >> 1, side = t & 1;
        dv = dv + f3(w.jdv[4 * k + 2 * side]);
        dw = dw + f3(w.jdv[4 * k + 2 * side + 1]);
      }
      w.bv[i] = f4(f3(w.bv[i]) + dv, 0.f);
      w.bw[i] = f4(f3(w.bw[i]) + dw, 0.f);
    }
    gsync(e);
  }
}

// ---------------------------------------------------------------------------
// a7: positions
// ---------------------------------------------------------------------------
static __device__ void stage_integrate_pos(const Params& p, const EnvInfo& e, const Ws& w, int sub) {
  for (int i = e.lane; i < e.D; i += e.nthr) {
    float4 x = w.bx[i], v = w.bv[i], wv = w.bw[i], q = w.bq[i];
    if (p.tape) {
      TapeLayout tl = tape_layout(p.L, p.S, p.N, p.max_dof);
      float* t = tape_env(p, e.env) + tl.t1 + 19LL * (sub * p.L.Dm + i) + 13;
      t[0] = v.x; t[1] = v.y; t[2] = v.z; t[3] = wv.x; t[4] = wv.y; t[5] = wv.z;
    }
    x.x = fmaf(v.x, p.h, x.x); x.y = fmaf(v.y, p.h, x.y); x.z = fmaf(v.z, p.h, x.z);
    Q4<float> wq; wq.w = 0.f; wq.x = wv.x; wq.y = wv.y; wq.z = wv.z;
    Q4<float> dq = qmul(wq, ldq4(q));
    float hh = p.h * 0.5f;
    float qw = fmaf(dq.w, hh, q.x), qx = fmaf(dq.x, hh, q.y), qy = fmaf(dq.y, hh, q.z), qz = fmaf(dq.z, hh, q.w);
    float nrm = sqrtf(fmaf(qw, qw, fmaf(qx, qx, fmaf(qy, qy, qz * qz))));
    w.bx[i] = x;
    w.bq[i] = make_float4(qw / nrm, qx / nrm, qy / nrm, qz / nrm);
  }
}

// ---------------------------------------------------------------------------
// Contact report (optional, once per step). The paper's success conditions
// and event labels (Sec. 3.3, Appendix A.4-A.5) use pairwise contact forces,
// the robot's cumulative collision force and a grasp indicator; the readings
// (identical in the oracle):
//   * contact c's force on its second body is its impulse (l_n n + l_t1 t1 +
//     l_t2 t2) summed over the step's substeps, divided by dt; the first body
//     receives the opposite;
//   * a step's robot collision force is the sum over robot links of the norm
//     of each link's net force from contacts with static boxes and with bodies
//     that are neither robot links nor the target;
//   * grasped: both fingers feel a force of at least f_min from the target,
//     within theta_max of the finger's opening direction (F.o >= cos |F||o|).
// ---------------------------------------------------------------------------
// After substep `sub`'s sweeps: add each contact's lambdas to its impulse sum.
static __device__ void stage_accum_impulse(const Params& p, const EnvInfo& e, const Ws& w, int sub) {
  if (!p.rep_on) return;
  const int nc = w.misc[MC_CONTACTS];
  for (int c = e.lane; c < nc; c += e.nthr) {
    const float4 l = w.klam[c];
    const float4 a = sub == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : w.crep[c];
    w.crep[c] = make_float4(a.x + l.x, a.y + l.y, a.z + l.z, 0.f);
  }
}

__device__ __forceinline__ float norm3f(float x, float y, float z) { return sqrtf(x * x + y * y + z * z); }

__device__ __forceinline__ bool rep_counts(const Params& p, const EnvInfo& e, int other, int target) {
  if (other >= e.D) return other < e.D + e.S;   // static boxes count, the plane does not
  return !(p.rep_flags[e.b0 + other] & 1) && other != target;
}

// At the end of the step (final poses); plain float arithmetic in the
// oracle's order (the library is built without FMA contraction).
static __device__ void stage_report(const Params& p, const EnvInfo& e, const Ws& w) {
  if (!p.rep_on) return;
  const int nc = w.misc[MC_CONTACTS];
  const int D = e.D;
  const int target = p.rep_target ? p.rep_target[e.env] : -1;
  for (int c = e.lane; c < nc; c += e.nthr) {
    const float4 n4 = w.cn[c], L = w.crep[c];
    V3<float> n = f3(n4), t1, t2;
    onb(n, t1, t2);
    const float px = (n.x * L.x + t1.x * L.y) + t2.x * L.z;
    const float py = (n.y * L.x + t1.y * L.y) + t2.y * L.z;
    const float pz = (n.z * L.x + t1.z * L.y) + t2.z * L.z;
    w.crep[c] = make_float4(px / p.dt, py / p.dt, pz / p.dt, 0.f);   // force on the second body
  }
  gsync(e);
  for (int i = e.lane; i < D; i += e.nthr) {
    const bool robot = p.rep_flags[e.b0 + i] & 1;
    float fx = 0.f, fy = 0.f, fz = 0.f, rx = 0.f, ry = 0.f, rz = 0.f;
    for (int c = 0; c < nc; ++c) {
      const int id = w.cid[c], a = id & 0xffff, b = id >> 16;
      if (a != i && b != i) continue;
      const float4 F = w.crep[c];
      if (a == i) {
        fx = fx - F.x; fy = fy - F.y; fz = fz - F.z;
        if (robot && rep_counts(p, e, b, target)) { rx = rx - F.x; ry = ry - F.y; rz = rz - F.z; }
      } else {
        fx = fx + F.x; fy = fy + F.y; fz = fz + F.z;
        if (robot && rep_counts(p, e, a, target)) { rx = rx + F.x; ry = ry + F.y; rz = rz + F.z; }
      }
    }
    if (p.rep_body_force) {
      float* o = p.rep_body_force + 3 * (size_t)(e.b0 + i);
      o[0] = fx; o[1] = fy; o[2] = fz;
    }
    w.bIw0[i] = make_float4(rx, ry, rz, 0.f);   // free after the last substep
  }
  gsync(e);
  if (e.lane == 0) {
    float inc = 0.f;
    for (int i = 0; i < D; ++i)
      if (p.rep_flags[e.b0 + i] & 1) { const float4 r = w.bIw0[i]; inc = inc + norm3f(r.x, r.y, r.z); }
    if (p.rep_robot_force) p.rep_robot_force[e.env] = p.rep_robot_force[e.env] + inc;
    const int f0 = p.rep_fingers ? p.rep_fingers[2 * e.env] : -1;
    const int f1 = p.rep_fingers ? p.rep_fingers[2 * e.env + 1] : -1;
    const int fing[2] = {f0, f1};
    float T[3] = {0.f, 0.f, 0.f}, Fg[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    if (target >= 0) {
      for (int c = 0; c < nc; ++c) {
        const int id = w.cid[c], a = id & 0xffff, b = id >> 16;
        const float4 F = w.crep[c];
        const bool ee_a = a < D && (p.rep_flags[e.b0 + a] & 2), ee_b = b < D && (p.rep_flags[e.b0 + b] & 2);
        if (ee_a && b == target) { T[0] = T[0] + F.x; T[1] = T[1] + F.y; T[2] = T[2] + F.z; }
        if (ee_b && a == target) { T[0] = T[0] - F.x; T[1] = T[1] - F.y; T[2] = T[2] - F.z; }
        for (int f = 0; f < 2; ++f) {
          if (fing[f] < 0) continue;
          if (a == fing[f] && b == target) { Fg[f][0] = Fg[f][0] - F.x; Fg[f][1] = Fg[f][1] - F.y; Fg[f][2] = Fg[f][2] - F.z; }
          if (b == fing[f] && a == target) { Fg[f][0] = Fg[f][0] + F.x; Fg[f][1] = Fg[f][1] + F.y; Fg[f][2] = Fg[f][2] + F.z; }
        }
      }
    }
    int grasped = 0;
    if (target >= 0 && f0 >= 0 && f1 >= 0) {
      int ok = 1;
      for (int f = 0; f < 2; ++f) {
        const float4 xa = w.bx[fing[f]], xb = w.bx[fing[1 - f]];
        const float ox = xa.x - xb.x, oy = xa.y - xb.y, oz = xa.z - xb.z;   // opening direction
        const float fn = norm3f(Fg[f][0], Fg[f][1], Fg[f][2]), on = norm3f(ox, oy, oz);
        const float d = Fg[f][0] * ox + Fg[f][1] * oy + Fg[f][2] * oz;
        if (!(fn >= p.rep_fmin) || !(d >= p.rep_cosmax * fn * on)) ok = 0;
      }
      grasped = ok;
    }
    if (p.rep_target_force) {
      float* o = p.rep_target_force + 3 * (size_t)e.env;
      o[0] = T[0]; o[1] = T[1]; o[2] = T[2];
    }
    if (p.rep_finger_force) {
      float* o = p.rep_finger_force + 6 * (size_t)e.env;
      for (int f = 0; f < 2; ++f) { o[3 * f] = Fg[f][0]; o[3 * f + 1] = Fg[f][1]; o[3 * f + 2] = Fg[f][2]; }
    }
    if (p.rep_grasped) p.rep_grasped[e.env] = grasped;
  }
  gsync(e);
}

// ---------------------------------------------------------------------------
// a8: write back, status
// ---------------------------------------------------------------------------
static __device__ void stage_store(const Params& p, const EnvInfo& e, const Ws& w) {
  int bad = 0;
  for (int i = e.lane; i < e.D; i += e.nthr) {
    int g = e.b0 + i;
    float4 x = w.bx[i], q = w.bq[i], v = w.bv[i], wv = w.bw[i];
    p.pos[3 * g] = x.x; p.pos[3 * g + 1] = x.y; p.pos[3 * g + 2] = x.z;
    p.quat[4 * g] = q.x; p.quat[4 * g + 1] = q.y; p.quat[4 * g + 2] = q.z; p.quat[4 * g + 3] = q.w;
    p.lv[3 * g] = v.x; p.lv[3 * g + 1] = v.y; p.lv[3 * g + 2] = v.z;
    p.av[3 * g] = wv.x; p.av[3 * g + 1] = wv.y; p.av[3 * g + 2] = wv.z;
    float s = x.x + x.y + x.z + q.x + q.y + q.z + q.w + v.x + v.y + v.z + wv.x + wv.y + wv.z;
    if (!isfinite(s)) bad = 1;
  }
  bad = gany(e, bad);
  if (e.lane == 0) {
    int st = w.misc[MC_STATUS] | (bad ? ST_NONFINITE : 0);
    if (st) p.status[e.env] |= st;
  }
}

}  // namespace msh
