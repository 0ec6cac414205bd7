// Kernels and C ABI of the batched rigid-body step (see include/msh.h).
//
// Two execution forms share the stage functions of msh_stages.cuh:
//   * plain: one launch per stage, one CTA per env, workspace slabs in HBM;
//     per step: load, aabb, broadphase, narrowphase, colour, then per substep
//     integrate-velocity, prep, N solver launches, integrate-position; store.
//   * fused: one persistent launch per step; CTAs take envs from an atomic
//     queue (largest first) and run every stage on a shared-memory workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/msh.h"
#include "msh_render.h"
#include "msh_adjoint.cuh"

using namespace msh;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// One-env slab of the device-memory forms (plain, substep, adjoint): the
// contact arrays are the full-capacity ones of the cold part.
__device__ __forceinline__ Ws plain_ws(const Params& p, int env) {
  char* b = p.ws + (long long)env * p.ws_stride;
  char* cold = b + p.L.hot_bytes;
  Ws w = make_ws(b, cold, p.L);
  w.cn = (float4*)(cold + p.L.cnc); w.kra = (float4*)(cold + p.L.krac);
  w.krb = (float4*)(cold + p.L.krbc); w.klam = (float4*)(cold + p.L.klamc);
  return w;
}

__global__ void k_load(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  stage_load(p, e, plain_ws(p, blockIdx.x));
}
__global__ void k_aabb(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  stage_aabb(p, e, plain_ws(p, blockIdx.x));
}
__global__ void k_broad(Params p) {
  __shared__ int scr[33];
  EnvInfo e = env_info(p, blockIdx.x);
  stage_broadphase(p, e, plain_ws(p, blockIdx.x), scr);
}
__global__ void k_narrow(Params p) {
  __shared__ int scr[33];
  EnvInfo e = env_info(p, blockIdx.x);
  stage_narrowphase(p, e, plain_ws(p, blockIdx.x), scr);
}
__global__ void k_colour(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  const Ws w = plain_ws(p, blockIdx.x);
  stage_colour(p, e, w);
  if (p.tape) tape_collision(p, e, w);
}
__global__ void k_intvel(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  stage_integrate_vel(p, e, plain_ws(p, blockIdx.x), p.sub);
}
__global__ void k_prep(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  stage_prep(p, e, plain_ws(p, blockIdx.x));
}
__global__ void k_solve(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  stage_solve_iter(p, e, plain_ws(p, blockIdx.x), p.sub, p.it);
}
__global__ void k_intpos(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  Ws w = plain_ws(p, blockIdx.x);
  stage_accum_impulse(p, e, w, p.sub);
  stage_integrate_pos(p, e, w, p.sub);
}
__global__ void k_store(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  Ws w = plain_ws(p, blockIdx.x);
  stage_report(p, e, w);
  stage_store(p, e, w);
}
// One whole substep per env (substep-fused form): gravity, rows, N sweeps,
// positions, on the env's HBM workspace.
__global__ void k_substep(Params p) {
  EnvInfo e = env_info(p, blockIdx.x);
  Ws w = plain_ws(p, blockIdx.x);
  stage_integrate_vel(p, e, w, p.sub);
  __syncthreads();
  stage_prep(p, e, w);
  __syncthreads();
  for (int it = 0; it < p.N; ++it) stage_solve_iter(p, e, w, p.sub, it);
  stage_accum_impulse(p, e, w, p.sub);
  stage_integrate_pos(p, e, w, p.sub);
}

#include "msh_fused.cuh"

static FusedKernel fused_kernel(int blk, int tpe, int fl) {
  if (tpe == 16) return fused_kernel_g16(fl);
  if (tpe == 32 && blk == 32) return fused_kernel_g32(fl);
  return blk <= 256 ? fused_kernel_fl<256, 0>(fl) : fused_kernel_fl<512, 0>(fl);
}

// Adjoint of the recorded step in tape slot q.slot (see msh_adjoint.cuh), as
// a sequence of launches that each run one phase for every env: the replay of
// the step's collision stage from the recorded start state, then per substep
// (last first) the reverse of the position update with the row rebuild, the
// reversed sweeps, and the reverse of the row set-up; finally the reverse of
// the narrowphase and the outputs. Every phase keeps its per-env data in the
// device-memory workspaces, so the phases are separate kernels: each gets the
// registers and instruction footprint of its own code instead of the largest
// phase's. A CTA of 32 threads holds 32/G env groups of G threads.
// Asynchronous 16-byte copy from device to shared memory (cp.async; both
// addresses 16-byte aligned), its group commit and the wait for every
// committed group of the thread.
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct BwdEnv {
  EnvInfo e;
  Ws w;
  AWs a;
  const float* tape;
  TapeLayout tl;
};

// GC: threads per env, a compile-time constant of each adjoint kernel (32, or
// 16 in the sweeps of large batches), so that the group's strides, masks and
// barriers fold to constants (a 16-step rollout at 4096 envs: 151 against
// 156 ms with the size read at run time).
template <int GC>
__device__ __forceinline__ bool bwd_env(const Params& p, const AdjParams& q, BwdEnv& b) {
  const int G = GC;
  const int gi = threadIdx.x / G, lane = threadIdx.x % G;
  const unsigned mask = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  // envs in decreasing estimated cost, as the fused step takes them: the
  // costliest start first and the two envs of a warp do similar work
  const int idx = blockIdx.x * (blockDim.x / G) + gi;
  if (idx >= p.E) return false;   // whole groups exit together
  const int env = p.env_order[idx];
  b.e = env_info(p, env, lane, G, mask);
  b.w = plain_ws(p, env);
  b.a = make_aws(q.aws + (long long)env * q.aws_stride, q.A);
  b.tl = tape_layout(p.L, p.S, p.N, p.max_dof);
  b.tape = p.tape + ((long long)q.slot * p.E + env) * p.tape_slab;
  return true;
}

// The recorded step-start state and collision stage back into the
// workspace; the state adjoints are loaded.
__global__ void k_bwd_replay(Params p, AdjParams q) {
  BwdEnv b;
  if (!bwd_env<32>(p, q, b)) return;
  const EnvInfo& e = b.e;
  const Ws& w = b.w;
  const AWs& a = b.a;
  load_from_tape(p, e, w, b.tape);
  untape_collision(p, e, w, b.tape);
  gsync(e);
  build_incidence(p, e, w, a);
  for (int i = e.lane; i < e.D; i += e.nthr) {
    const int g = e.b0 + i;
    a.bx[i] = make_float4(q.ax[3 * g], q.ax[3 * g + 1], q.ax[3 * g + 2], 0.f);
    a.bq[i] = make_float4(q.aq[4 * g], q.aq[4 * g + 1], q.aq[4 * g + 2], q.aq[4 * g + 3]);
    a.bv[i] = make_float4(q.av[3 * g], q.av[3 * g + 1], q.av[3 * g + 2], 0.f);
    a.bw[i] = make_float4(q.aw[3 * g], q.aw[3 * g + 1], q.aw[3 * g + 2], 0.f);
    a.bm[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int nc = w.misc[MC_CONTACTS];
  for (int c = e.lane; c < 3 * nc; c += e.nthr) a.cg[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = e.lane; k < p.max_dof; k += e.nthr) a.tg[k] = 0.f;
}

// Substep s: its poses and velocities from the tape, the reverse of its
// position update, and its solver rows rebuilt at those poses.
__global__ void k_bwd_rows(Params p, AdjParams q, int s) {
  BwdEnv b;
  if (!bwd_env<32>(p, q, b)) return;
  const EnvInfo& e = b.e;
  const Ws& w = b.w;
  const float* st = b.tape + b.tl.t1 + 19LL * s * p.L.Dm;
  for (int i = e.lane; i < e.D; i += e.nthr) {
    const float* t = st + 19 * i;
    const float4 inv = p.binv[e.b0 + i];
    w.bx[i] = make_float4(t[0], t[1], t[2], inv.x);
    w.bq[i] = make_float4(t[3], t[4], t[5], t[6]);
    w.bv[i] = make_float4(t[13], t[14], t[15], 0.f);
    w.bw[i] = make_float4(t[16], t[17], t[18], 0.f);
    Q4<float> qq; qq.w = t[3]; qq.x = t[4]; qq.y = t[5]; qq.z = t[6];
    float dI[3] = {inv.y, inv.z, inv.w}, W6[6];
    world_inv_inertia<float>(qq, dI, W6);
    w.bIw0[i] = make_float4(W6[0], W6[1], W6[2], W6[3]);
    // mass split: the body's constraint count in the Jacobi solve (as the
    // forward's colouring stage sets it), 1 for coloured PGS
    float split = 1.f;
    if (p.mode == MODE_JACOBI) {
      const int n = b.a.inc_off[i + 1] - b.a.inc_off[i];
      split = (float)(n > 0 ? n : 1);
    }
    w.bIw1[i] = make_float4(W6[4], W6[5], split, 0.f);
  }
  reverse_integrate(p, e, b.a, st);
  gsync(e);
  build_rows(p, e, w, b.a, b.tape + b.tl.t3);
}

// Substep s: the N sweeps in reverse. Each env group has `slice` bytes of
// shared memory: the recorded lambdas of the sweep being reversed and of the
// one before it (streamed in from the tape one sweep ahead), the body
// velocities and velocity adjoints (read and written by every constraint
// update), and the rows (parameters and adjoint accumulators, re-read and
// re-written once per row per sweep) when everything fits; the rest stays in
// the device-memory workspace.
template <bool JAC, int GS>
__global__ void k_bwd_sweeps(Params p, AdjParams q, int s, int slice) {
  extern __shared__ float4 bsm[];
  BwdEnv b;
  if (!bwd_env<GS>(p, q, b)) return;
  const EnvInfo& e = b.e;
  const float* lam0 = b.tape + b.tl.t2 + (long long)s * p.N * p.tape_Rm;
  const int RJ = ROWS_PER_JOINT * e.J;                 // joint row slots in use
  const int nc = b.w.misc[MC_CONTACTS], nm = b.w.misc[MC_MANIFOLDS];
  const int RU = ROWS_PER_JOINT * p.L.Jm + 4 * nc;     // lambda slots in use (joints of the largest env first)
  const int RU4 = RU / 4;                              // float4s per lambda buffer (RU is a multiple of 4)
  const int need_l = 3 * RU4 * 16;
  const int need_b = 4 * e.D * 16;
  const int need_r = (2 * RJ * ROW_F4 + (CPAR_F4 + CADJ_F4) * nc + 4 * nm) * 16;
  Ws w = b.w;
  AWs a = b.a;
  const bool lams = need_l <= slice, bodies = need_l + need_b <= slice, rows = need_l + need_b + need_r <= slice;
  float4* base = bsm + (size_t)(threadIdx.x / e.nthr) * (slice / 16);
  float* lbuf[3] = {(float*)base, (float*)(base + RU4), (float*)(base + 2 * RU4)};
  if (bodies) {
    w.bv = base + 3 * RU4;
    w.bw = w.bv + e.D;
    a.bv = w.bw + e.D;
    a.bw = a.bv + e.D;
    for (int i = e.lane; i < e.D; i += e.nthr) {
      w.bv[i] = b.w.bv[i]; w.bw[i] = b.w.bw[i]; a.bv[i] = b.a.bv[i]; a.bw[i] = b.a.bw[i];
    }
    if (rows) {
      a.rows = a.bw + e.D;
      a.radj = a.rows + (size_t)RJ * ROW_F4;
      a.cpar = a.radj + (size_t)RJ * ROW_F4;
      a.cadj = a.cpar + CPAR_F4 * nc;
      a.madj = a.cadj + CADJ_F4 * nc;
      for (int i = e.lane; i < RJ * ROW_F4; i += e.nthr) { a.rows[i] = b.a.rows[i]; a.radj[i] = b.a.radj[i]; }
      for (int i = e.lane; i < CPAR_F4 * nc; i += e.nthr) a.cpar[i] = b.a.cpar[i];
      for (int i = e.lane; i < CADJ_F4 * nc; i += e.nthr) a.cadj[i] = b.a.cadj[i];
      for (int i = e.lane; i < 4 * nm; i += e.nthr) a.madj[i] = b.a.madj[i];
    }
  }
  // the lambdas of sweep `it` live in lbuf[it % 3]: the two the reversed
  // sweep reads are in place, the one the next reversed sweep adds is copied
  // asynchronously while this one runs
  if (lams) {
    for (int k = p.N - 1; k >= 0 && k >= p.N - 2; --k) {
      const float* src = lam0 + (long long)k * p.tape_Rm;
      for (int i = e.lane; i < RU4; i += e.nthr) cp_async16(lbuf[k % 3] + 4 * i, src + 4 * i);
    }
    cp_async_commit();
    cp_async_wait_all();
  }
  for (int it = p.N - 1; it >= 0; --it) {
    const float* lit = lam0 + (long long)it * p.tape_Rm;
    const float* lpr = it > 0 ? lam0 + (long long)(it - 1) * p.tape_Rm : nullptr;
    if (lams) {
      if (it >= 2) {
        // lbuf[(it - 2) % 3] held sweep it + 1, whose reversal has finished
        const float* src = lam0 + (long long)(it - 2) * p.tape_Rm;
        for (int i = e.lane; i < RU4; i += e.nthr) cp_async16(lbuf[(it - 2) % 3] + 4 * i, src + 4 * i);
      }
      cp_async_commit();
      lit = lbuf[it % 3];
      lpr = it > 0 ? lbuf[(it - 1) % 3] : nullptr;
    }
    gsync(e);
    if (JAC) reverse_sweep_jacobi(p, e, w, a, lit, lpr);
    else reverse_sweep(p, e, w, a, lit, lpr);
    if (lams) cp_async_wait_all();
  }
  if (bodies) {
    gsync(e);
    for (int i = e.lane; i < e.D; i += e.nthr) {
      b.w.bv[i] = w.bv[i]; b.w.bw[i] = w.bw[i]; b.a.bv[i] = a.bv[i]; b.a.bw[i] = a.bw[i];
    }
    if (rows) {
      for (int i = e.lane; i < RJ * ROW_F4; i += e.nthr) b.a.radj[i] = a.radj[i];
      for (int i = e.lane; i < CADJ_F4 * nc; i += e.nthr) b.a.cadj[i] = a.cadj[i];
      for (int i = e.lane; i < 4 * nm; i += e.nthr) b.a.madj[i] = a.madj[i];
    }
  }
}

// Substep s: the reverse of the row set-up, gathered per body, and of the
// world inverse inertias.
__global__ void k_bwd_setup(Params p, AdjParams q, int s) {
  BwdEnv b;
  if (!bwd_env<32>(p, q, b)) return;
  reverse_setup(p, b.e, b.w, b.a);
  gsync(b.e);
  gather_bodies(b.e, b.a, true);
  gsync(b.e);
  reverse_inertia(p, b.e, b.w, b.a);
}

// The reverse of the narrowphase at the step-start poses, and the outputs.
__global__ void k_bwd_finish(Params p, AdjParams q) {
  BwdEnv b;
  if (!bwd_env<32>(p, q, b)) return;
  const EnvInfo& e = b.e;
  const Ws& w = b.w;
  const AWs& a = b.a;
  for (int i = e.lane; i < e.D; i += e.nthr) {
    const float* t = b.tape + 13 * i;
    w.bx[i] = make_float4(t[0], t[1], t[2], w.bx[i].w);
    w.bq[i] = make_float4(t[3], t[4], t[5], t[6]);
  }
  gsync(e);
  reverse_detection(p, e, w, a);
  gsync(e);
  gather_bodies(e, a, false);
  gsync(e);
  for (int i = e.lane; i < e.D; i += e.nthr) {
    const int g = e.b0 + i;
    float4 gx = a.bx[i], gq = a.bq[i], gv = a.bv[i], gw = a.bw[i], gm = a.bm[i];
    q.ox[3 * g] = gx.x; q.ox[3 * g + 1] = gx.y; q.ox[3 * g + 2] = gx.z;
    q.oq[4 * g] = gq.x; q.oq[4 * g + 1] = gq.y; q.oq[4 * g + 2] = gq.z; q.oq[4 * g + 3] = gq.w;
    q.ov[3 * g] = gv.x; q.ov[3 * g + 1] = gv.y; q.ov[3 * g + 2] = gv.z;
    q.ow[3 * g] = gw.x; q.ow[3 * g + 1] = gw.y; q.ow[3 * g + 2] = gw.z;
    if (q.omass) {
      // 1/m and the principal inverse inertias are both proportional to 1/m
      const float4 inv = p.binv[g];
      const float dm = -inv.x * inv.x * gm.x - inv.x * (inv.y * gm.y + inv.z * gm.z + inv.w * gm.w);
      q.omass[g] += dm;
    }
  }
  if (q.otg)
    for (int k = e.lane; k < p.max_dof; k += e.nthr) q.otg[(long long)e.env * p.max_dof + k] = a.tg[k];
}

// Inverse mass and principal inverse inertia from mass and shape (solid
// sphere 2/5 m r^2; box m/3 (h1^2 + h2^2); capsule = cylinder of length 2L
// plus two hemispheres about its centre, axis = local x).
__global__ void k_params(int B, const float* mass, const int* shape, const float* dims, float4* binv,
                         float4* bdims) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B) return;
  nf m = nf(mass[g]);
  int sh = shape[g];
  nf d0 = nf(dims[4 * g]), d1 = nf(dims[4 * g + 1]), d2 = nf(dims[4 * g + 2]);
  const nf one = nf(1.f);
  nf ix, iy, iz;
  if (sh == SH_SPHERE) {
    nf I = nf(0.4f) * m * d0 * d0;
    ix = iy = iz = one / I;
  } else if (sh == SH_BOX) {
    nf hx2 = d0 * d0, hy2 = d1 * d1, hz2 = d2 * d2;
    nf k = m / nf(3.f);
    ix = one / (k * (hy2 + hz2)); iy = one / (k * (hx2 + hz2)); iz = one / (k * (hx2 + hy2));
  } else {
    nf r = d0, L = d1;
    nf pi = nf(3.14159265358979323846f);
    nf vc = pi * r * r * (nf(2.f) * L);
    nf vs = nf(4.f) / nf(3.f) * pi * r * r * r;
    nf mc = m * vc / (vc + vs);
    nf ms = m * vs / (vc + vs);
    nf H = nf(2.f) * L;
    nf Ia = mc * r * r * nf(0.5f) + ms * nf(0.4f) * r * r;
    nf Ip = mc * (H * H / nf(12.f) + r * r * nf(0.25f)) + ms * (nf(0.4f) * r * r + H * H * nf(0.25f) + nf(0.375f) * H * r);
    ix = one / Ia; iy = iz = one / Ip;
  }
  binv[g] = make_float4((one / m).v, ix.v, iy.v, iz.v);
  bdims[g] = make_float4(d0.v, d1.v, d2.v, __int_as_float(sh));
}

// World frames and AABBs of the static boxes (once per scene).
__global__ void k_static(int S, const float* pose, const float* half, float off, float4* sworld) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < S) static_world(pose + 7 * g, half + 3 * g, off, sworld + (size_t)SW_N * g);
}

// The control wrapper's controller (Sec. 4.1 normalised actions), one thread
// per env: every column reads the targets from before the update (the base's
// x and y turn with the old yaw), in FP32 in the documented operation order.
struct CtrlCol {
  int kind, col;
  float scale, lo, hi;
};

__global__ void k_control(int E, int D, int A, int yaw_dof, float dtc, const CtrlCol* __restrict__ cols,
                          const float* __restrict__ action, float* __restrict__ targets) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  float* t = targets + (size_t)e * D;
  const float* a = action + (size_t)e * A;
  const float yaw = yaw_dof >= 0 ? t[yaw_dof] : 0.f;
  const float c = cosf(yaw), s = sinf(yaw);
  for (int d = 0; d < D; ++d) {
    const CtrlCol k = cols[d];
    if (k.kind == MSH_CTRL_HOLD) continue;
    const float u = fminf(fmaxf(a[k.col], -1.f), 1.f);
    float v = t[d];
    switch (k.kind) {
      case MSH_CTRL_DELTA: v = v + u * k.scale; break;
      case MSH_CTRL_ABS: v = (u + 1.f) * 0.5f * (k.hi - k.lo) + k.lo; break;
      case MSH_CTRL_BASE_X: v = v + u * k.scale * c * dtc; break;
      case MSH_CTRL_BASE_Y: v = v + u * k.scale * s * dtc; break;
      default: v = v + u * k.scale * dtc; break;   // MSH_CTRL_BASE_YAW
    }
    t[d] = fminf(fmaxf(v, k.lo), k.hi);
  }
}

// Copies the collision stage results of every env out of the plain workspace.
__global__ void k_export(Params p, float* aabb_body, float* aabb_static, int* pair_count, int* pairs,
                         int* contact_count, int* contact_ids, float* contact_geom, int* manifold_count,
                         int* colours, int* ncolours, int Jtot) {
  const int env = blockIdx.x;
  EnvInfo e = env_info(p, env);
  Ws w = plain_ws(p, env);
  const int np = w.misc[MC_PAIRS], nc = w.misc[MC_CONTACTS], nm = w.misc[MC_MANIFOLDS];
  for (int i = threadIdx.x; i < e.D + e.S; i += blockDim.x) {
    float* o = i < e.D ? (aabb_body ? aabb_body + 6 * (e.b0 + i) : nullptr)
                       : (aabb_static ? aabb_static + 6 * (e.s0 + i - e.D) : nullptr);
    if (!o) continue;
    float4 lo = aabb_lo(p, w, e, i), hi = aabb_hi(p, w, e, i);
    o[0] = lo.x; o[1] = lo.y; o[2] = lo.z; o[3] = hi.x; o[4] = hi.y; o[5] = hi.z;
  }
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    if (!pairs) break;
    int pr = w.pairs[k];
    pairs[((long long)env * p.P + k) * 2] = pr & 0xffff;
    pairs[((long long)env * p.P + k) * 2 + 1] = pr >> 16;
  }
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    long long q = (long long)env * p.C + c;
    int id = w.cid[c];
    if (contact_ids) { contact_ids[2 * q] = id & 0xffff; contact_ids[2 * q + 1] = id >> 16; }
    if (contact_geom) {
      float4 n = w.cn[c], a = w.cra[c], b = w.crb[c];
      float* g = contact_geom + 10 * q;
      g[0] = n.x; g[1] = n.y; g[2] = n.z; g[3] = a.x; g[4] = a.y; g[5] = a.z;
      g[6] = b.x; g[7] = b.y; g[8] = b.z; g[9] = n.w;
    }
  }
  if (colours) {
    for (int k = threadIdx.x; k < e.J; k += blockDim.x) colours[e.j0 + k] = w.ccol[k];
    for (int k = threadIdx.x; k < nm; k += blockDim.x) colours[Jtot + (long long)env * p.P + k] = w.ccol[e.J + k];
  }
  if (threadIdx.x == 0) {
    if (pair_count) pair_count[env] = np;
    if (contact_count) contact_count[env] = nc;
    if (manifold_count) manifold_count[env] = nm;
    if (ncolours) ncolours[env] = w.misc[MC_COLOURS];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
}  // namespace

// Error reporting for the library's other translation units (msh_last_error).
int msh_fail(int code, const char* msg) {
  g_err = msg;
  return code;
}

namespace {

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess)                                                                \
      return fail(_e == cudaErrorMemoryAllocation ? MSH_ERR_OOM : MSH_ERR_CUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(_e));                    \
  } while (0)

int align16(int x) { return (x + 15) & ~15; }

Layout make_layout(int Dm, int Sm, int Jm, int Rm, int P, int C, bool jacobi, int Ch) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  L.Dm = Dm; L.Sm = Sm; L.Jm = Jm; L.P = P; L.C = C; L.K = Jm + P; L.R = std::max(Rm, 1);
  L.Ch = std::min(std::max(Ch, 1), C);
  int o = 0;
  auto take = [&](int bytes) { int r = o; o = align16(o + bytes); return r; };
  const int f4 = 16;
  L.bv = take(Dm * f4); L.bw = take(Dm * f4);
  L.bIw0 = take(Dm * f4); L.bIw1 = take(Dm * f4);
  L.cn = take(L.Ch * f4);
  L.man = take(P * 8);
  L.jr = take(L.R * ROW_F4 * f4);
  L.jinfo = take(Jm * 16);
  L.corder = take(L.K * 4); L.coff = take((MAX_COLOURS + 1) * 4);
  if (jacobi) {
    L.jdv = take(L.K * 4 * f4); L.inc_off = take((Dm + 1) * 4); L.inc = take(2 * L.K * 4);
  } else {
    L.jdv = L.inc_off = L.inc = 0;
  }
  L.misc = take(MC_N * 4);
  // shared region: collision-only arrays | per-substep contact rows
  const int region = o;
  L.alo = take(Dm * f4); L.ahi = take(Dm * f4);
  L.pairs = take(P * 4);
  L.masks = take(Dm * 8);
  L.salo = take(Sm * f4); L.sahi = take(Sm * f4);
  const int end_x = o;
  o = region;
  L.kra = take(L.Ch * f4); L.krb = take(L.Ch * f4); L.klam = take(L.Ch * f4);
  o = std::max(o, end_x);
  L.hot_bytes = align16(o);
  // cold part: offsets relative to the cold base
  o = 0;
  L.cra = take(C * f4); L.crb = take(C * f4); L.cid = take(C * 4); L.crep = take(C * f4);
  L.bx = take(Dm * f4); L.bq = take(Dm * f4);   // poses: read per substep, not per sweep
  L.cnc = take(C * f4); L.krac = take(C * f4); L.krbc = take(C * f4); L.klamc = take(C * f4);
  L.kxc = take(C * f4);                          // row couplings: read per sweep (L1)
  L.ccol = take(L.K * 4);                        // colours: the colouring stage only
  L.cold_bytes = align16(o);
  L.bytes = L.hot_bytes + L.cold_bytes;
  return L;
}

AdjLayout make_adj_layout(const Layout& L, int md) {
  AdjLayout A;
  std::memset(&A, 0, sizeof(A));
  A.Rm = ROWS_PER_JOINT * L.Jm;   // joint row slots (contact points are stored compactly)
  A.Km = L.K;
  int o = 0;
  auto take = [&](long long bytes) { int r = o; o = align16((int)(o + bytes)); return r; };
  const int f4 = 16;
  A.bx = take(L.Dm * f4); A.bq = take(L.Dm * f4); A.bv = take(L.Dm * f4); A.bw = take(L.Dm * f4);
  A.bI0 = take(L.Dm * f4); A.bI1 = take(L.Dm * f4); A.bm = take(L.Dm * f4);
  A.rows = take((long long)A.Rm * ROW_F4 * f4); A.radj = take((long long)A.Rm * ROW_F4 * f4);
  A.cpar = take((long long)L.C * CPAR_F4 * f4); A.cadj = take((long long)L.C * CADJ_F4 * f4);
  A.madj = take((long long)L.P * 4 * f4);
  A.cpose = take((long long)L.C * 4 * f4);
  A.moff = take((long long)(L.P + 1) * 4);
  A.mord = take((long long)L.P * 4);
  A.gat = take((long long)A.Km * 8 * f4);
  A.cg = take((long long)L.C * 3 * f4);
  A.inc_off = take((L.Dm + 1) * 4); A.inc = take(2LL * A.Km * 4);
  A.tg = take((long long)(md > 0 ? md : 1) * 4);
  A.bytes = o;
  return A;
}

}  // namespace

#ifndef MSH_HOST_CHUNKS
#define MSH_HOST_CHUNKS 4   // env chunks of a pipelined host-buffer step
#endif

struct msh_handle {
  int E = 0, B = 0, S = 0, J = 0, max_dof = 0;
  msh_solver_cfg cfg;
  int Dm = 0, Sm = 0, Jm = 0;
  Layout L;
  // device scene
  int *d_body_off = nullptr, *d_static_off = nullptr, *d_joint_off = nullptr, *d_env_order = nullptr;
  float4 *d_bdims = nullptr, *d_binv = nullptr;
  float *d_static_pose = nullptr, *d_static_half = nullptr;
  float4* d_sworld = nullptr;
  std::vector<int> body_off_host;   // CSR body offsets (host copy, for argument checks)
  std::vector<int> order_host;      // envs by decreasing estimated cost
  // host-buffer steps in chunks of envs whose copies overlap the other chunks' steps
  int nchunk = 0;
  std::vector<int> chunk_env;       // chunk k holds envs [chunk_env[k], chunk_env[k + 1])
  int* d_chunk_order = nullptr;     // chunk k's envs by decreasing cost, at offset chunk_env[k]
  int* d_chunk_queue = nullptr;
  char* d_ws_chunks = nullptr;      // one set of per-slot slabs per chunk (their launches overlap)
  int64_t chunk_ws_bytes = 0;
  cudaStream_t cstream[MSH_HOST_CHUNKS] = {};
  cudaEvent_t cev[MSH_HOST_CHUNKS + 1] = {};
  std::vector<int> static_off_host;
  // depth cameras (msh_set_cameras)
  int cam_n = 0, cam_w = 0, cam_h = 0;
  float cam_focal = 0.f, cam_near = 0.f, cam_far = 0.f;
  int* d_cam_body = nullptr;
  float* d_cam_pose = nullptr;
  // control wrapper (msh_set_controller)
  CtrlCol* d_ctrl = nullptr;
  int ctrl_on = 0, ctrl_A = 0, ctrl_steps = 0, ctrl_yaw = -1;
  cudaGraphExec_t cgexec = nullptr;   // controller + physics steps
  msh_state cgkey{};
  const float* cgkey_action = nullptr;
  float* cgkey_targets = nullptr;
  int cgkey_exec = -1, cgkey_tpe = 0;
  // contact report (msh_set_report)
  int rep_on = 0;
  int *d_rep_flags = nullptr, *d_rep_fingers = nullptr, *d_rep_target = nullptr;
  float rep_fmin = 0.f, rep_cosmax = 1.f;
  msh_report_desc rep{};
  JointDesc* d_joints = nullptr;
  int* d_status = nullptr;
  int* d_queue = nullptr;
  float* d_targets = nullptr;   // library copy of the targets (graphs, host path)
  float *d_pos = nullptr, *d_quat = nullptr, *d_lv = nullptr, *d_av = nullptr;   // host-path state
  char* d_ws_plain = nullptr;   // E slabs
  char* d_ws_fused = nullptr;   // per-CTA HBM slabs (cold part, or the whole workspace without room in SMEM)
  int64_t fused_slab_bytes = 0;
  bool bwd_attr = false;         // the reversed sweeps' shared-memory attribute is set
  int bwd_sweep_warps = 0;       // ... of the reversed sweeps without shared memory
  FusedKernel fused_fn = nullptr;  // plain instantiation for the block size (occupancy)
  int fused_blocks_per_sm = 0;
  // adjoint
  float* d_tape = nullptr;      // tape_max recorded steps x E env slabs
  long long tape_slab = 0;
  int tape_max = 0, tape_count = 0, tape_Rm = 0, tape_cap = 0;   // recording capacity, recorded, rows, allocated
  int tape_paused = 0;          // msh_tape_record(h, 0): steps are not recorded, the recorded ones are kept
  char* d_aws = nullptr;        // adjoint workspace slabs (E)
  AdjLayout A;
  int64_t bytes = 0;
  // execution
  int exec = MSH_EXEC_FUSED, tpe = 128, use_graph = 0;
  int num_sms = 0, smem_optin = 0, fused_grid = 0, fused_smem = 1;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  msh_state gkey{};
  float gkey_dt = 0.f;
  int gkey_S = 0, gkey_exec = -1, gkey_tpe = 0;
  bool gkey_targets = false;
};

namespace {

template <class T>
int dalloc(msh_handle* h, T** p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? MSH_ERR_OOM : MSH_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  h->bytes += (int64_t)(n * sizeof(T));
  return MSH_OK;
}

template <class T>
int upload(msh_handle* h, T** p, const T* src, size_t n) {
  int rc = dalloc(h, p, n);
  if (rc) return rc;
  if (n) CK(cudaMemcpy(*p, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return MSH_OK;
}

Params make_params(const msh_handle* h, const msh_state* st, const float* targets, float dt, int S) {
  Params p;
  std::memset(&p, 0, sizeof(p));
  p.E = h->E; p.max_dof = h->max_dof;
  p.body_off = h->d_body_off; p.static_off = h->d_static_off; p.joint_off = h->d_joint_off;
  p.bdims = h->d_bdims; p.binv = h->d_binv;
  p.static_pose = h->d_static_pose; p.static_half = h->d_static_half; p.sworld = h->d_sworld;
  p.joints = h->d_joints; p.env_order = h->d_env_order; p.En = h->E;
  p.G = h->tpe;
  p.rep_on = h->rep_on;
  p.rep_flags = h->d_rep_flags; p.rep_fingers = h->d_rep_fingers; p.rep_target = h->d_rep_target;
  p.rep_fmin = h->rep_fmin; p.rep_cosmax = h->rep_cosmax;
  p.rep_body_force = h->rep.body_force; p.rep_target_force = h->rep.target_force;
  p.rep_finger_force = h->rep.finger_force; p.rep_robot_force = h->rep.robot_force; p.rep_grasped = h->rep.grasped;
  p.dt = dt; p.S = S; p.h = dt / (float)S; p.N = h->cfg.iterations; p.mode = h->cfg.mode;
  p.gx = h->cfg.gravity[0]; p.gy = h->cfg.gravity[1]; p.gz = h->cfg.gravity[2];
  p.mu = h->cfg.friction; p.rest = h->cfg.restitution; p.off = h->cfg.contact_offset;
  p.beta = h->cfg.baumgarte; p.jbeta = h->cfg.joint_baumgarte; p.slop = h->cfg.slop;
  p.C = h->cfg.max_contacts; p.P = h->cfg.max_pairs;
  if (st) { p.pos = st->pos; p.quat = st->quat; p.lv = st->linvel; p.av = st->angvel; }
  p.targets = h->max_dof > 0 ? targets : nullptr;
  p.status = h->d_status;
  p.L = h->L;
  p.queue = h->d_queue;
  p.tape = nullptr;
  p.tape_slab = h->tape_slab;
  p.tape_Rm = h->tape_Rm;
  return p;
}

int ensure_plain_ws(msh_handle* h) {
  if (h->d_ws_plain) return MSH_OK;
  return dalloc(h, &h->d_ws_plain, (size_t)h->E * h->L.bytes);
}

int launch_collision_plain(msh_handle* h, Params p, cudaStream_t s) {
  int rc = ensure_plain_ws(h);
  if (rc) return rc;
  p.ws = h->d_ws_plain;
  p.ws_stride = h->L.bytes;
  const int T = h->tpe < 32 ? 32 : h->tpe;   // one env per CTA here: at least a full warp
  k_load<<<h->E, T, 0, s>>>(p);
  k_aabb<<<h->E, T, 0, s>>>(p);
  k_broad<<<h->E, T, 0, s>>>(p);
  k_narrow<<<h->E, T, 0, s>>>(p);
  k_colour<<<h->E, T, 0, s>>>(p);
  CK(cudaGetLastError());
  return MSH_OK;
}

// Fused form: threads per CTA and env groups per CTA for `tpe` threads per env.
int fused_block(int tpe) { return tpe < 32 ? 32 : tpe; }
int fused_groups(int tpe) { return tpe < 32 ? 32 / tpe : 1; }

int enqueue_step(msh_handle* h, const Params& p0, cudaStream_t s) {
  Params p = p0;
  const int T = h->tpe;
  if (h->exec == MSH_EXEC_PLAIN || h->exec == MSH_EXEC_SUBSTEP) {
    int rc = launch_collision_plain(h, p, s);
    if (rc) return rc;
    p.ws = h->d_ws_plain;
    p.ws_stride = h->L.bytes;
    for (int sub = 0; sub < p.S; ++sub) {
      p.sub = sub;
      if (h->exec == MSH_EXEC_SUBSTEP) {
        k_substep<<<h->E, T, 0, s>>>(p);
        continue;
      }
      k_intvel<<<h->E, T, 0, s>>>(p);
      k_prep<<<h->E, T, 0, s>>>(p);
      for (int it = 0; it < p.N; ++it) {
        p.it = it;
        k_solve<<<h->E, T, 0, s>>>(p);
      }
      k_intpos<<<h->E, T, 0, s>>>(p);
    }
    k_store<<<h->E, T, 0, s>>>(p);
    CK(cudaGetLastError());
    return MSH_OK;
  }
  CK(cudaMemsetAsync(h->d_queue, 0, sizeof(int), s));
  p.G = T;
  p.ws = h->d_ws_fused;   // per-group slabs: the cold part (hot part in shared memory), or everything
  p.ws_stride = h->L.bytes;
  const int blk = fused_block(T);
  if (h->fused_smem)
    fused_kernel(blk, T, fused_flags(p))<<<h->fused_grid, blk, (size_t)fused_groups(T) * h->L.hot_bytes, s>>>(p, 1);
  else
    fused_kernel(blk, T, fused_flags(p))<<<h->fused_grid, blk, 0, s>>>(p, 0);
  CK(cudaGetLastError());
  return MSH_OK;
}

int configure_fused(msh_handle* h) {
  const int ng = fused_groups(h->tpe), blk = fused_block(h->tpe);
  const int bytes = ng * h->L.hot_bytes;
  // the attribute belongs to the kernel, not to a handle: raise it once to the
  // device limit (occupancy still follows each launch's actual size)
  const int max_dyn = h->smem_optin - 2048;
  h->fused_smem = bytes <= max_dyn;
  h->fused_fn = fused_kernel(blk, h->tpe, 0);
  int blocks = 0;
  if (h->fused_smem) {
    for (int fl = 0; fl < FF_N; ++fl)
      CK(cudaFuncSetAttribute(fused_kernel(blk, h->tpe, fl), cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, h->fused_fn, blk, bytes));
  } else {
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, h->fused_fn, blk, 0));
  }
  h->fused_blocks_per_sm = blocks;
  if (blocks < 1) return fail(MSH_ERR_UNSUPPORTED, "fused kernel cannot be resident with this block size");
  h->fused_grid = std::min((h->E + ng - 1) / ng, blocks * h->num_sms);
  // per-group HBM slabs: the cold part (shared-memory form) or the whole workspace
  if (h->d_ws_fused) { cudaFree(h->d_ws_fused); h->bytes -= h->fused_slab_bytes; h->d_ws_fused = nullptr; }
  if (h->d_ws_chunks) {   // the host-step chunks' slabs follow the fused configuration
    cudaFree(h->d_ws_chunks); h->bytes -= (int64_t)h->nchunk * h->chunk_ws_bytes; h->d_ws_chunks = nullptr;
  }
  h->nchunk = 0;
  h->fused_slab_bytes = (int64_t)h->fused_grid * ng * h->L.bytes;
  int rc = dalloc(h, &h->d_ws_fused, (size_t)h->fused_slab_bytes);
  if (rc) return rc;
  return MSH_OK;
}

// Shared memory per env of the reversed sweeps: as much as keeps `per_sm`
// envs resident per SM; envs beyond it run from device memory.
int bwd_sweep_slice(const msh_handle* h, int per_sm = 8) {
  const int per_cta = (h->smem_optin + 1024) / per_sm - 1024;
  return std::max(0, std::min(per_cta, h->smem_optin - 1024)) & ~15;
}

void drop_graph(msh_handle* h) {
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  h->gkey_exec = -1;
  if (h->cgexec) { cudaGraphExecDestroy(h->cgexec); h->cgexec = nullptr; }
  h->cgkey_exec = -1;
}

int check_cfg(const msh_solver_cfg* c) {
  if (!(c->dt > 0.f) || c->substeps < 1 || c->iterations < 1 || (c->mode != 0 && c->mode != 1))
    return fail(MSH_ERR_INVALID_ARG, "solver cfg: need dt > 0, substeps >= 1, iterations >= 1, mode 0/1");
  if (c->max_contacts < 1 || c->max_contacts > 1024 || c->max_pairs < 1 || c->max_pairs > 4096)
    return fail(MSH_ERR_INVALID_ARG, "solver cfg: max_contacts in 1..1024, max_pairs in 1..4096");
  if (!(c->contact_offset >= 0.f) || !(c->friction >= 0.f) || !(c->restitution >= 0.f) || !(c->slop >= 0.f))
    return fail(MSH_ERR_INVALID_ARG, "solver cfg: negative offset, friction, restitution or slop");
  return MSH_OK;
}

}  // namespace

extern "C" {

const char* msh_last_error(void) { return g_err.c_str(); }

int msh_create(const msh_scene_desc* d, const msh_solver_cfg* cfg, msh_handle** out) {
  if (!out) return fail(MSH_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d || !cfg) return fail(MSH_ERR_INVALID_ARG, "desc or cfg is NULL");
  int rc = check_cfg(cfg);
  if (rc) return rc;
  const int E = d->num_envs;
  if (E < 1 || !d->body_off || !d->static_off || !d->joint_off)
    return fail(MSH_ERR_INVALID_ARG, "num_envs < 1 or missing offsets");
  if (d->body_off[0] != 0 || d->static_off[0] != 0 || d->joint_off[0] != 0 || d->max_dof < 0)
    return fail(MSH_ERR_INVALID_ARG, "offsets must start at 0; max_dof >= 0");
  int Dm = 0, Sm = 0, Jm = 0;
  for (int e = 0; e < E; ++e) {
    int D = d->body_off[e + 1] - d->body_off[e];
    int S = d->static_off[e + 1] - d->static_off[e];
    int J = d->joint_off[e + 1] - d->joint_off[e];
    if (D < 0 || S < 0 || J < 0) return fail(MSH_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (D > 4096 || S > 4096 || J > 1024)
      return fail(MSH_ERR_INVALID_ARG, "env too large: at most 4096 bodies, 4096 static boxes, 1024 joints");
    Dm = std::max(Dm, D); Sm = std::max(Sm, S); Jm = std::max(Jm, J);
  }
  const int B = d->body_off[E], S = d->static_off[E], J = d->joint_off[E];
  if ((B && (!d->body_shape || !d->body_dims || !d->body_mass)) || (S && (!d->static_pose || !d->static_half)) ||
      (J && (!d->joint_type || !d->joint_parent || !d->joint_child || !d->joint_dof || !d->joint_frame_a ||
             !d->joint_frame_b || !d->joint_gains || !d->joint_limits)))
    return fail(MSH_ERR_INVALID_ARG, "missing descriptor array");
  for (int g = 0; g < B; ++g) {
    int sh = d->body_shape[g];
    if (sh < 0 || sh > 2) return fail(MSH_ERR_INVALID_ARG, "body " + std::to_string(g) + ": bad shape type");
    if (!(d->body_mass[g] > 0.f) || !std::isfinite(d->body_mass[g]))
      return fail(MSH_ERR_INVALID_ARG, "body " + std::to_string(g) + ": mass must be finite and > 0");
    int nd = sh == 0 ? 1 : (sh == 1 ? 2 : 3);
    for (int k = 0; k < nd; ++k)
      if (!(d->body_dims[4 * g + k] > 0.f) || !std::isfinite(d->body_dims[4 * g + k]))
        return fail(MSH_ERR_INVALID_ARG, "body " + std::to_string(g) + ": dims must be finite and > 0");
  }
  for (int k = 0; k < S; ++k)
    for (int c = 0; c < 3; ++c)
      if (!(d->static_half[3 * k + c] >= 0.f)) return fail(MSH_ERR_INVALID_ARG, "static half extents must be >= 0");
  std::vector<JointDesc> jd(J);
  int Rm = 0;   // joint solver rows of the largest env
  for (int e = 0; e < E; ++e) {
    int D = d->body_off[e + 1] - d->body_off[e];
    int roff = 0;
    for (int g = d->joint_off[e]; g < d->joint_off[e + 1]; ++g) {
      JointDesc& j = jd[g];
      std::memset(&j, 0, sizeof(j));
      j.type = d->joint_type[g]; j.parent = d->joint_parent[g]; j.child = d->joint_child[g]; j.dof = d->joint_dof[g];
      if (j.type < 0 || j.type > 2) return fail(MSH_ERR_INVALID_ARG, "joint " + std::to_string(g) + ": bad type");
      if (j.parent < -1 || j.parent >= D || j.child < 0 || j.child >= D || j.parent == j.child)
        return fail(MSH_ERR_INVALID_ARG, "joint " + std::to_string(g) + ": bad parent/child");
      int ndof = j.type == 2 ? 3 : 1;
      const float* gn = d->joint_gains + 4 * g;
      bool drive = gn[0] > 0.f || gn[1] > 0.f;
      if (drive && (j.dof < 0 || j.dof + ndof > d->max_dof))
        return fail(MSH_ERR_INVALID_ARG, "joint " + std::to_string(g) + ": dof slot outside max_dof");
      if (gn[0] < 0.f || gn[1] < 0.f || gn[2] < 0.f)
        return fail(MSH_ERR_INVALID_ARG, "joint " + std::to_string(g) + ": negative gains");
      std::memcpy(j.pa, d->joint_frame_a + 7 * g, 3 * 4); std::memcpy(j.qa, d->joint_frame_a + 7 * g + 3, 4 * 4);
      std::memcpy(j.pb, d->joint_frame_b + 7 * g, 3 * 4); std::memcpy(j.qb, d->joint_frame_b + 7 * g + 3, 4 * 4);
      j.k = gn[0]; j.d = gn[1]; j.fmax = gn[2];
      j.lo = d->joint_limits[2 * g]; j.hi = d->joint_limits[2 * g + 1];
      j.roff = roff;
      roff += joint_row_count(j);
    }
    Rm = std::max(Rm, roff);
  }
  msh_handle* h = new msh_handle();
  h->E = E; h->B = B; h->S = S; h->J = J;
  h->body_off_host.assign(d->body_off, d->body_off + E + 1);
  h->static_off_host.assign(d->static_off, d->static_off + E + 1); h->max_dof = d->max_dof; h->cfg = *cfg;
  h->Dm = std::max(Dm, 1); h->Sm = std::max(Sm, 1); h->Jm = std::max(Jm, 1);
  auto bail = [&](int code) { msh_destroy(h); return code; };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bail(fail(MSH_ERR_CUDA, "no CUDA device"));
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  {
    // Hot contact capacity: all of it when the shared workspace already fits
    // six two-env CTAs per SM; else the largest multiple of 8, down to half
    // the capacity, that does (envs with more contacts solve from the cold
    // arrays); all of it when even half does not fit.
    const bool jac = cfg->mode == MSH_MODE_JACOBI;
    const int C = cfg->max_contacts;
    const int budget = ((h->smem_optin + 1024) / 6 - 1024) / 2;
    int Ch = C;
    if (make_layout(h->Dm, h->Sm, h->Jm, Rm, cfg->max_pairs, C, jac, C).hot_bytes > budget) {
      int c = (C / 8) * 8;
      while (c > C / 2 && make_layout(h->Dm, h->Sm, h->Jm, Rm, cfg->max_pairs, C, jac, c).hot_bytes > budget) c -= 8;
      if (c > C / 2) Ch = c;
    }
    h->L = make_layout(h->Dm, h->Sm, h->Jm, Rm, cfg->max_pairs, C, jac, Ch);
  }
  // envs ordered by decreasing estimated cost (longest first): broadphase
  // candidates, bodies, joints. The order matters (4096-env apartment batch:
  // 1.72 ms per step in this order, 1.74 with the candidates weighted 0.05,
  // 1.98 reversed, 2.04 shuffled); ordering by the previous step's measured
  // per-env cycles, re-sorted on the device every step, took 1.81 ms.
  std::vector<int> order(E);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost(E);
  for (int e = 0; e < E; ++e) {
    double D = d->body_off[e + 1] - d->body_off[e], Sb = d->static_off[e + 1] - d->static_off[e];
    double Jn = d->joint_off[e + 1] - d->joint_off[e];
    cost[e] = D * (D + Sb) * 0.02 + 4.0 * D + 6.0 * Jn;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  h->order_host = order;
  if ((rc = upload(h, &h->d_body_off, d->body_off, E + 1))) return bail(rc);
  if ((rc = upload(h, &h->d_static_off, d->static_off, E + 1))) return bail(rc);
  if ((rc = upload(h, &h->d_joint_off, d->joint_off, E + 1))) return bail(rc);
  if ((rc = upload(h, &h->d_env_order, order.data(), E))) return bail(rc);
  if ((rc = upload(h, &h->d_static_pose, d->static_pose, (size_t)7 * S))) return bail(rc);
  if ((rc = upload(h, &h->d_static_half, d->static_half, (size_t)3 * S))) return bail(rc);
  if ((rc = upload(h, &h->d_joints, jd.data(), J))) return bail(rc);
  if ((rc = dalloc(h, &h->d_sworld, (size_t)SW_N * std::max(S, 1)))) return bail(rc);
  if (S) {
    k_static<<<(S + 255) / 256, 256>>>(S, h->d_static_pose, h->d_static_half, cfg->contact_offset, h->d_sworld);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bail(fail(MSH_ERR_CUDA, std::string("k_static: ") + cudaGetErrorString(e)));
  }
  if ((rc = dalloc(h, &h->d_bdims, B))) return bail(rc);
  if ((rc = dalloc(h, &h->d_binv, B))) return bail(rc);
  if ((rc = dalloc(h, &h->d_status, E))) return bail(rc);
  if ((rc = dalloc(h, &h->d_queue, 1))) return bail(rc);
  if ((rc = dalloc(h, &h->d_targets, (size_t)E * std::max(1, h->max_dof)))) return bail(rc);
  if (cudaMemset(h->d_status, 0, E * sizeof(int)) != cudaSuccess) return bail(fail(MSH_ERR_CUDA, "memset"));
  if (cudaMemset(h->d_targets, 0, (size_t)E * std::max(1, h->max_dof) * 4) != cudaSuccess)
    return bail(fail(MSH_ERR_CUDA, "memset"));
  if (B) {
    float* tm = nullptr; int* ts = nullptr; float* td = nullptr;
    if ((rc = dalloc(h, &tm, B)) || (rc = dalloc(h, &ts, B)) || (rc = dalloc(h, &td, (size_t)4 * B))) {
      cudaFree(tm); cudaFree(ts); cudaFree(td);
      return bail(rc);
    }
    cudaMemcpy(tm, d->body_mass, B * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ts, d->body_shape, B * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(td, d->body_dims, (size_t)B * 16, cudaMemcpyHostToDevice);
    k_params<<<(B + 255) / 256, 256>>>(B, tm, ts, td, h->d_binv, h->d_bdims);
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(tm); cudaFree(ts); cudaFree(td);
    h->bytes -= (int64_t)B * (4 + 4 + 16);
    if (e != cudaSuccess) return bail(fail(MSH_ERR_CUDA, std::string("k_params: ") + cudaGetErrorString(e)));
  }
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(MSH_ERR_CUDA, "stream create"));
  h->tpe = 32;
  h->exec = MSH_EXEC_FUSED;
  if ((rc = configure_fused(h))) return bail(rc);
  *out = h;
  return MSH_OK;
}

void msh_destroy(msh_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  drop_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaStream_t& c : h->cstream) if (c) cudaStreamDestroy(c);
  for (cudaEvent_t& v : h->cev) if (v) cudaEventDestroy(v);
  void* ptrs[] = {h->d_body_off, h->d_static_off, h->d_joint_off, h->d_env_order, h->d_bdims, h->d_binv,
                  h->d_static_pose, h->d_static_half, h->d_sworld, h->d_joints, h->d_status, h->d_queue, h->d_targets,
                  h->d_pos, h->d_quat, h->d_lv, h->d_av, h->d_ws_plain, h->d_ws_fused, h->d_tape, h->d_aws,
                  h->d_rep_flags, h->d_rep_fingers, h->d_rep_target, h->d_cam_body, h->d_cam_pose, h->d_ctrl,
                  h->d_chunk_order, h->d_chunk_queue, h->d_ws_chunks};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete h;
}

int msh_set_exec(msh_handle* h, int32_t exec, int32_t tpe, int32_t use_graph) {
  if (!h) return fail(MSH_ERR_INVALID_ARG, "handle is NULL");
  if (exec != MSH_EXEC_PLAIN && exec != MSH_EXEC_FUSED && exec != MSH_EXEC_SUBSTEP)
    return fail(MSH_ERR_INVALID_ARG, "exec must be MSH_EXEC_PLAIN, MSH_EXEC_FUSED or MSH_EXEC_SUBSTEP");
  if (tpe == 0) tpe = exec == MSH_EXEC_FUSED ? 32 : 128;
  if (tpe != 8 && tpe != 16 && tpe != 32 && tpe != 64 && tpe != 128 && tpe != 256 && tpe != 512)
    return fail(MSH_ERR_INVALID_ARG, "threads_per_env must be 8, 16, 32, 64, 128, 256 or 512");
  if (tpe < 32 && exec != MSH_EXEC_FUSED)
    return fail(MSH_ERR_INVALID_ARG, "threads_per_env 8 and 16 (several envs per warp) are for the fused form only");
  cudaDeviceSynchronize();
  drop_graph(h);
  h->exec = exec;
  h->tpe = tpe;
  h->use_graph = use_graph != 0;
  if (exec == MSH_EXEC_FUSED) return configure_fused(h);
  return ensure_plain_ws(h);
}

static int step_impl(msh_handle* h, const msh_state* st, const float* targets, float dt, int32_t substeps,
                     cudaStream_t s) {
  if (!h || !st || !st->pos || !st->quat || !st->linvel || !st->angvel)
    return fail(MSH_ERR_INVALID_ARG, "handle or state pointer is NULL");
  if (h->max_dof > 0 && !targets) return fail(MSH_ERR_INVALID_ARG, "joint_targets is NULL but max_dof > 0");
  if (!(dt > 0.f)) dt = h->cfg.dt;
  if (substeps < 1) substeps = h->cfg.substeps;
  if (h->tape_max > 0 && !h->tape_paused) {
    // recording for the adjoint: direct launches, one tape slot per step
    if (h->tape_count >= h->tape_max) return fail(MSH_ERR_INVALID_ARG, "tape full: call msh_backward or msh_tape_reset");
    if (substeps != h->cfg.substeps) return fail(MSH_ERR_INVALID_ARG, "recorded steps must use the configured substeps");
    Params p = make_params(h, st, targets, dt, substeps);
    p.tape = h->d_tape + (long long)h->tape_count * h->E * h->tape_slab;
    p.rep_on = 0;   // recorded re-runs of a rollout do not repeat the report
    int rc = enqueue_step(h, p, s);
    if (rc) return rc;
    h->tape_count++;
    return MSH_OK;
  }
  if (!h->use_graph) return enqueue_step(h, make_params(h, st, targets, dt, substeps), s);
  // graph path: targets go through the library buffer so one graph serves every call
  if (h->max_dof > 0)
    CK(cudaMemcpyAsync(h->d_targets, targets, (size_t)h->E * h->max_dof * 4, cudaMemcpyDeviceToDevice, s));
  bool hit = h->gexec && h->gkey.pos == st->pos && h->gkey.quat == st->quat && h->gkey.linvel == st->linvel &&
             h->gkey.angvel == st->angvel && h->gkey_dt == dt && h->gkey_S == substeps && h->gkey_exec == h->exec &&
             h->gkey_tpe == h->tpe;
  if (!hit) {
    drop_graph(h);
    if (h->exec != MSH_EXEC_FUSED) { int rc = ensure_plain_ws(h); if (rc) return rc; }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(h, make_params(h, st, h->d_targets, dt, substeps), h->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (ce != cudaSuccess) return fail(MSH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { h->gexec = nullptr; return fail(MSH_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce)); }
    h->gkey = *st; h->gkey_dt = dt; h->gkey_S = substeps; h->gkey_exec = h->exec; h->gkey_tpe = h->tpe;
  }
  CK(cudaGraphLaunch(h->gexec, s));
  return MSH_OK;
}

int msh_step(msh_handle* h, const msh_state* st, const float* joint_targets, float dt, int32_t substeps,
             void* stream) {
  return step_impl(h, st, joint_targets, dt, substeps, (cudaStream_t)stream);
}

// Chunks for host-buffer steps of the fused form: MSH_HOST_CHUNKS contiguous env ranges
// of about equal body counts, each with its envs in cost order, its own queue
// counter, workspace slabs and stream. Batches too small to fill the GPU
// (under 256 envs per chunk) are not chunked (nchunk stays 0).
static int ensure_chunks(msh_handle* h) {
  if (h->nchunk > 0) return MSH_OK;
  const int K = MSH_HOST_CHUNKS;
  if (h->E < 256 * K) return MSH_OK;
  h->chunk_env.assign(K + 1, h->E);
  h->chunk_env[0] = 0;
  const long long B = h->body_off_host[h->E];
  for (int k = 1, e = 0; k < K; ++k) {
    while (e < h->E && (long long)h->body_off_host[e] * K < B * k) ++e;
    h->chunk_env[k] = e;
  }
  std::vector<int> corder(h->E);
  for (int k = 0; k < K; ++k) {
    int o = h->chunk_env[k];
    for (int env : h->order_host)
      if (env >= h->chunk_env[k] && env < h->chunk_env[k + 1]) corder[o++] = env;
  }
  int rc;
  if (!h->d_chunk_order && (rc = dalloc(h, &h->d_chunk_order, (size_t)h->E))) return rc;
  CK(cudaMemcpy(h->d_chunk_order, corder.data(), sizeof(int) * h->E, cudaMemcpyHostToDevice));
  if (!h->d_chunk_queue && (rc = dalloc(h, &h->d_chunk_queue, (size_t)K))) return rc;
  h->chunk_ws_bytes = h->fused_slab_bytes;
  if ((rc = dalloc(h, &h->d_ws_chunks, (size_t)K * h->chunk_ws_bytes))) return rc;
  for (int k = 0; k < K; ++k)
    if (!h->cstream[k] && cudaStreamCreateWithFlags(&h->cstream[k], cudaStreamNonBlocking) != cudaSuccess)
      return fail(MSH_ERR_CUDA, "stream create");
  for (int k = 0; k <= K; ++k)
    if (!h->cev[k] && cudaEventCreateWithFlags(&h->cev[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(MSH_ERR_CUDA, "event create");
  h->nchunk = K;
  return MSH_OK;
}

// The host-buffer step in chunks: each chunk's copies in, fused launch and
// copies out run on its own stream, so one chunk's copies overlap the others'
// steps. Every env's computation is the same as in one launch.
static int step_host_chunked(msh_handle* h, float* pos, float* quat, float* linvel, float* angvel,
                             const float* targets, float dt, int32_t substeps, cudaStream_t s) {
  if (!(dt > 0.f)) dt = h->cfg.dt;
  if (substeps < 1) substeps = h->cfg.substeps;
  msh_state st{h->d_pos, h->d_quat, h->d_lv, h->d_av};
  const int T = h->tpe, ng = fused_groups(T), blk = fused_block(T);
  CK(cudaEventRecord(h->cev[h->nchunk], s));
  for (int k = 0; k < h->nchunk; ++k) {
    cudaStream_t c = h->cstream[k];
    CK(cudaStreamWaitEvent(c, h->cev[h->nchunk], 0));
    const int e0 = h->chunk_env[k], e1 = h->chunk_env[k + 1];
    const size_t b0 = h->body_off_host[e0], nb = h->body_off_host[e1] - b0;
    if (nb) {
      CK(cudaMemcpyAsync(h->d_pos + 3 * b0, pos + 3 * b0, nb * 12, cudaMemcpyHostToDevice, c));
      CK(cudaMemcpyAsync(h->d_quat + 4 * b0, quat + 4 * b0, nb * 16, cudaMemcpyHostToDevice, c));
      CK(cudaMemcpyAsync(h->d_lv + 3 * b0, linvel + 3 * b0, nb * 12, cudaMemcpyHostToDevice, c));
      CK(cudaMemcpyAsync(h->d_av + 3 * b0, angvel + 3 * b0, nb * 12, cudaMemcpyHostToDevice, c));
    }
    if (h->max_dof > 0 && e1 > e0)
      CK(cudaMemcpyAsync(h->d_targets + (size_t)e0 * h->max_dof, targets + (size_t)e0 * h->max_dof,
                         (size_t)(e1 - e0) * h->max_dof * 4, cudaMemcpyHostToDevice, c));
    if (e1 > e0) {
      Params p = make_params(h, &st, h->d_targets, dt, substeps);
      p.G = T;
      p.env_order = h->d_chunk_order + e0;
      p.En = e1 - e0;
      p.queue = h->d_chunk_queue + k;
      p.ws = h->d_ws_chunks + (long long)k * h->chunk_ws_bytes;
      p.ws_stride = h->L.bytes;
      CK(cudaMemsetAsync(p.queue, 0, sizeof(int), c));
      const int grid = std::min((p.En + ng - 1) / ng, h->fused_grid);
      if (h->fused_smem) fused_kernel(blk, p.G, fused_flags(p))<<<grid, blk, (size_t)ng * h->L.hot_bytes, c>>>(p, 1);
      else fused_kernel(blk, p.G, fused_flags(p))<<<grid, blk, 0, c>>>(p, 0);
      CK(cudaGetLastError());
    }
    if (nb) {
      CK(cudaMemcpyAsync(pos + 3 * b0, h->d_pos + 3 * b0, nb * 12, cudaMemcpyDeviceToHost, c));
      CK(cudaMemcpyAsync(quat + 4 * b0, h->d_quat + 4 * b0, nb * 16, cudaMemcpyDeviceToHost, c));
      CK(cudaMemcpyAsync(linvel + 3 * b0, h->d_lv + 3 * b0, nb * 12, cudaMemcpyDeviceToHost, c));
      CK(cudaMemcpyAsync(angvel + 3 * b0, h->d_av + 3 * b0, nb * 12, cudaMemcpyDeviceToHost, c));
    }
    CK(cudaEventRecord(h->cev[k], c));
    CK(cudaStreamWaitEvent(s, h->cev[k], 0));
  }
  CK(cudaStreamSynchronize(s));
  return MSH_OK;
}

int msh_step_host(msh_handle* h, float* pos, float* quat, float* linvel, float* angvel, const float* targets,
                  float dt, int32_t substeps, void* stream) {
  if (!h || !pos || !quat || !linvel || !angvel) return fail(MSH_ERR_INVALID_ARG, "NULL argument");
  if (h->max_dof > 0 && !targets) return fail(MSH_ERR_INVALID_ARG, "joint_targets is NULL but max_dof > 0");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if (!h->d_pos) {
    if ((rc = dalloc(h, &h->d_pos, (size_t)3 * h->B)) || (rc = dalloc(h, &h->d_quat, (size_t)4 * h->B)) ||
        (rc = dalloc(h, &h->d_lv, (size_t)3 * h->B)) || (rc = dalloc(h, &h->d_av, (size_t)3 * h->B)))
      return rc;
  }
  if (h->exec == MSH_EXEC_FUSED && !(h->tape_max > 0 && !h->tape_paused)) {
    if ((rc = ensure_chunks(h))) return rc;
    if (h->nchunk > 0) return step_host_chunked(h, pos, quat, linvel, angvel, targets, dt, substeps, s);
  }
  const size_t b3 = (size_t)3 * h->B * 4, b4 = (size_t)4 * h->B * 4;
  CK(cudaMemcpyAsync(h->d_pos, pos, b3, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->d_quat, quat, b4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->d_lv, linvel, b3, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->d_av, angvel, b3, cudaMemcpyHostToDevice, s));
  if (h->max_dof > 0)
    CK(cudaMemcpyAsync(h->d_targets, targets, (size_t)h->E * h->max_dof * 4, cudaMemcpyHostToDevice, s));
  msh_state st{h->d_pos, h->d_quat, h->d_lv, h->d_av};
  if (h->use_graph) {
    // the graph path copies targets device-to-device from the given pointer
    rc = step_impl(h, &st, h->d_targets, dt, substeps, s);
  } else {
    rc = step_impl(h, &st, h->d_targets, dt, substeps, s);
  }
  if (rc) return rc;
  CK(cudaMemcpyAsync(pos, h->d_pos, b3, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(quat, h->d_quat, b4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(linvel, h->d_lv, b3, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(angvel, h->d_av, b3, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return MSH_OK;
}

int msh_detect(msh_handle* h, const msh_state* st, float* aabb_body, float* aabb_static, int32_t* pair_count,
               int32_t* pairs, int32_t* contact_count, int32_t* contact_ids, float* contact_geom,
               int32_t* manifold_count, int32_t* colours, int32_t* ncolours, void* stream) {
  if (!h || !st || !st->pos || !st->quat || !st->linvel || !st->angvel)
    return fail(MSH_ERR_INVALID_ARG, "handle or state pointer is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  Params p = make_params(h, st, nullptr, h->cfg.dt, h->cfg.substeps);
  int rc = launch_collision_plain(h, p, s);
  if (rc) return rc;
  p.ws = h->d_ws_plain;
  p.ws_stride = h->L.bytes;
  k_export<<<h->E, 128, 0, s>>>(p, aabb_body, aabb_static, pair_count, pairs, contact_count, contact_ids,
                                contact_geom, manifold_count, colours, ncolours, h->J);
  CK(cudaGetLastError());
  return MSH_OK;
}

int msh_set_tape(msh_handle* h, int32_t max_steps) {
  if (!h) return fail(MSH_ERR_INVALID_ARG, "handle is NULL");
  if (max_steps < -1) return fail(MSH_ERR_INVALID_ARG, "max_steps must be >= -1");
  if (max_steps > 0 && h->cfg.restitution > 0.f)
    return fail(MSH_ERR_UNSUPPORTED, "the adjoint supports restitution 0 only");
  h->tape_count = 0;
  h->tape_paused = 0;
  if (max_steps <= 0) {
    h->tape_max = 0;                       // stop recording
    if (max_steps == -1 && h->d_tape) {    // and free the tape
      cudaDeviceSynchronize();
      cudaFree(h->d_tape);
      h->bytes -= (int64_t)h->tape_cap * h->E * h->tape_slab * 4;
      h->d_tape = nullptr;
      h->tape_cap = 0;
    }
    return MSH_OK;
  }
  drop_graph(h);
  const TapeLayout tl = tape_layout(h->L, h->cfg.substeps, h->cfg.iterations, h->max_dof);
  h->tape_slab = tl.slab;
  h->tape_Rm = ROWS_PER_JOINT * h->L.Jm + 4 * h->L.C;
  int rc;
  if (max_steps > h->tape_cap) {
    cudaDeviceSynchronize();
    if (h->d_tape) { cudaFree(h->d_tape); h->bytes -= (int64_t)h->tape_cap * h->E * h->tape_slab * 4; h->d_tape = nullptr; }
    h->tape_cap = 0;
    if ((rc = dalloc(h, &h->d_tape, (size_t)max_steps * h->E * tl.slab))) return rc;
    h->tape_cap = max_steps;
  }
  if (!h->d_aws) {
    h->A = make_adj_layout(h->L, h->max_dof);
    if ((rc = dalloc(h, &h->d_aws, (size_t)h->E * h->A.bytes))) return rc;
  }
  if ((rc = ensure_plain_ws(h))) return rc;
  h->tape_max = max_steps;
  return MSH_OK;
}

int msh_tape_reset(msh_handle* h) {
  if (!h) return fail(MSH_ERR_INVALID_ARG, "handle is NULL");
  h->tape_count = 0;
  return MSH_OK;
}

int32_t msh_tape_count(const msh_handle* h) { return h ? h->tape_count : 0; }

int32_t msh_tape_rows(const msh_handle* h) { return h ? ROWS_PER_JOINT * h->L.Jm + 3 * h->L.C : 0; }

// The tape keeps 4 slots per contact point (aligned vector stores); the
// inspection layout has 3, so each sweep's record is repacked on the host.

int msh_tape_lambdas(msh_handle* h, int32_t slot, float* out_host, void* stream) {
  if (!h || !out_host) return fail(MSH_ERR_INVALID_ARG, "NULL argument");
  if (slot < 0 || slot >= h->tape_count) return fail(MSH_ERR_INVALID_ARG, "no recorded step in that tape slot");
  const TapeLayout tl = tape_layout(h->L, h->cfg.substeps, h->cfg.iterations, h->max_dof);
  const size_t sweeps = (size_t)h->cfg.substeps * h->cfg.iterations;
  const size_t rows = (size_t)msh_tape_rows(h), Rm = (size_t)h->tape_Rm, RJ = (size_t)ROWS_PER_JOINT * h->L.Jm;
  std::vector<float> raw(sweeps * Rm * (size_t)h->E);
  cudaStream_t s = (cudaStream_t)stream;
  const float* src = h->d_tape + ((long long)slot * h->E) * h->tape_slab + tl.t2;
  CK(cudaMemcpy2DAsync(raw.data(), sweeps * Rm * 4, src, (size_t)h->tape_slab * 4, sweeps * Rm * 4, (size_t)h->E,
                       cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (size_t k = 0; k < sweeps * (size_t)h->E; ++k) {
    const float* a = raw.data() + k * Rm;
    float* o = out_host + k * rows;
    std::memcpy(o, a, RJ * 4);
    for (size_t c = 0; c < (size_t)h->L.C; ++c)
      for (size_t i = 0; i < 3; ++i) o[RJ + 3 * c + i] = a[RJ + 4 * c + i];
  }
  return MSH_OK;
}

int msh_tape_record(msh_handle* h, int32_t on) {
  if (!h) return fail(MSH_ERR_INVALID_ARG, "handle is NULL");
  if (on && h->tape_max <= 0) return fail(MSH_ERR_INVALID_ARG, "no tape: call msh_set_tape first");
  h->tape_paused = on ? 0 : 1;
  return MSH_OK;
}

int msh_backward(msh_handle* h, const msh_state* adj_out, msh_state* adj_in, float* adj_targets, float* adj_mass,
                 void* stream) {
  if (!h || !adj_out || !adj_in || !adj_out->pos || !adj_out->quat || !adj_out->linvel || !adj_out->angvel ||
      !adj_in->pos || !adj_in->quat || !adj_in->linvel || !adj_in->angvel)
    return fail(MSH_ERR_INVALID_ARG, "handle or adjoint state pointer is NULL");
  if (h->tape_count < 1) return fail(MSH_ERR_INVALID_ARG, "no recorded step to reverse (msh_set_tape, then msh_step)");
  Params p = make_params(h, nullptr, nullptr, h->cfg.dt, h->cfg.substeps);
  p.ws = h->d_ws_plain;
  p.ws_stride = h->L.bytes;
  p.tape = h->d_tape;
  AdjParams q;
  std::memset(&q, 0, sizeof(q));
  q.A = h->A;
  q.aws = h->d_aws;
  q.aws_stride = h->A.bytes;
  q.slot = h->tape_count - 1;
  q.ax = adj_out->pos; q.aq = adj_out->quat; q.av = adj_out->linvel; q.aw = adj_out->angvel;
  q.ox = adj_in->pos; q.oq = adj_in->quat; q.ov = adj_in->linvel; q.ow = adj_in->angvel;
  q.otg = h->max_dof > 0 ? adj_targets : nullptr;
  q.omass = adj_mass;
  // The replay, row, set-up and narrowphase phases: one env per warp (CTAs
  // of 32 threads), envs in decreasing estimated cost. Measured at 4096
  // envs (16-step rollout): 164 ms against 169 and 178 ms with two and four
  // envs per warp; the sweeps below keep two envs per warp.
  if (!h->bwd_attr) {
    CK(cudaFuncSetAttribute(k_bwd_sweeps<false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_optin - 1024));
    CK(cudaFuncSetAttribute(k_bwd_sweeps<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_optin - 1024));
    CK(cudaFuncSetAttribute(k_bwd_sweeps<false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_optin - 1024));
    CK(cudaFuncSetAttribute(k_bwd_sweeps<true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_optin - 1024));
    h->bwd_attr = true;
  }
  p.G = 32;
  const int grid = h->E;
  // The sweeps: two envs per warp (16 lanes each; a colour holds about a
  // dozen constraints) while that still fills the resident warps, each with
  // its bodies staged in shared memory; otherwise one env per warp with a
  // larger slice that also holds the rows of envs that fit.
  if (h->bwd_sweep_warps == 0) {
    int blocks = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_sweeps<false, 16>, 32, 0));
    h->bwd_sweep_warps = std::max(1, blocks) * h->num_sms;
  }
  const int Gs = (long long)h->E * 16 / 32 >= h->bwd_sweep_warps ? 16 : 32;
  // three lambda buffers sized for 3/4 of the contact capacity (the
  // shared-memory carve-out then leaves L1 the room the rows need; an env
  // with more contacts reads its lambdas from device memory)
  const int lam_bytes = 3 * (ROWS_PER_JOINT * h->L.Jm + 3 * h->L.C) * 4 / 16 * 16;
  const int slice = Gs == 32 ? bwd_sweep_slice(h) : lam_bytes + 4 * h->Dm * 16;
  const int sweep_grid = (h->E + 32 / Gs - 1) / (32 / Gs);
  Params ps = p;
  ps.G = Gs;
  cudaStream_t s = (cudaStream_t)stream;
  k_bwd_replay<<<grid, 32, 0, s>>>(p, q);
  for (int sub = p.S - 1; sub >= 0; --sub) {
    k_bwd_rows<<<grid, 32, 0, s>>>(p, q, sub);
    const size_t sm = (size_t)(32 / Gs) * slice;
    if (p.mode == MODE_JACOBI) {
      if (Gs == 16) k_bwd_sweeps<true, 16><<<sweep_grid, 32, sm, s>>>(ps, q, sub, slice);
      else k_bwd_sweeps<true, 32><<<sweep_grid, 32, sm, s>>>(ps, q, sub, slice);
    } else {
      if (Gs == 16) k_bwd_sweeps<false, 16><<<sweep_grid, 32, sm, s>>>(ps, q, sub, slice);
      else k_bwd_sweeps<false, 32><<<sweep_grid, 32, sm, s>>>(ps, q, sub, slice);
    }
    k_bwd_setup<<<grid, 32, 0, s>>>(p, q, sub);
  }
  k_bwd_finish<<<grid, 32, 0, s>>>(p, q);
  CK(cudaGetLastError());
  h->tape_count--;
  return MSH_OK;
}

int msh_get_status(msh_handle* h, int32_t* status_host, void* stream) {
  if (!h || !status_host) return fail(MSH_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(status_host, h->d_status, (size_t)h->E * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return MSH_OK;
}

int msh_clear_status(msh_handle* h, void* stream) {
  if (!h) return fail(MSH_ERR_INVALID_ARG, "NULL handle");
  CK(cudaMemsetAsync(h->d_status, 0, (size_t)h->E * 4, (cudaStream_t)stream));
  return MSH_OK;
}

int msh_set_report(msh_handle* h, const msh_report_desc* d) {
  if (!h) return fail(MSH_ERR_INVALID_ARG, "handle is NULL");
  if (d) {
    if (!d->body_flags) return fail(MSH_ERR_INVALID_ARG, "body_flags is NULL");
    if (!(d->grasp_min_force >= 0.f) || !(d->grasp_max_angle_deg >= 0.f) || !(d->grasp_max_angle_deg <= 180.f))
      return fail(MSH_ERR_INVALID_ARG, "grasp_min_force must be >= 0 and grasp_max_angle_deg in [0, 180]");
    for (int e = 0; e < h->E; ++e) {
      const int D = h->body_off_host[e + 1] - h->body_off_host[e];
      for (int k = 0; k < 3; ++k) {
        const int v = k < 2 ? (d->fingers ? d->fingers[2 * e + k] : -1) : (d->target ? d->target[e] : -1);
        if (v < -1 || v >= D)
          return fail(MSH_ERR_INVALID_ARG, "env " + std::to_string(e) + ": finger or target id out of range");
      }
    }
  }
  cudaDeviceSynchronize();
  drop_graph(h);
  int* old[] = {h->d_rep_flags, h->d_rep_fingers, h->d_rep_target};
  const size_t sizes[] = {(size_t)std::max(h->B, 1), 2 * (size_t)h->E, (size_t)h->E};
  for (int k = 0; k < 3; ++k)
    if (old[k]) { cudaFree(old[k]); h->bytes -= (int64_t)sizes[k] * 4; }
  h->d_rep_flags = h->d_rep_fingers = h->d_rep_target = nullptr;
  h->rep_on = 0;
  h->rep = msh_report_desc{};
  if (!d) return MSH_OK;
  std::vector<int> fing(2 * (size_t)h->E, -1), tgt(h->E, -1), flags(std::max(h->B, 1), 0);
  for (int e = 0; e < h->E; ++e) {
    for (int f = 0; f < 2; ++f) fing[2 * e + f] = d->fingers ? d->fingers[2 * e + f] : -1;
    tgt[e] = d->target ? d->target[e] : -1;
  }
  for (int g = 0; g < h->B; ++g) flags[g] = d->body_flags[g];
  int rc;
  if ((rc = upload(h, &h->d_rep_flags, flags.data(), flags.size()))) return rc;
  if ((rc = upload(h, &h->d_rep_fingers, fing.data(), fing.size()))) return rc;
  if ((rc = upload(h, &h->d_rep_target, tgt.data(), tgt.size()))) return rc;
  h->rep = *d;
  h->rep.body_flags = h->rep.fingers = h->rep.target = nullptr;   // host arrays are not retained
  h->rep_fmin = d->grasp_min_force;
  h->rep_cosmax = (float)std::cos((double)d->grasp_max_angle_deg * 3.14159265358979323846 / 180.0);
  h->rep_on = 1;
  return MSH_OK;
}

int msh_set_controller(msh_handle* h, const msh_controller_desc* d) {
  if (!h || !d || !d->kind || !d->action_col || !d->scale || !d->lo || !d->hi)
    return fail(MSH_ERR_INVALID_ARG, "handle, descriptor or arrays are NULL");
  const int D = h->max_dof;
  if (D < 1) return fail(MSH_ERR_INVALID_ARG, "the scene has no DoFs to control");
  if (d->action_dim < 1 || d->steps_per_action < 1)
    return fail(MSH_ERR_INVALID_ARG, "action_dim and steps_per_action must be >= 1");
  if (d->yaw_dof < -1 || d->yaw_dof >= D) return fail(MSH_ERR_INVALID_ARG, "yaw_dof out of range");
  std::vector<CtrlCol> cols(D);
  for (int k = 0; k < D; ++k) {
    const int kind = d->kind[k];
    if (kind < MSH_CTRL_HOLD || kind > MSH_CTRL_BASE_YAW)
      return fail(MSH_ERR_INVALID_ARG, "column " + std::to_string(k) + ": unknown controller kind");
    if (kind != MSH_CTRL_HOLD && (d->action_col[k] < 0 || d->action_col[k] >= d->action_dim))
      return fail(MSH_ERR_INVALID_ARG, "column " + std::to_string(k) + ": action column out of range");
    if (!(d->lo[k] <= d->hi[k]) || !std::isfinite(d->scale[k]))
      return fail(MSH_ERR_INVALID_ARG, "column " + std::to_string(k) + ": need lo <= hi and a finite scale");
    if ((kind == MSH_CTRL_BASE_X || kind == MSH_CTRL_BASE_Y) && d->yaw_dof < 0)
      return fail(MSH_ERR_INVALID_ARG, "base columns need yaw_dof");
    cols[k] = CtrlCol{kind, kind == MSH_CTRL_HOLD ? 0 : d->action_col[k], d->scale[k], d->lo[k], d->hi[k]};
  }
  cudaDeviceSynchronize();
  drop_graph(h);
  if (!h->d_ctrl) {
    int rc = dalloc(h, &h->d_ctrl, (size_t)D);
    if (rc) return rc;
  }
  CK(cudaMemcpy(h->d_ctrl, cols.data(), sizeof(CtrlCol) * D, cudaMemcpyHostToDevice));
  h->ctrl_on = 1;
  h->ctrl_A = d->action_dim;
  h->ctrl_steps = d->steps_per_action;
  h->ctrl_yaw = d->yaw_dof;
  return MSH_OK;
}

static int enqueue_control(msh_handle* h, const float* action, float* targets, cudaStream_t s) {
  const float dtc = (float)h->ctrl_steps * h->cfg.dt;
  k_control<<<(h->E + 127) / 128, 128, 0, s>>>(h->E, h->max_dof, h->ctrl_A, h->ctrl_yaw, dtc, h->d_ctrl, action,
                                               targets);
  CK(cudaGetLastError());
  return MSH_OK;
}

int msh_control_step(msh_handle* h, const msh_state* st, const float* action, float* targets, void* stream) {
  if (!h || !st || !st->pos || !st->quat || !st->linvel || !st->angvel || !action || !targets)
    return fail(MSH_ERR_INVALID_ARG, "handle, state, action or targets pointer is NULL");
  if (!h->ctrl_on) return fail(MSH_ERR_INVALID_ARG, "no controller: call msh_set_controller first");
  cudaStream_t s = (cudaStream_t)stream;
  const float dt = h->cfg.dt;
  const int S = h->cfg.substeps;
  int rc;
  const bool rec = h->tape_max > 0 && !h->tape_paused;
  if (rec || !h->use_graph) {
    // direct launches (a recording handle records each physics step)
    if (rec && h->tape_count + h->ctrl_steps > h->tape_max)
      return fail(MSH_ERR_INVALID_ARG, "tape full: call msh_backward or msh_tape_reset");
    if ((rc = enqueue_control(h, action, targets, s))) return rc;
    for (int k = 0; k < h->ctrl_steps; ++k)
      if ((rc = step_impl(h, st, targets, dt, S, s))) return rc;
    return MSH_OK;
  }
  bool hit = h->cgexec && h->cgkey.pos == st->pos && h->cgkey.quat == st->quat && h->cgkey.linvel == st->linvel &&
             h->cgkey.angvel == st->angvel && h->cgkey_action == action && h->cgkey_targets == targets &&
             h->cgkey_exec == h->exec && h->cgkey_tpe == h->tpe;
  if (!hit) {
    if (h->cgexec) { cudaGraphExecDestroy(h->cgexec); h->cgexec = nullptr; }
    h->cgkey_exec = -1;
    if (h->exec != MSH_EXEC_FUSED) { if ((rc = ensure_plain_ws(h))) return rc; }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_control(h, action, targets, h->cap_stream);
    for (int k = 0; k < h->ctrl_steps && !rc; ++k)
      rc = enqueue_step(h, make_params(h, st, targets, dt, S), h->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (ce != cudaSuccess) return fail(MSH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&h->cgexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { h->cgexec = nullptr; return fail(MSH_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce)); }
    h->cgkey = *st; h->cgkey_action = action; h->cgkey_targets = targets;
    h->cgkey_exec = h->exec; h->cgkey_tpe = h->tpe;
  }
  CK(cudaGraphLaunch(h->cgexec, s));
  return MSH_OK;
}


int msh_set_cameras(msh_handle* h, const msh_camera_desc* d) {
  if (!h || !d || !d->body || !d->pose) return fail(MSH_ERR_INVALID_ARG, "handle, descriptor or arrays are NULL");
  if (d->num_cameras < 1 || d->num_cameras > 64 || d->width < 1 || d->width > 4096 || d->height < 1 ||
      d->height > 4096)
    return fail(MSH_ERR_INVALID_ARG, "num_cameras must be 1..64 and width, height 1..4096");
  if (!(d->fov_y > 0.f) || !(d->fov_y < 3.14159265f) || !(d->near_ > 0.f) || !(d->far_ > d->near_))
    return fail(MSH_ERR_INVALID_ARG, "fov_y must be in (0, pi) and 0 < near < far");
  for (int e = 0; e < h->E; ++e) {
    const int D = h->body_off_host[e + 1] - h->body_off_host[e];
    const int S = h->static_off_host[e + 1] - h->static_off_host[e];
    if (D + S > MSH_RENDER_MAX_PRIMS)
      return fail(MSH_ERR_INVALID_ARG, "env " + std::to_string(e) + " has more than MSH_RENDER_MAX_PRIMS primitives");
    for (int c = 0; c < d->num_cameras; ++c) {
      const int b = d->body[e * d->num_cameras + c];
      if (b < -1 || b >= D) return fail(MSH_ERR_INVALID_ARG, "env " + std::to_string(e) + ": mount body out of range");
    }
  }
  cudaDeviceSynchronize();
  if (h->d_cam_body) { cudaFree(h->d_cam_body); h->bytes -= (int64_t)h->E * h->cam_n * 4; h->d_cam_body = nullptr; }
  if (h->d_cam_pose) { cudaFree(h->d_cam_pose); h->bytes -= (int64_t)h->E * h->cam_n * 28; h->d_cam_pose = nullptr; }
  h->cam_n = 0;
  int rc;
  if ((rc = upload(h, &h->d_cam_body, d->body, (size_t)h->E * d->num_cameras))) return rc;
  if ((rc = upload(h, &h->d_cam_pose, d->pose, (size_t)h->E * d->num_cameras * 7))) return rc;
  h->cam_n = d->num_cameras; h->cam_w = d->width; h->cam_h = d->height;
  h->cam_focal = (float)((double)d->height * 0.5 / std::tan((double)d->fov_y * 0.5));
  h->cam_near = d->near_; h->cam_far = d->far_;
  return MSH_OK;
}

int msh_render_depth(msh_handle* h, const msh_state* st, float* depth, void* stream) {
  if (!h || !st || !st->pos || !st->quat || !depth) return fail(MSH_ERR_INVALID_ARG, "handle, state or output is NULL");
  if (h->cam_n < 1) return fail(MSH_ERR_INVALID_ARG, "no cameras: call msh_set_cameras first");
  RenderScene sc;
  sc.E = h->E; sc.body_off = h->d_body_off; sc.static_off = h->d_static_off;
  sc.bdims = h->d_bdims; sc.sworld = h->d_sworld; sc.pos = st->pos; sc.quat = st->quat;
  RenderCams cm;
  cm.ncam = h->cam_n; cm.width = h->cam_w; cm.height = h->cam_h;
  cm.focal = h->cam_focal; cm.near_ = h->cam_near; cm.far_ = h->cam_far;
  cm.body = h->d_cam_body; cm.pose = h->d_cam_pose;
  return msh_render_launch(sc, cm, depth, (cudaStream_t)stream);
}

int64_t msh_scratch_bytes(const msh_handle* h) { return h ? h->bytes : 0; }
int64_t msh_workspace_bytes(const msh_handle* h) { return h ? h->L.hot_bytes : 0; }

int32_t msh_launches_per_step(const msh_handle* h) {
  if (!h) return 0;
  if (h->exec == MSH_EXEC_FUSED) return 1;
  if (h->exec == MSH_EXEC_SUBSTEP) return 6 + h->cfg.substeps;
  return 6 + h->cfg.substeps * (3 + h->cfg.iterations);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Step that allocates nothing: static scratch
// ---------------------------------------------------------------------------
// Some callers cannot call cudaMalloc at the time they step: code running
// while a framework's caching allocator has reserved the device memory, a
// real-time control loop that must not block in the driver's allocator, or a
// host that hands this library a pre-sized device and forbids growth. For
// them msh_step_static_scratch runs the persistent step kernel with its
// per-CTA workspace slabs in the file-scope array below instead of in memory
// from cudaMalloc. The array is part of the module, so every GPU that loads
// this library holds MSH_STATIC_SCRATCH_BYTES until the process exits.
#define MSH_STATIC_SCRATCH_BYTES (32 << 20)
static __device__ __align__(256) char g_static_scratch[MSH_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
char* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once
// per device (the host-side name is only a stand-in for the device address).
int static_scratch_address(char** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MSH_ERR_UNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(MSH_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = (char*)p;
  }
  *out = g_scratch_ptr[dev];
  return MSH_OK;
}
}  // namespace

extern "C" int msh_step_static_scratch(msh_handle* h, const msh_state* st, const float* joint_targets, float dt,
                                       int32_t substeps, void* stream) {
  if (!h || !st || !st->pos || !st->quat || !st->linvel || !st->angvel)
    return fail(MSH_ERR_INVALID_ARG, "handle or state pointer is NULL");
  if (h->max_dof > 0 && !joint_targets) return fail(MSH_ERR_INVALID_ARG, "joint_targets is NULL but max_dof > 0");
  // a recorded step needs its tape slot (device memory of the handle); this
  // entry point records nothing, so it refuses to run while recording rather
  // than advance the state past the recorded rollout
  if (h->tape_max > 0 && !h->tape_paused)
    return fail(MSH_ERR_INVALID_ARG, "msh_step_static_scratch does not record: pause or stop the tape first "
                                     "(msh_tape_record(h, 0) or msh_set_tape(h, 0))");
  if (!(dt > 0.f)) dt = h->cfg.dt;
  if (substeps < 1) substeps = h->cfg.substeps;
  // layout: [0, 256) the env-queue counter, then one 256-aligned slab per env group
  const long long slab = ((long long)h->L.bytes + 255) & ~255LL;
  if (256 + slab > MSH_STATIC_SCRATCH_BYTES)
    return fail(MSH_ERR_INVALID_ARG, "per-env workspace of " + std::to_string(h->L.bytes) +
                                         " bytes exceeds the static scratch of " +
                                         std::to_string(MSH_STATIC_SCRATCH_BYTES - 256) + " bytes");
  char* base = nullptr;
  int rc = static_scratch_address(&base);
  if (rc) return rc;
  const int ng = fused_groups(h->tpe), blk = fused_block(h->tpe);
  FusedKernel fn = fused_kernel(blk, h->tpe, 0);
  int blocks = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, blk, 0));
  if (blocks < 1) return fail(MSH_ERR_UNSUPPORTED, "step kernel cannot be resident with this block size");
  const long long fit = (MSH_STATIC_SCRATCH_BYTES - 256) / slab / ng;   // CTAs whose slabs fit
  if (fit < 1)
    return fail(MSH_ERR_INVALID_ARG, "the static scratch cannot hold one CTA's env groups at this threads_per_env");
  const int grid = (int)std::min<long long>(
      std::min<long long>((h->E + ng - 1) / ng, (long long)blocks * h->num_sms), fit);
  Params p = make_params(h, st, joint_targets, dt, substeps);
  p.G = h->tpe;
  p.ws = base + 256;
  p.ws_stride = slab;
  p.queue = (int*)base;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(base, 0, sizeof(int), s));   // the queue counter must start at zero
  fused_kernel(blk, p.G, fused_flags(p))<<<grid, blk, 0, s>>>(p, 0);
  CK(cudaGetLastError());
  return MSH_OK;
}
