// The fused step kernel: one persistent launch per step (see msh.cu), shared
// by the translation units that instantiate it.
#pragma once
#include "msh_adjoint.cuh"

using namespace msh;

// One whole step per env; persistent CTAs pull envs from an atomic queue.
// With p.G < 32 a warp holds 32 / p.G env groups, each with its own
// workspace slice, queue entries and group-local barriers. GC > 0 fixes the
// group size at compile time (it must equal p.G): the group's strides,
// masks and barrier choice are then constants.
template <int GC>
__device__ __forceinline__ void fused_body(Params& p, int smem_ws) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int scr[33];
  __shared__ int s_next;
  const int G = GC > 0 ? GC : p.G > 0 && p.G < (int)blockDim.x ? p.G : (int)blockDim.x;   // threads per env
  const int gi = threadIdx.x / G, lane = threadIdx.x % G;
  const unsigned mask = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const long long slot = (long long)blockIdx.x * (blockDim.x / G) + gi;   // workspace slot of this group
  char* slab = p.ws + slot * p.ws_stride;   // per-slot HBM slab (cold part, or all)
  char* base = smem_ws ? smem + (size_t)gi * p.L.hot_bytes : slab;
  Ws w = make_ws(base, slab + p.L.hot_bytes, p.L);
  for (;;) {
    int idx;
    if (G < 32) {
      int v = 0;
      if (lane == 0) v = atomicAdd(p.queue, 1);
      idx = __shfl_sync(mask, v, 0, G);
    } else {
      if (threadIdx.x == 0) s_next = atomicAdd(p.queue, 1);
      __syncthreads();
      idx = s_next;
    }
    if (idx >= p.En) break;
    EnvInfo e = env_info(p, p.env_order[idx], lane, G, mask);
    stage_load(p, e, w);
    gsync(e);
    stage_aabb(p, e, w);
    gsync(e);
    stage_broadphase(p, e, w, scr);
    // contacts first land in the full-capacity cold arrays; an env with at
    // most L.Ch of them moves them into the hot part and solves there, a
    // larger one solves from the cold arrays (same arithmetic, other memory)
    char* cold = slab + p.L.hot_bytes;
    w.cn = (float4*)(cold + p.L.cnc);
    stage_narrowphase(p, e, w, scr);
    {
      const int nc = w.misc[MC_CONTACTS];
      if (nc <= p.L.Ch) {
        float4* hcn = (float4*)(base + p.L.cn);
        for (int i = e.lane; i < nc; i += e.nthr) hcn[i] = w.cn[i];
        w.cn = hcn;
        w.kra = (float4*)(base + p.L.kra); w.krb = (float4*)(base + p.L.krb); w.klam = (float4*)(base + p.L.klam);
      } else {
        w.kra = (float4*)(cold + p.L.krac); w.krb = (float4*)(cold + p.L.krbc); w.klam = (float4*)(cold + p.L.klamc);
      }
      gsync(e);
    }
    stage_colour(p, e, w);
    if (p.tape) tape_collision(p, e, w);
    for (int s = 0; s < p.S; ++s) {
      stage_integrate_vel(p, e, w, s);
      gsync(e);
      stage_prep(p, e, w);
      gsync(e);
      for (int it = 0; it < p.N; ++it) stage_solve_iter(p, e, w, s, it);
      stage_accum_impulse(p, e, w, s);
      stage_integrate_pos(p, e, w, s);
      gsync(e);
    }
    stage_report(p, e, w);
    stage_store(p, e, w);
    gsync(e);
  }
}

// Up to 256 threads per CTA the compiler's own register choice is kept
// (measured on the 4096-env apartment batch: caps of 224, 200 or 168
// registers, for 9, 10 or 12 one-warp CTAs per SM, were no faster or
// slower); 512-thread CTAs need a 128-register budget.
// One instantiation per combination of the step's optional features (the
// Jacobi solver, tape recording, the contact report): the others' branches
// and code drop out of the persistent loop, so it runs fewer instructions and
// keeps a smaller instruction footprint (the 4096-env apartment batch: 1.82
// against 1.90 ms per step); the group sizes of 16 and 32 threads per env,
// the autotuner's usual choices, have their own instantiations with the size
// fixed (1.78 against 1.82 ms at 16). Results do not depend on the
// instantiation.
enum { FF_JACOBI = 1, FF_TAPE = 2, FF_REPORT = 4, FF_N = 8 };
template <int MAXT, int FL, int GC>
__global__ void __launch_bounds__(MAXT) k_fused(Params p, int smem_ws) {
  p.mode = (FL & FF_JACOBI) ? MODE_JACOBI : MODE_COLOURED;
  if (!(FL & FF_TAPE)) p.tape = nullptr;
  if (!(FL & FF_REPORT)) p.rep_on = 0;
  fused_body<GC>(p, smem_ws);
}

using FusedKernel = void (*)(Params, int);

// The instantiation for a launch's parameters.
static inline int fused_flags(const Params& p) {
  return (p.mode == MODE_JACOBI ? FF_JACOBI : 0) | (p.tape ? FF_TAPE : 0) | (p.rep_on ? FF_REPORT : 0);
}
template <int MAXT, int GC>
static FusedKernel fused_kernel_fl(int fl) {
  switch (fl) {
    case 0: return k_fused<MAXT, 0, GC>; case 1: return k_fused<MAXT, 1, GC>; case 2: return k_fused<MAXT, 2, GC>;
    case 3: return k_fused<MAXT, 3, GC>; case 4: return k_fused<MAXT, 4, GC>; case 5: return k_fused<MAXT, 5, GC>;
    case 6: return k_fused<MAXT, 6, GC>; default: return k_fused<MAXT, 7, GC>;
  }
}

// The instantiations with 16 and 32 threads per env (msh_fused16.cu,
// msh_fused32.cu: translation units of their own, so that the library's
// sources compile in parallel).
FusedKernel fused_kernel_g16(int fl);
FusedKernel fused_kernel_g32(int fl);
