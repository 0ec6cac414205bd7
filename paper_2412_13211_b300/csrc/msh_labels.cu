// Event labeling and trajectory categorization (paper Sec. 3.3, Appendix A.5)
// as one batched scan over per-step records.
//
// One thread per trajectory walks t = 1..len-1, evaluates the subtask's events
// in the appendix's order from the records at t-1 and t, appends them to the
// trajectory's chronological list, and at the end reads the success or
// failure mode off the list with the appendix's formulas. Records are [T][N]
// (step-major), so a warp's loads of one step are contiguous. The scan is
// HBM-bound: 9 bytes per record for Pick/Place, 13 for Open/Close.
//
// Readings where the appendix is ambiguous (shared with the oracle):
// contact needs |F_t| > 0; an event index is its last occurrence; Pick
// winding success starts (contact, grasped) and ends with success; Open/Close
// success mode iii requires excessive collisions in E; modes are tested in
// the listed order, 0 when none holds; thresholds are FP32 multiply-then-add.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/msh.h"

int msh_fail(int code, const char* msg);   // msh.cu: sets msh_last_error

namespace {

enum { PK_CONTACT = 0, PK_GRASPED, PK_DROPPED, PK_SUCCESS, PK_EXCESSIVE };
enum { PL_GRASPED = 0, PL_AT_GOAL, PL_RELEASED_AT, PL_RELEASED_OUT, PL_LEFT_GOAL, PL_SUCCESS, PL_EXCESSIVE };
enum { OP_CONTACT = 0, OP_OPENED, OP_SLIGHTLY_OPENED, OP_CLOSED, OP_SUCCESS, OP_EXCESSIVE };
enum { CL_CONTACT = 0, CL_CLOSED, CL_SLIGHTLY_CLOSED, CL_OPENED, CL_SUCCESS, CL_EXCESSIVE };
enum { MAX_TYPES = 8 };

// Summary of a chronological event list (or of one time segment of it): its
// length, its first three and its last code, and the last index of every
// event type. Summaries of consecutive segments merge associatively, which is
// what lets several threads scan one trajectory.
struct Summary {
  int n;
  int first[3];
  int lastcode;
  int last[MAX_TYPES];
  __device__ void init() {
    n = 0; lastcode = -1;
    first[0] = first[1] = first[2] = -1;
#pragma unroll
    for (int k = 0; k < MAX_TYPES; ++k) last[k] = -1;
  }
  __device__ __forceinline__ bool has(int code) const { return last[code] >= 0; }
};

// 128 threads per block, 8 blocks per SM (64 registers), 8-step load chunks:
// measured fastest among chunks of 4/8/16, 8-16 blocks per SM and
// double-buffered chunks on 262144 x 200-step Pick and Open batches.
enum { LBL_THREADS = 128, LBL_MINB = 8, LBL_CHUNK = 8 };

// frac (qmax - qmin) + qmin, FP32 multiply then add
__device__ __forceinline__ float frac_of(float frac, float qmin, float qmax) {
  return __fadd_rn(__fmul_rn(frac, __fsub_rn(qmax, qmin)), qmin);
}

__device__ int pick_mode(const Summary& E) {
  const bool exc = E.has(PK_EXCESSIVE);
  const int ig = E.last[PK_GRASPED], id = E.last[PK_DROPPED];
  if (E.has(PK_SUCCESS)) {
    if (E.n == 3 && E.first[0] == PK_CONTACT && E.first[1] == PK_GRASPED && E.first[2] == PK_SUCCESS) return 1;
    if (E.n > 3 && E.first[0] == PK_CONTACT && E.first[1] == PK_GRASPED && E.lastcode == PK_SUCCESS && !exc) return 2;
    if (E.has(PK_DROPPED) && id > ig && !exc) return 3;
    if (exc) return 4;
    return 0;
  }
  if (exc) return 5;
  if (E.n == 0) return 6;
  if (E.n == 1 && E.first[0] == PK_CONTACT) return 7;
  if (E.has(PK_DROPPED) && id > ig) return 8;
  if (E.has(PK_GRASPED) && ig > id) return 9;
  return 0;
}

__device__ int place_mode(const Summary& E, bool near0) {
  const bool exc = E.has(PL_EXCESSIVE);
  const int ig = E.last[PL_GRASPED], iat = E.last[PL_AT_GOAL], irat = E.last[PL_RELEASED_AT];
  const int irout = E.last[PL_RELEASED_OUT], ileft = E.last[PL_LEFT_GOAL];
  if (E.has(PL_SUCCESS)) {
    if (E.n <= 4 && (E.has(PL_RELEASED_AT) || near0) && ileft <= iat && !exc) return 1;
    if (E.n <= 4 && (E.has(PL_RELEASED_OUT) || !near0) && ileft <= iat && !exc) return 2;
    if (iat < ileft && !exc) return 3;
    if (E.n > 4 && iat > ileft && !exc) return 4;
    if (exc) return 5;
    return 0;
  }
  if (exc) return 6;
  if (E.n == 0) return 7;
  if (!E.has(PL_AT_GOAL)) return 8;
  const bool placed_latest = (E.n <= 2 && near0) || (irat > irout && irat > ig);
  if (placed_latest && ileft > iat) return 9;
  const bool dropped_latest = (E.n <= 2 && !near0) || (irout > irat && irout > ig);
  if (dropped_latest && ileft > iat) return 10;
  if (ig > irat && ig > irout) return 11;
  return 12;
}

__device__ int open_mode(const Summary& E) {
  const bool exc = E.has(OP_EXCESSIVE);
  const int io = E.last[OP_OPENED], ic = E.last[OP_CLOSED], is = E.last[OP_SLIGHTLY_OPENED];
  if (E.has(OP_SUCCESS)) {
    if (!exc && io > ic) return 1;
    if (!exc && io < ic) return 2;
    if (exc) return 3;
    return 0;
  }
  if (exc) return 4;
  if (!E.has(OP_CONTACT)) return 5;
  if (E.has(OP_CLOSED) && ic > io && ic > is) return 6;
  if (is > io && is > ic) return 7;
  if (E.has(OP_OPENED)) return 8;
  return 9;
}

__device__ int close_mode(const Summary& E) {
  const bool exc = E.has(CL_EXCESSIVE);
  const int ic = E.last[CL_CLOSED], io = E.last[CL_OPENED], is = E.last[CL_SLIGHTLY_CLOSED];
  if (E.has(CL_SUCCESS)) {
    if (!exc && ic > io) return 1;
    if (!exc && ic < io) return 2;
    if (exc) return 3;
    return 0;
  }
  if (exc) return 4;
  if (!E.has(CL_CONTACT)) return 5;
  if (E.has(CL_CLOSED) && io > ic && io > is) return 6;
  if (is > ic && is > io) return 7;
  if (E.has(CL_CLOSED)) return 8;
  return 9;
}

// One thread per trajectory. Each thread loads a chunk of LBL_CHUNK steps
// (independent loads in flight) and then scans it: the step's events form a
// branch-free bit mask in the appendix's order, and the rare steps with
// events append them, lowest bit first. The first max_ev codes are staged in
// shared memory and leave as 16-byte stores.
template <int TASK>
__device__ __forceinline__ void label_one(const msh_traj_batch& b, float limit, float radius, int max_ev, int k,
                                          int8_t* mine, int32_t* num_events, int32_t* label) {
  const int N = b.num_traj;
  int len = b.length ? b.length[k] : b.num_steps;
  len = len < b.num_steps ? len : b.num_steps;
  Summary E;
  E.init();
  float qmin = 0.f, qmax = 1.f, thr_open = 0.f, thr_slight = 0.f, thr_closed = 0.f;
  if (TASK == MSH_TASK_OPEN || TASK == MSH_TASK_CLOSE) {
    qmin = b.art_range[2 * k];
    qmax = b.art_range[2 * k + 1];
    const bool fridge = b.art_fridge ? b.art_fridge[k] != 0 : false;
    thr_open = frac_of(fridge ? 0.75f : 0.9f, qmin, qmax);
    thr_closed = frac_of(0.01f, qmin, qmax);
    if (TASK == MSH_TASK_OPEN) thr_slight = frac_of(0.1f, qmin, qmax);
    else if (b.num_steps > 0) thr_slight = __fsub_rn(b.artq[k], __fmul_rn(0.05f, __fsub_rn(qmax, qmin)));
  }
  constexpr bool with_force = TASK != MSH_TASK_PLACE;
  constexpr bool with_dist = TASK == MSH_TASK_PLACE;
  constexpr bool with_q = TASK == MSH_TASK_OPEN || TASK == MSH_TASK_CLOSE;
  float pf = 0.f, pc = 0.f, pd = 0.f, pq = 0.f;
  unsigned pg = 0;
  bool near0 = false;
  if (b.num_steps > 0) {   // the records at t = 0 (the initial state)
    pc = b.cumcol[k];
    pg = b.flags[k];
    if (with_force) pf = b.force[k];
    if (with_dist) { pd = b.dist[k]; near0 = pd <= radius; }
    if (with_q) pq = b.artq[k];
  }
  for (int t0 = 1; t0 < len; t0 += LBL_CHUNK) {
    float cc[LBL_CHUNK], ff[LBL_CHUNK], dd[LBL_CHUNK], qq[LBL_CHUNK];
    unsigned gg[LBL_CHUNK];
#pragma unroll
    for (int u = 0; u < LBL_CHUNK; ++u) {
      const int t = t0 + u;
      if (t < len) {
        const size_t o = (size_t)t * N + k;
        cc[u] = b.cumcol[o];
        gg[u] = b.flags[o];
        ff[u] = with_force ? b.force[o] : 0.f;
        dd[u] = with_dist ? b.dist[o] : 0.f;
        qq[u] = with_q ? b.artq[o] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < LBL_CHUNK; ++u) {
      if (t0 + u >= len) break;
      const float c = cc[u], f = ff[u], d = dd[u], q = qq[u];
      const unsigned fl = gg[u];
      const unsigned g0 = pg & 1u, g1 = fl & 1u, s0 = (pg >> 1) & 1u, s1 = (fl >> 1) & 1u;
      const unsigned exc = (pc <= limit) & (c > limit);
      const unsigned succ = (s0 ^ 1u) & s1;
      unsigned m;
      if (TASK == MSH_TASK_PICK) {
        m = ((unsigned)(pf == 0.f) & (unsigned)(f > 0.f)) << PK_CONTACT | ((g0 ^ 1u) & g1) << PK_GRASPED |
            (g0 & (g1 ^ 1u)) << PK_DROPPED | succ << PK_SUCCESS | exc << PK_EXCESSIVE;
      } else if (TASK == MSH_TASK_PLACE) {
        // both comparisons spelled out, as in the definitions (a NaN distance is neither in nor out)
        const unsigned in0 = pd <= radius, in1 = d <= radius, out0 = pd > radius, out1 = d > radius;
        const unsigned rel = g0 & (g1 ^ 1u);
        m = ((g0 ^ 1u) & g1) << PL_GRASPED | (out0 & in1) << PL_AT_GOAL | (in1 & rel) << PL_RELEASED_AT |
            (out1 & rel) << PL_RELEASED_OUT | (in0 & out1) << PL_LEFT_GOAL | succ << PL_SUCCESS |
            exc << PL_EXCESSIVE;
      } else if (TASK == MSH_TASK_OPEN) {
        const unsigned o0 = pq >= thr_open, o1 = q >= thr_open, so0 = pq >= thr_slight, so1 = q >= thr_slight;
        m = ((unsigned)(pf == 0.f) & (unsigned)(f > 0.f)) << OP_CONTACT | ((o0 ^ 1u) & o1) << OP_OPENED |
            ((so0 ^ 1u) & so1) << OP_SLIGHTLY_OPENED | (o0 & (o1 ^ 1u)) << OP_CLOSED | succ << OP_SUCCESS |
            exc << OP_EXCESSIVE;
      } else {
        const unsigned c0 = pq <= thr_closed, c1 = q <= thr_closed, sc0 = pq < thr_slight, sc1 = q < thr_slight;
        m = ((unsigned)(pf == 0.f) & (unsigned)(f > 0.f)) << CL_CONTACT | ((c0 ^ 1u) & c1) << CL_CLOSED |
            ((sc0 ^ 1u) & sc1) << CL_SLIGHTLY_CLOSED | (c0 & (c1 ^ 1u)) << CL_OPENED | succ << CL_SUCCESS |
            exc << CL_EXCESSIVE;
      }
      while (m) {   // lowest bit first: the appendix's order within a step
        const int code = __ffs(m) - 1;
        m &= m - 1;
        if (E.n < 3) E.first[E.n] = code;
        if (E.n < max_ev) mine[E.n] = (int8_t)code;
        E.last[code] = E.n;
        E.lastcode = code;
        ++E.n;
      }
      pf = f; pc = c; pd = d; pq = q; pg = fl;
    }
  }
  num_events[k] = E.n;
  int mode;
  if (TASK == MSH_TASK_PICK) mode = pick_mode(E);
  else if (TASK == MSH_TASK_PLACE) mode = place_mode(E, near0);
  else if (TASK == MSH_TASK_OPEN) mode = open_mode(E);
  else mode = close_mode(E);
  label[k] = mode;
}

template <int TASK>
__global__ void __launch_bounds__(LBL_THREADS, LBL_MINB) k_label(msh_traj_batch b, float limit, float radius, int max_ev,
                                                          int row, int8_t* events, int32_t* num_events,
                                                          int32_t* label) {
  extern __shared__ __align__(16) int8_t s_ev[];   // LBL_THREADS rows of `row` bytes (max_ev rounded up to 16)
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  int8_t* mine = s_ev + (size_t)threadIdx.x * row;
  for (int m = 0; m < row; m += 16) *(int4*)(mine + m) = make_int4(-1, -1, -1, -1);
  if (k >= b.num_traj) return;
  label_one<TASK>(b, limit, radius, max_ev, k, mine, num_events, label);
  int8_t* dst = events + (size_t)k * max_ev;
  if ((max_ev & 15) == 0 && (((uintptr_t)events) & 15) == 0) {
    for (int m = 0; m < max_ev; m += 16) *(int4*)(dst + m) = *(const int4*)(mine + m);
  } else {
    for (int m = 0; m < max_ev; ++m) dst[m] = mine[m];
  }
}

}  // namespace

extern "C" int msh_label_events(int32_t task, const msh_traj_batch* b, int32_t max_events, int8_t* events,
                                int32_t* num_events, int32_t* label, void* stream) {
  if (!b || !events || !num_events || !label) return msh_fail(MSH_ERR_INVALID_ARG, "NULL batch or output");
  if (task < MSH_TASK_PICK || task > MSH_TASK_CLOSE) return msh_fail(MSH_ERR_INVALID_ARG, "unknown task");
  if (b->num_traj < 0 || b->num_steps < 0 || max_events < 1 || max_events > 127)
    return msh_fail(MSH_ERR_INVALID_ARG, "negative sizes or max_events outside 1..127");
  if (!b->cumcol || !b->flags) return msh_fail(MSH_ERR_INVALID_ARG, "cumcol and flags are required");
  if (task != MSH_TASK_PLACE && !b->force) return msh_fail(MSH_ERR_INVALID_ARG, "force is required for this task");
  if (task == MSH_TASK_PLACE && !b->dist) return msh_fail(MSH_ERR_INVALID_ARG, "dist is required for Place");
  if ((task == MSH_TASK_OPEN || task == MSH_TASK_CLOSE) && (!b->artq || !b->art_range))
    return msh_fail(MSH_ERR_INVALID_ARG, "artq and art_range are required for Open and Close");
  if (b->num_traj == 0) return MSH_OK;
  const float def_limit[4] = {5000.f, 7500.f, 10000.f, 10000.f};
  const float limit = b->collision_limit > 0.f ? b->collision_limit : def_limit[task];
  const float radius = b->goal_radius > 0.f ? b->goal_radius : 0.15f;
  const int T = LBL_THREADS, G = (b->num_traj + T - 1) / T;
  const int row = (max_events + 15) & ~15;
  const size_t smem = (size_t)T * row;   // <= 16 KB
  cudaStream_t s = (cudaStream_t)stream;
#define MSH_LABEL_LAUNCH(TK) k_label<TK><<<G, T, smem, s>>>( \
      *b, limit, radius, max_events, row, events, num_events, label)
  switch (task) {
    case MSH_TASK_PICK: MSH_LABEL_LAUNCH(MSH_TASK_PICK); break;
    case MSH_TASK_PLACE: MSH_LABEL_LAUNCH(MSH_TASK_PLACE); break;
    case MSH_TASK_OPEN: MSH_LABEL_LAUNCH(MSH_TASK_OPEN); break;
    default: MSH_LABEL_LAUNCH(MSH_TASK_CLOSE); break;
  }
#undef MSH_LABEL_LAUNCH
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MSH_OK : msh_fail(MSH_ERR_CUDA, cudaGetErrorString(e));
}
