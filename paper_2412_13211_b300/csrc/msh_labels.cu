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

// The chronological list of one trajectory: its length, the first three and
// the last code, the last index of every event type, and the first max_ev
// codes written out.
struct EventList {
  int n;
  int first[3];
  int lastcode;
  int last[MAX_TYPES];
  int8_t* out;
  int max_ev;
  __device__ void init(int8_t* o, int m) {
    n = 0; lastcode = -1; out = o; max_ev = m;
    for (int k = 0; k < 3; ++k) first[k] = -1;
    for (int k = 0; k < MAX_TYPES; ++k) last[k] = -1;
  }
  __device__ __forceinline__ void add(int code) {
    if (n < 3) first[n] = code;
    if (n < max_ev) out[n] = (int8_t)code;
    last[code] = n;
    lastcode = code;
    ++n;
  }
  __device__ __forceinline__ bool has(int code) const { return last[code] >= 0; }
};

// frac (qmax - qmin) + qmin, FP32 multiply then add
__device__ __forceinline__ float frac_of(float frac, float qmin, float qmax) {
  return __fadd_rn(__fmul_rn(frac, __fsub_rn(qmax, qmin)), qmin);
}

__device__ int pick_mode(const EventList& E) {
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

__device__ int place_mode(const EventList& E, bool near0) {
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

__device__ int open_mode(const EventList& E) {
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

__device__ int close_mode(const EventList& E) {
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

template <int TASK>
__global__ void k_label(msh_traj_batch b, float limit, float radius, int max_ev, int8_t* events, int32_t* num_events,
                        int32_t* label) {
  const int N = b.num_traj;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int len = b.length ? b.length[k] : b.num_steps;
  len = len < b.num_steps ? len : b.num_steps;
  EventList E;
  E.init(events + (size_t)k * max_ev, max_ev);
  for (int m = 0; m < max_ev; ++m) E.out[m] = -1;
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
  const bool with_force = TASK != MSH_TASK_PLACE;
  const bool with_dist = TASK == MSH_TASK_PLACE;
  const bool with_q = TASK == MSH_TASK_OPEN || TASK == MSH_TASK_CLOSE;
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
  for (int t = 1; t < len; ++t) {
    const size_t o = (size_t)t * N + k;
    const float c = b.cumcol[o];
    const unsigned fl = b.flags[o];
    const float f = with_force ? b.force[o] : 0.f;
    const float d = with_dist ? b.dist[o] : 0.f;
    const float q = with_q ? b.artq[o] : 0.f;
    const bool g0 = pg & 1u, g1 = fl & 1u, s0 = (pg >> 1) & 1u, s1 = (fl >> 1) & 1u;
    const bool exc = pc <= limit && c > limit;
    if (TASK == MSH_TASK_PICK) {
      if (pf == 0.f && f > 0.f) E.add(PK_CONTACT);
      if (!g0 && g1) E.add(PK_GRASPED);
      if (g0 && !g1) E.add(PK_DROPPED);
      if (!s0 && s1) E.add(PK_SUCCESS);
      if (exc) E.add(PK_EXCESSIVE);
    } else if (TASK == MSH_TASK_PLACE) {
      if (!g0 && g1) E.add(PL_GRASPED);
      if (pd > radius && d <= radius) E.add(PL_AT_GOAL);
      if (d <= radius && g0 && !g1) E.add(PL_RELEASED_AT);
      if (d > radius && g0 && !g1) E.add(PL_RELEASED_OUT);
      if (pd <= radius && d > radius) E.add(PL_LEFT_GOAL);
      if (!s0 && s1) E.add(PL_SUCCESS);
      if (exc) E.add(PL_EXCESSIVE);
    } else if (TASK == MSH_TASK_OPEN) {
      const bool o0 = pq >= thr_open, o1 = q >= thr_open;
      if (pf == 0.f && f > 0.f) E.add(OP_CONTACT);
      if (!o0 && o1) E.add(OP_OPENED);
      if (!(pq >= thr_slight) && q >= thr_slight) E.add(OP_SLIGHTLY_OPENED);
      if (o0 && !o1) E.add(OP_CLOSED);
      if (!s0 && s1) E.add(OP_SUCCESS);
      if (exc) E.add(OP_EXCESSIVE);
    } else {
      const bool c0 = pq <= thr_closed, c1 = q <= thr_closed;
      if (pf == 0.f && f > 0.f) E.add(CL_CONTACT);
      if (!c0 && c1) E.add(CL_CLOSED);
      if (!(pq < thr_slight) && q < thr_slight) E.add(CL_SLIGHTLY_CLOSED);
      if (c0 && !c1) E.add(CL_OPENED);
      if (!s0 && s1) E.add(CL_SUCCESS);
      if (exc) E.add(CL_EXCESSIVE);
    }
    pf = f; pc = c; pd = d; pq = q; pg = fl;
  }
  num_events[k] = E.n;
  int mode;
  if (TASK == MSH_TASK_PICK) mode = pick_mode(E);
  else if (TASK == MSH_TASK_PLACE) mode = place_mode(E, near0);
  else if (TASK == MSH_TASK_OPEN) mode = open_mode(E);
  else mode = close_mode(E);
  label[k] = mode;
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
  const int T = 128, G = (b->num_traj + T - 1) / T;
  cudaStream_t s = (cudaStream_t)stream;
  switch (task) {
    case MSH_TASK_PICK: k_label<MSH_TASK_PICK><<<G, T, 0, s>>>(*b, limit, radius, max_events, events, num_events, label); break;
    case MSH_TASK_PLACE: k_label<MSH_TASK_PLACE><<<G, T, 0, s>>>(*b, limit, radius, max_events, events, num_events, label); break;
    case MSH_TASK_OPEN: k_label<MSH_TASK_OPEN><<<G, T, 0, s>>>(*b, limit, radius, max_events, events, num_events, label); break;
    default: k_label<MSH_TASK_CLOSE><<<G, T, 0, s>>>(*b, limit, radius, max_events, events, num_events, label); break;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MSH_OK : msh_fail(MSH_ERR_CUDA, cudaGetErrorString(e));
}
