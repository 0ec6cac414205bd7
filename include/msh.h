/*
 * msh.h -- C ABI of the B300-native batched rigid-body step.
 *
 * The ManiSkill-HAB paper (Sec. 4.1-4.2, "Environment Design and
 * Benchmarking") steps thousands of home-rearrangement environments in
 * parallel on one GPU: a 100 Hz physics rate under a 20 Hz control rate, PD
 * joint position targets for the arm and velocity control of the base, and a
 * robot that collides with several dynamic objects. It does not describe the
 * physics step itself. This library implements that step for a batch of
 * independent environments:
 *   a1 integrate velocities (gravity), per substep
 *   a2 world AABBs of every body and static box (inflated by the contact offset)
 *   a3 broadphase: all (i<j) pairs with overlapping AABBs, canonical order
 *   a4 narrowphase: primitive pairs to contact manifolds (<= 4 points)
 *   a5 greedy graph colouring of joints and manifolds; per substep row set-up
 *   a6 fixed-iteration coloured projected Gauss-Seidel (or mass-split Jacobi)
 *   a7 integrate positions, per substep
 * Every environment is a set of dynamic bodies (spheres, capsules, boxes), a
 * set of static boxes, the ground plane z = 0, and joints (revolute,
 * prismatic, planar) with soft PD drives, in maximal coordinates.
 *
 * Conventions: SI units, z up, quaternions (w, x, y, z). Shapes: 0 sphere
 * (dims r), 1 capsule (r, half segment length along local x), 2 box (half
 * extents). Joints: 0 revolute, 1 prismatic (axis = joint frame x), 2 planar
 * (normal = joint frame z; DoFs x, y, yaw).
 *
 * Threading: a handle may be used from one host thread at a time. Every
 * device pointer passed in must stay valid until the work queued on `stream`
 * has finished. `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).
 *
 * Errors: every function returns an int status, MSH_OK (0) or a negative
 * MSH_ERR_* code; msh_last_error() describes the last failure of the calling
 * thread. Conditions met inside the step (capacity overflow, non-finite
 * state) never trap: they set bits in a per-environment status word that
 * msh_get_status() returns.
 */
#ifndef MSH_H_
#define MSH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MSH_OK = 0,
  MSH_ERR_INVALID_ARG = -1,  /* bad pointer, size, descriptor or configuration */
  MSH_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  MSH_ERR_OOM = -3,          /* device allocation failed */
  MSH_ERR_TIMEOUT = -4,      /* a bounded device wait expired */
  MSH_ERR_UNSUPPORTED = -5   /* request outside what this build supports */
};

/* Per-environment status bits (accumulated until msh_clear_status). */
enum {
  MSH_ST_PAIR_OVERFLOW = 1,     /* more broadphase pairs than max_pairs; trailing pairs dropped */
  MSH_ST_CONTACT_OVERFLOW = 2,  /* more contact points than max_contacts; trailing points dropped */
  MSH_ST_COLOUR_OVERFLOW = 4,   /* a constraint found none of 64 colours free; it is skipped */
  MSH_ST_NONFINITE = 8          /* a body state became NaN/Inf */
};

/* Execution forms of the step (msh_set_exec). */
enum {
  MSH_EXEC_PLAIN = 0,    /* one launch per stage, workspace in HBM, S x N solver launches */
  MSH_EXEC_FUSED = 1,    /* one persistent launch per step: env work queue, workspace in shared memory */
  MSH_EXEC_SUBSTEP = 2   /* collision launches, then one launch per substep, workspace in HBM */
};

/* Solver modes. */
enum { MSH_MODE_COLOURED = 0, MSH_MODE_JACOBI = 1 };

/*
 * Scene descriptor: HOST arrays, read during msh_create and not retained.
 * CSR offsets per environment (length num_envs + 1, starting at 0) index the
 * flat body, static-box and joint arrays; body, static and joint indices
 * inside joints and contacts are env-local.
 */
typedef struct msh_scene_desc {
  int32_t num_envs;
  const int32_t* body_off;      /* [E+1] */
  const int32_t* static_off;    /* [E+1] */
  const int32_t* joint_off;     /* [E+1] */
  int32_t max_dof;              /* joint-target slots per env (>= 0) */
  const int32_t* body_shape;    /* [B]   0 sphere, 1 capsule, 2 box */
  const float* body_dims;       /* [B,4] */
  const float* body_mass;       /* [B]   > 0 */
  const float* static_pose;     /* [S,7] position, unit quaternion */
  const float* static_half;     /* [S,3] half extents */
  const int32_t* joint_type;    /* [J]   0 revolute, 1 prismatic, 2 planar */
  const int32_t* joint_parent;  /* [J]   env-local body, or -1 for the world */
  const int32_t* joint_child;   /* [J]   env-local body */
  const int32_t* joint_dof;     /* [J]   first target slot (planar uses 3) */
  const float* joint_frame_a;   /* [J,7] joint frame in the parent frame (world if parent = -1) */
  const float* joint_frame_b;   /* [J,7] joint frame in the child frame */
  const float* joint_gains;     /* [J,4] stiffness, damping, force limit, unused */
  const float* joint_limits;    /* [J,2] prismatic lower/upper (others ignore) */
} msh_scene_desc;

/* Solver parameters. */
typedef struct msh_solver_cfg {
  float dt;                /* step length [s] */
  int32_t substeps;        /* S >= 1 */
  int32_t iterations;      /* N >= 1 solver sweeps per substep */
  int32_t mode;            /* MSH_MODE_COLOURED or MSH_MODE_JACOBI */
  float gravity[3];
  float friction;          /* Coulomb coefficient, per tangent axis */
  float restitution;       /* applied to approach speeds above 1 m/s */
  float contact_offset;    /* AABB inflation and contact keep distance [m] */
  float baumgarte;         /* contact position correction factor */
  float joint_baumgarte;   /* joint position correction factor */
  float slop;              /* allowed contact penetration [m] */
  int32_t max_contacts;    /* contact points per env, 1..1024 */
  int32_t max_pairs;       /* broadphase pairs per env, 1..4096 */
} msh_solver_cfg;

/* Body state, structure of arrays over all bodies of all envs (DEVICE
 * pointers, caller-owned, float32): pos [B,3], quat [B,4], linvel [B,3],
 * angvel [B,3]. msh_step reads and overwrites them in place. */
typedef struct msh_state {
  float* pos;
  float* quat;
  float* linvel;
  float* angvel;
} msh_state;

typedef struct msh_handle msh_handle;

/*
 * Validates the descriptor, uploads the scene to library-owned device memory
 * (inverse masses and inertias are derived on the device), and sizes the
 * per-env workspace from the largest env and the configured capacities.
 * Allocates with cudaMalloc on the current device. On failure *out is NULL.
 */
int msh_create(const msh_scene_desc* desc, const msh_solver_cfg* cfg, msh_handle** out);

/* Frees everything the handle owns (synchronises its streams first). */
void msh_destroy(msh_handle* h);

/* Message of the last failed call on this host thread ("" if none). */
const char* msh_last_error(void);

/*
 * Chooses the execution form: MSH_EXEC_PLAIN, MSH_EXEC_FUSED or
 * MSH_EXEC_SUBSTEP; threads_per_env in {32, 64, 128, 256, 512}, and for the
 * fused form also 8 or 16 (4 or 2 envs share one warp, each with its own
 * workspace and group-local barriers); 0 = the form's default: 32 fused,
 * 128 otherwise. All forms give bitwise identical results;
 * use_graph != 0 captures the step's launches in a CUDA graph on first use
 * (re-captured when the state pointers, dt or substeps change).
 * Returns MSH_ERR_UNSUPPORTED if the fused form cannot hold the workspace.
 */
int msh_set_exec(msh_handle* h, int32_t exec, int32_t threads_per_env, int32_t use_graph);

/*
 * One step of every env (Sec. 4.2: 100 Hz physics, i.e. dt = 0.01 s).
 * joint_targets: DEVICE [num_envs, max_dof] absolute PD targets (rad or m),
 * may be NULL when max_dof == 0. dt > 0 and substeps >= 1 override the
 * configured values. Asynchronous on `stream`.
 */
int msh_step(msh_handle* h, const msh_state* st, const float* joint_targets, float dt,
             int32_t substeps, void* stream);

/*
 * Same step with HOST state and targets: copies pos/quat/linvel/angvel and
 * the targets into library-owned device buffers, steps, copies the state
 * back, and synchronises `stream`. Host buffers should be pinned for speed.
 */
int msh_step_host(msh_handle* h, float* pos, float* quat, float* linvel, float* angvel,
                  const float* joint_targets, float dt, int32_t substeps, void* stream);

/*
 * Collision stage only (a2-a5) at the given poses, for inspection and
 * parity tests. DEVICE outputs (any may be NULL): aabb_body [B,6],
 * aabb_static [S,6], pair_count [E], pairs [E,max_pairs,2], contact_count
 * [E], contact_ids [E,max_contacts,2] (body a, collision index b: dynamic
 * body, D + static box, or D + S for the plane), contact_geom
 * [E,max_contacts,10] (normal a->b, anchor on a in a's frame, anchor on b in
 * b's frame or world for statics, separation), manifold_count [E], colours
 * [J + E*max_pairs] (joints, then manifolds per env), ncolours [E].
 */
int msh_detect(msh_handle* h, const msh_state* st, float* aabb_body, float* aabb_static,
               int32_t* pair_count, int32_t* pairs, int32_t* contact_count,
               int32_t* contact_ids, float* contact_geom, int32_t* manifold_count,
               int32_t* colours, int32_t* ncolours, void* stream);

/*
 * The step without any device allocation. The paper has no counterpart;
 * this entry point exists for callers that cannot call cudaMalloc when they
 * step -- for example code running while a framework's caching allocator
 * holds the device memory, or a real-time loop that must not block in the
 * allocator. The handle still comes from msh_create (at start-up); this call
 * itself allocates nothing. It runs the persistent step with its per-CTA
 * workspace in a static device array of 32 MiB that every GPU loading this
 * library holds until the process exits; workspaces larger than that are
 * rejected (MSH_ERR_INVALID_ARG). The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. All calls share the
 * array: calls that overlap on the GPU (other streams, other handles) race
 * and must be serialised by the caller. Results equal msh_step's (bit for
 * bit) when no tape is recording. It records nothing: while the handle is
 * recording (msh_set_tape with n > 0, not paused by msh_tape_record) it
 * returns MSH_ERR_INVALID_ARG and leaves the state untouched.
 */
int msh_step_static_scratch(msh_handle* h, const msh_state* st, const float* joint_targets, float dt,
                            int32_t substeps, void* stream);

/*
 * Contact report, written by every msh_step (and msh_step_static_scratch)
 * while enabled; recorded steps (msh_set_tape) do not write it. It carries
 * what the paper's subtask success conditions and event labels consume
 * (Sec. 3.3, Appendix A.4-A.5): pairwise contact forces F_{a,b,t} in N, the
 * robot's cumulative collision force, and whether the target is grasped.
 *   - The force of a contact on its second body is its impulse
 *     (l_n n + l_t1 t1 + l_t2 t2) summed over the step's substeps and divided
 *     by dt; the first body receives the opposite force.
 *   - body_force [num_bodies][3]: the net contact force on each body.
 *   - target_force [num_envs][3]: the force on the target from the
 *     end-effector links.
 *   - finger_force [num_envs][2][3]: the force on each finger from the target.
 *   - robot_force [num_envs]: each step ADDS the sum over robot links of the
 *     norm of the link's net force from contacts with static boxes and with
 *     bodies that are neither robot links nor the target (the caller zeroes it
 *     at episode start).
 *   - grasped [num_envs]: 1 when both fingers feel at least grasp_min_force
 *     from the target, each within grasp_max_angle_deg of the finger's opening
 *     direction (from the other finger towards it).
 * body_flags, fingers and target are HOST arrays read during the call (not
 * retained); fingers and target hold env-local body ids (-1: none; NULL: all
 * -1). The outputs are caller-owned DEVICE pointers kept by the handle; any
 * may be NULL (not written). msh_set_report(h, NULL) turns the report off.
 * Returns MSH_ERR_INVALID_ARG on a NULL body_flags or out-of-range ids.
 */
typedef struct msh_report_desc {
  const int32_t* body_flags;   /* [num_bodies]: bit 0 robot link, bit 1 end-effector link */
  const int32_t* fingers;      /* [num_envs][2] */
  const int32_t* target;       /* [num_envs] */
  float grasp_min_force;       /* N (>= 0) */
  float grasp_max_angle_deg;   /* [0, 180] */
  float* body_force;
  float* target_force;
  float* finger_force;
  float* robot_force;
  int32_t* grasped;
} msh_report_desc;

int msh_set_report(msh_handle* h, const msh_report_desc* desc);

/*
 * Control wrapper (Sec. 4.1: PD joint delta-position control of the arm,
 * linear and angular velocity of the base, actions normalised to [-1, 1];
 * Sec. 4.2: 100 Hz physics under 20 Hz control). One control step applies
 * the controller to every env's joint targets, then runs steps_per_action
 * physics steps (the configured dt and substeps) with the new targets. Each
 * DoF column d (shared by every env) has a kind:
 *   MSH_CTRL_HOLD      the target is kept (passive joints);
 *   MSH_CTRL_DELTA     t += a * scale, a = action[e][action_col[d]];
 *   MSH_CTRL_ABS       t = ((a + 1) * 0.5) * (hi - lo) + lo;
 *   MSH_CTRL_BASE_X    t += ((a * scale) * cos(yaw)) * dt_c;
 *   MSH_CTRL_BASE_Y    t += ((a * scale) * sin(yaw)) * dt_c;
 *   MSH_CTRL_BASE_YAW  t += (a * scale) * dt_c;
 * where a is the action component clipped to [-1, 1] (fmaxf then fminf, so
 * NaN counts as -1), yaw is column yaw_dof's target before this update,
 * dt_c = steps_per_action * dt in FP32, and every written target is then
 * clipped to [lo[d], hi[d]]. All in FP32 in the order shown, without FMA
 * contraction. kind, action_col, scale, lo and hi are HOST arrays of
 * max_dof entries read during msh_set_controller (not retained).
 * Returns MSH_ERR_INVALID_ARG for a bad kind, an action column outside
 * [0, action_dim), lo > hi, a base column without yaw_dof, or a handle with
 * no DoFs.
 */
enum { MSH_CTRL_HOLD = 0, MSH_CTRL_DELTA = 1, MSH_CTRL_ABS = 2, MSH_CTRL_BASE_X = 3, MSH_CTRL_BASE_Y = 4,
       MSH_CTRL_BASE_YAW = 5 };

typedef struct msh_controller_desc {
  int32_t action_dim;        /* action components per env, >= 1 */
  int32_t steps_per_action;  /* physics steps per control step, >= 1 (5: 100 Hz under 20 Hz) */
  int32_t yaw_dof;           /* the base's yaw column, -1 when no column is MSH_CTRL_BASE_X/Y */
  const int32_t* kind;       /* [max_dof] MSH_CTRL_* */
  const int32_t* action_col; /* [max_dof] action column; ignored for MSH_CTRL_HOLD */
  const float* scale;        /* [max_dof] rad or m per unit action (DELTA), m/s or rad/s (BASE_*) */
  const float* lo;           /* [max_dof] target range */
  const float* hi;
} msh_controller_desc;

int msh_set_controller(msh_handle* h, const msh_controller_desc* desc);

/*
 * One control step of every env: the controller reads action, DEVICE
 * [num_envs][action_dim], and updates targets, DEVICE [num_envs][max_dof]
 * (the caller-owned PD targets, read and written in place), then
 * steps_per_action physics steps run with them (recorded one by one while a
 * tape is set, writing the contact report while one is set). With use_graph
 * (msh_set_exec) the controller and the physics steps are one CUDA graph,
 * captured on first use and re-captured when the state, action or targets
 * pointers change. Asynchronous on `stream`. Returns MSH_ERR_INVALID_ARG
 * without a controller or with NULL pointers.
 */
int msh_control_step(msh_handle* h, const msh_state* st, const float* action, float* targets, void* stream);

/*
 * Depth cameras (the paper's per-env RGB-D cameras, Sec. 4.2; the depth
 * channel, ray-cast against the env's primitives instead of rasterised).
 * Pinhole camera looking along its frame's +x (image right = -y, image down
 * = -z), pixel (row, col) centred at (col + 1/2, row + 1/2), focal length
 * f = (height/2) / tan(fov_y/2) pixels. A camera is mounted on a body
 * (env-local id; its pose is composed with the body's) or on the world (-1).
 * The depth of a pixel is the z-depth (distance along the optical axis) of
 * the nearest hit in [near, far] among spheres, capsules, boxes, static boxes
 * and the ground plane, or 0 when nothing is hit. body and pose are HOST
 * arrays read during msh_set_cameras (not retained). Envs may hold at most
 * MSH_RENDER_MAX_PRIMS bodies plus static boxes. Returns MSH_ERR_INVALID_ARG
 * on bad sizes, angles, clip distances or ids.
 */
enum { MSH_RENDER_MAX_PRIMS = 256 };

typedef struct msh_camera_desc {
  int32_t num_cameras;   /* per env, >= 1 */
  int32_t width, height; /* pixels, 1..4096 */
  float fov_y;           /* vertical field of view, radians, in (0, pi) */
  float near_, far_;     /* clip distances along the optical axis, 0 < near < far */
  const int32_t* body;   /* [num_envs][num_cameras] env-local mount body, -1 = world */
  const float* pose;     /* [num_envs][num_cameras][7] mount-local position and quaternion (w,x,y,z) */
} msh_camera_desc;

int msh_set_cameras(msh_handle* h, const msh_camera_desc* desc);

/* Renders every camera of every env at the state st (DEVICE) into depth,
 * DEVICE float [num_envs][num_cameras][height][width]; asynchronous. */
int msh_render_depth(msh_handle* h, const msh_state* st, float* depth, void* stream);

/*
 * Differentiation (reverse mode). msh_set_tape(h, n), n > 0, makes room for
 * n recorded steps (reusing a large enough tape) and starts recording
 * (either solver mode; zero restitution only); n = 0 stops recording and
 * keeps the memory, n = -1 stops and frees it. Setting the tape drops any
 * recorded steps. While recording, every msh_step records the step (start state, per-substep poses and
 * velocities, the lambdas after every sweep, the targets) into the next slot;
 * graphs are not used for recorded steps. msh_backward reverses the most
 * recently recorded step and pops it: given adj_out, the adjoint of the state
 * after that step (DEVICE, same layout as msh_state), it writes adj_in, the
 * adjoint of the state before it (may alias adj_out), the adjoint of that
 * step's joint targets into adj_targets [num_envs, max_dof] (may be NULL), and
 * ADDS the adjoint of the body masses into adj_mass [B] (may be NULL). The
 * step is differentiated with its discrete decisions frozen: contact set and
 * features, colouring, and the clamp states of every row update.
 * msh_tape_reset drops every recorded step; msh_tape_count returns how many
 * are recorded.
 */
int msh_set_tape(msh_handle* h, int32_t max_steps);
int msh_tape_reset(msh_handle* h);
int32_t msh_tape_count(const msh_handle* h);
/* Pauses (on = 0) or resumes (on != 0) recording without dropping the
 * recorded steps: while paused, steps run as without a tape and msh_backward
 * still reverses the recorded ones. Resuming needs a tape (msh_set_tape);
 * msh_set_tape resumes as well. */
int msh_tape_record(msh_handle* h, int32_t on);
int msh_backward(msh_handle* h, const msh_state* adj_out, msh_state* adj_in, float* adj_targets,
                 float* adj_mass, void* stream);

/*
 * Inspection of a recorded step (for tests and debugging; the paper has no
 * counterpart). msh_tape_lambdas copies the impulses that tape slot `slot`
 * (0 = the oldest recorded step still on the tape) holds after every sweep
 * into out_host, a HOST buffer of num_envs * substeps * iterations *
 * msh_tape_rows(h) floats, laid out [env][substep][sweep][row]. Rows of an
 * env: joint k's row r at k * 8 + r (8 slots per joint of the largest env),
 * then contact point c's normal, first and second friction row at
 * 8 * Jmax + 3 c + {0, 1, 2}; slots the step does not use are unspecified.
 * (The tape itself keeps 4 slots per contact point so that the step writes
 * aligned vectors; this copy is repacked to the 3-slot layout on the host.)
 * Synchronises `stream`. Returns MSH_ERR_INVALID_ARG for an empty slot.
 */
int32_t msh_tape_rows(const msh_handle* h);
int msh_tape_lambdas(msh_handle* h, int32_t slot, float* out_host, void* stream);

/* Copies the per-env status words to host memory [num_envs] (synchronises
 * `stream`). */
int msh_get_status(msh_handle* h, int32_t* status_host, void* stream);

/* Zeroes the per-env status words. */
int msh_clear_status(msh_handle* h, void* stream);

/* Bytes of device memory owned by the handle. */
int64_t msh_scratch_bytes(const msh_handle* h);

/* Per-env shared-memory workspace bytes of the fused form (the hot part: body
   state, contact normals, solver rows, colouring). Contact anchors and ids
   (read once per substep) live in device memory beside it. */
int64_t msh_workspace_bytes(const msh_handle* h);

/* Number of kernel launches one msh_step issues in the current form. */
int32_t msh_launches_per_step(const msh_handle* h);

/*
 * Event labeling and trajectory categorization (Sec. 3.3, Appendix A.5): a
 * batched scan over per-step records of N trajectories of one subtask. For
 * t = 1..length-1 the subtask's events are evaluated in the appendix's order
 * from the records at t-1 and t and appended to the trajectory's
 * chronological list; the list then decides the success or failure mode.
 *   Pick:  contact, grasped, dropped, success, excessive_collisions
 *   Place: grasped, obj_at_goal, released_at_goal, released_outside_goal,
 *          obj_left_goal, success, excessive_collisions
 *   Open:  contact, opened, slightly_opened, closed, success, excessive_collisions
 *   Close: contact, closed, slightly_closed, opened, success, excessive_collisions
 * (event codes are the 0-based positions in these lists). Modes are the
 * appendix's roman numerals (Pick 1-9, Place 1-12, Open and Close 1-9), tested
 * in order; 0 when none holds. Readings: contact needs a nonzero force; an
 * event's index is its last occurrence; Open/Close success mode iii requires
 * excessive collisions in the list; thresholds are formed and compared in FP32.
 * All arrays are DEVICE pointers; records are step-major [num_steps][num_traj].
 */
enum { MSH_TASK_PICK = 0, MSH_TASK_PLACE = 1, MSH_TASK_OPEN = 2, MSH_TASK_CLOSE = 3 };

typedef struct msh_traj_batch {
  int32_t num_traj, num_steps;
  const float* force;        /* [T][N] |F_{ee,target}| in N (Pick, Open, Close) */
  const float* cumcol;       /* [T][N] cumulative robot collision force in N */
  const float* dist;         /* [T][N] target-to-goal distance in m (Place) */
  const float* artq;         /* [T][N] articulation joint position (Open, Close) */
  const uint8_t* flags;      /* [T][N] bit 0 grasped(target), bit 1 success */
  const int32_t* length;     /* [N] valid records per trajectory (clipped to T); NULL: T */
  const float* art_range;    /* [N][2] qmin, qmax (Open, Close) */
  const uint8_t* art_fridge; /* [N] 1: fridge (opens at 0.75 of the range), 0: drawer (0.9); NULL: drawers */
  float collision_limit;     /* N; <= 0: 5000 Pick, 7500 Place, 10000 Open/Close */
  float goal_radius;         /* m; <= 0: 0.15 */
} msh_traj_batch;

/*
 * Writes num_events [N] (the list's length), the first max_events (1..127)
 * codes of each list into events [N][max_events] (int8, -1 padded) and the
 * mode into label [N]; all DEVICE, asynchronous on `stream`. Returns
 * MSH_ERR_INVALID_ARG for a bad task, NULL arrays the task needs or bad sizes.
 */
int msh_label_events(int32_t task, const msh_traj_batch* batch, int32_t max_events, int8_t* events,
                     int32_t* num_events, int32_t* label, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MSH_H_ */
