/*
 * orchard.h — C ABI of the batched compliant-tree step (liborchard.so, sm_103a).
 *
 * The library steps many independent worlds, each a kinematic tree of branch-segment bodies
 * on compliant bending joints carrying apples on stem tethers (arxiv 2607.06337, Sec. IV):
 *   - joint rest transform T = (0,0,l_parent) * q_rel, stress-free at rest (Sec. IV, Eq. 3);
 *   - each compliant joint has up to two bending DOFs (Cardan x then y' of a twist-locked D6)
 *     with torsional spring-damper tau = -k theta - kd omega, k = E I / l (Sec. IV-A, Eq. 4);
 *   - rupture when k |theta| > sigma_r pi r^3 / 4 for N_b consecutive steps, after which the
 *     joint is a free hinge (its gain rows zeroed in place, Sec. IV-B, Eq. 5) whose torn-fibre
 *     friction ramps up over about 1.5 s (read as an implicit viscous damper), and the apples
 *     of the snapped sub-tree no longer load it (applied forces disabled, App. B);
 *   - apples as 3-DOF free bodies on tethers f = -k_s (x - x_hang) - c_s v whose elastic part
 *     minus the static weight reacts on the spur, clamped (Sec. IV-C, Eqs. 6-7); they detach
 *     on a sustained pull above f_detach or a longer tension above gamma f_detach (Sec. IV-C).
 * One step: forward kinematics, RNE bias forces, CRBA mass matrix, H = M + dt D' (+ dt^2 K'),
 * tree-sparse LDL^T factor and solve, semi-implicit update, apple update, break and detach
 * tests. Worlds may differ in topology, size and every parameter (Sec. IV-D generalised).
 *
 * Conventions
 *   - Every call is asynchronous on the given CUDA stream (passed as void*, a cudaStream_t;
 *     NULL is the legacy default stream), except ot_tree_model_upload's host validation and
 *     the *_bytes size queries, which are host-only.
 *   - The library never allocates device memory: every device buffer is allocated by the
 *     caller (for example as a torch tensor) and passed as a pointer with its byte size.
 *     Handles (ot_model, ot_state) are small host structs freed by *_release.
 *   - Errors are negative ot_status codes; a call that fails leaves its outputs unchanged
 *     unless stated. Per-world runtime faults (a non-finite state) do not fail a call: they
 *     set bits in the per-world status word and freeze that world.
 *   - Floating point on the device is FP32 (FMA contraction allowed). Descriptors are FP64
 *     on the host and converted at upload.
 *
 * Layout of a descriptor (packed CSR over worlds; indices inside a world are world-local):
 *   bodies of world w are [body_off[w], body_off[w+1]); they must be in breadth-first order:
 *   parent[0] = -1 for the root, 0 <= parent[i] < i and parent non-decreasing for i >= 1
 *   (so each level and each body's children are contiguous). Apples of world w are
 *   [apple_off[w], apple_off[w+1]) sorted by apple_body (non-decreasing). Tips likewise.
 *   The DOFs of a world are numbered body by body, each body's ndof DOFs consecutively.
 */
#ifndef ORCHARD_H
#define ORCHARD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ot_status;
#define OT_OK 0
#define OT_EINVAL (-1)      /* null pointer, size mismatch, buffer too small, bad flag value */
#define OT_ETOPO (-2)       /* not breadth-first, parent out of range, ndof not in {0,1,2} */
#define OT_ENONFINITE (-3)  /* a descriptor value is NaN or infinite, or a mass is not > 0 */
#define OT_ECAPACITY (-4)   /* a world exceeds a hard limit (32767 DOFs, 255 children/apples per body) */
#define OT_ECUDA (-5)       /* a CUDA call failed; ot_last_cuda_error() gives its code */
#define OT_ESTATE (-6)      /* call out of order (e.g. backward without a recorded forward) */

/* per-world status bits (ot_world_status) */
#define OT_WORLD_NONFINITE 1u   /* the state became non-finite; the world is frozen */

typedef struct ot_model ot_model; /* opaque: device layout of the uploaded forest (no ownership) */
typedef struct ot_state ot_state; /* opaque: view over a caller-owned device state buffer */

/* Host description of a forest (FP64). Per-body arrays have body_off[n_worlds] entries,
 * per-apple arrays apple_off[n_worlds], per-tip arrays tip_off[n_worlds]. */
typedef struct ot_tree_desc {
  int32_t n_worlds;
  const int32_t* body_off;   /* [W+1] */
  const int32_t* apple_off;  /* [W+1] */
  const int32_t* tip_off;    /* [W+1] */
  const int32_t* parent;     /* world-local parent, -1 for the root */
  const int32_t* ndof;       /* 0 (welded), 1 (hinge about x) or 2 (x then y') */
  const double* jpos;        /* [nb][3] joint origin in the parent body frame */
  const double* qrel;        /* [nb][4] rest rotation relative to the parent (w,x,y,z) */
  const double* com;         /* [nb][3] centre of mass in the body frame */
  const double* mass;        /* [nb] > 0 */
  const double* inertia;     /* [nb][3] principal moments about the com along body axes */
  const double* k;           /* [nb] joint stiffness (N m / rad), shared by the joint's DOFs */
  const double* kd;          /* [nb] joint damping (N m s / rad) */
  const double* armature;    /* [nb] added to the diagonal of H for the joint's DOFs */
  const double* m_max;       /* [nb] rupture moment (N m) */
  const int32_t* apple_body; /* [na] world-local body */
  const double* hang_local;  /* [na][3] tether hang point in the body frame */
  const double* apple_mass;  /* [na] > 0 */
  const double* k_s;         /* [na] tether stiffness */
  const double* c_s;         /* [na] tether damping (acts on the apple only) */
  const double* f_detach;    /* [na] detach force */
  const int32_t* tip_body;   /* [nt] world-local body of each recorded tip point */
  const double* tip_local;   /* [nt][3] tip point in the body frame */
  const double* gravity;     /* [W][3] */
  const double* diam;        /* [nb] segment diameter (m); may be NULL unless fp64_twig_diam > 0 */
  /* Per-body geometry and material of generated trees, for ot_model_randomize (all four, with
     diam, or none: NULL). */
  const double* length;      /* [nb] segment length (m) */
  const double* rho;         /* [nb] wood density (kg/m^3) */
  const double* youngs;      /* [nb] Young's modulus (Pa) */
  const double* sigma_r;     /* [nb] modulus of rupture (Pa) */
} ot_tree_desc;

/* Switchable readings of the model (defaults in parentheses). */
typedef struct ot_model_flags {
  int32_t alpha_implicit_spring; /* (1) 1: springs implicit, H += dt^2 K'; 0: explicit */
  int32_t tether_implicit;       /* (1) 1: tether by coupled backward Euler; 0: explicit reaction */
  int32_t n_break;               /* (5) N_b */
  int32_t n_pull;                /* (3) N_p */
  int32_t n_tension;             /* (10) N_t */
  double gamma_tension;          /* (1.2) tension threshold factor */
  double clamp_factor;           /* (1.2) reaction clamp = clamp_factor * f_detach */
  double break_ramp_s;           /* (1.5) a broken joint keeps a friction surrogate: a viscous */
  double break_ramp_factor;      /* (5.0) damper ramping from kd to factor * kd over ramp_s (s) */
  double fp64_twig_diam;         /* (0) joints of segments thinner than this (m) invert their
                                    factorisation pivot block in FP64; 0: none */
  /* Velocity-proportional damping of every segment body (Sec. IV-A), a force -c_v m v_c and a
     torque -c_omega I_c omega at its centre of mass, taken explicitly at the step's start
     velocities; on a snapped sub-tree the linear part is scaled by snapped_lin_damping
     (Sec. IV-B). All >= 0. */
  double lin_damping;            /* (0) c_v, 1/s */
  double ang_damping;            /* (0) c_omega, 1/s */
  double snapped_lin_damping;    /* (0.1) factor on c_v on a snapped sub-tree */
  /* Rails on an apple's applied force (App. B), at the step's start velocity v: (1) impulse
     cap, dt |f| / m <= v_lim; (2) power fade, the component of f pushing along v scaled by
     (v_lim - |v|) / (v_lim - v_fade) between v_fade and v_lim (0 above); (3) speed brake,
     -c_b m (|v| - v_lim) v / |v| added above v_lim. Only where an applied force acts. */
  double rail_speed;             /* (0) v_lim, m/s; 0: rails off */
  double rail_fade_speed;        /* (0) v_fade, m/s, 0 <= v_fade < v_lim when the rails are on */
  double rail_brake;             /* (0) c_b, 1/s, >= 0 */
} ot_model_flags;

/* Launch schedule of a rollout for one size class of worlds (set by the autotuner or by hand). */
typedef struct ot_schedule {
  int32_t threads_per_world;   /* 32, 64, 128, 256 or 512 */
  int32_t worlds_per_block;    /* groups of threads_per_world threads in one block */
  int32_t blocks;              /* persistent grid size (0: enough for one wave) */
  int32_t global_workspace;    /* 1: per-step temporaries in the state's scratch area (fixed
                                  at upload for classes too large for shared memory);
                                  0: all in shared memory; 2 (lean: classes of one world per
                                  SM, 128-512 threads per world): the state, apple records and
                                  snapped flags in global memory, the rest in shared memory
                                  (a rollout that writes the adjoint's tape runs such a class
                                  with 0, at the worlds per block that fit) */
  int32_t stage;               /* model records copied into shared memory per world, for all its
                                  steps (classes in shared memory only): -1 automatic, each of
                                  the parts (1 sweep topology and frames, 8 ancestor rows,
                                  4 joint rows, 2 stiffness, 64 force and apple records,
                                  16 factorisation records, 32 factorisation targets), in that
                                  order, that fits at the class's resident blocks per SM;
                                  0 none; > 0 this mask (OT_ECAPACITY at launch when it does
                                  not fit in shared memory) */
} ot_schedule;

/* What a size class resolves to under its current schedule: out[0] worlds, [1] largest world's
 * bodies, [2] per-world step temporaries in the placement used (bytes; with the lean placement
 * its shared-memory part), [3] the staged parts (mask), [4] their bytes
 * per world, [5] dynamic shared memory per block (bytes), [6] resident blocks per SM, [7] the
 * persistent grid's blocks. Sets the kernel's attributes (not inside a stream capture). */
ot_status ot_class_info(ot_model* model, int32_t size_class, int64_t out[8]);

/* ---------------------------------------------------------------------------------------
 * Model upload.
 * ot_model_bytes: device bytes the packed model needs. Host only.
 * ot_tree_model_upload: validates desc (topology, finiteness, limits), packs it to FP32 SoA,
 *   sorts worlds by estimated cost into the work queue, splits them into size classes and
 *   copies everything into dev_buf (caller-allocated, >= ot_model_bytes, 256-byte aligned)
 *   on `stream`. The host call returns after the copies are enqueued; dev_buf must stay alive
 *   while the model is used. On error *out is untouched and nothing is copied.
 * ot_model_release: frees the host handle only. */
ot_status ot_model_bytes(const ot_tree_desc* desc, size_t* bytes);
ot_status ot_tree_model_upload(const ot_tree_desc* desc, const ot_model_flags* flags, void* dev_buf,
                               size_t dev_bytes, void* stream, ot_model** out);
void ot_model_release(ot_model* model);

/* ---------------------------------------------------------------------------------------
 * Domain randomisation on the device (Sec. IV-D and VII-A: per-world geometry and material, built on the
 * GPU). factors: device [W][6] floats per world (s_len, s_diam, s_rho, s_E, s_sigma, c_d). Each
 * world's segment lengths and every body-frame point (joint origins, centres of mass, apple hang
 * points, tip points) are scaled by s_len, its diameters by s_diam, its wood density, Young's
 * modulus and modulus of rupture by s_rho, s_E, s_sigma, relative to the uploaded model, and
 * every derived per-body value is rebuilt: mass and inertia (solid cylinders, or capsule links
 * when capsule_links = 1), k = E I / l for compliant joints (I = pi r^4 / 4), kd = c_d k
 * (Sec. IV-A, Eq. 4) and the rupture moment sigma_r pi r^3 / 4 (Sec. IV-B, Eq. 5). Topology,
 * rest rotations, armature, the apples' own parameters, the size classes, schedules and the
 * FP64-pivot choice (from the uploaded diameters) are kept. Asynchronous on `stream`; rollouts
 * and graphs captured before it read the new values. Errors: OT_EINVAL for a null argument or
 * a model uploaded without length, rho, youngs, sigma_r and diam. Factors are not checked on
 * the device: non-positive ones give a non-physical model (status bits may then be set). */
ot_status ot_model_randomize(ot_model* model, const float* factors, int32_t capsule_links, void* stream);

/* Counts of the uploaded forest: worlds, bodies, DOFs, apples, tips, size classes. */
ot_status ot_model_counts(const ot_model* model, int64_t counts[6]);

/* Replace the joint stiffness k and damping kd of every body (Sec. IV-A, Eq. 4 and the damping
 * that follows it) in the uploaded model, in place, on `stream`: k, kd are device arrays [nb]
 * in the forest's body order (either may be NULL to keep the current values). Values are
 * taken as given (no check for sign or finiteness: that is the caller's). Steps and graphs
 * enqueued after this call see the new values; nothing else of the model changes. This is
 * how the differentiable rollout feeds k and kd from tensors. */
ot_status ot_model_set_gains(ot_model* model, const float* k, const float* kd, void* stream);

/* ---------------------------------------------------------------------------------------
 * World state: q, qd (FP32 per DOF), apple positions and velocities, break and detach flags,
 * counters and event steps, per-world status, plus the scratch area used by classes whose
 * per-step temporaries do not fit in shared memory.
 * ot_state_bytes: bytes of the state buffer (host only).
 * ot_world_state_alloc: makes a state view over dev_buf (>= ot_state_bytes, 256-byte aligned).
 *   Nothing is initialised: call ot_state_set. */
ot_status ot_state_bytes(const ot_model* model, size_t* bytes);
ot_status ot_world_state_alloc(const ot_model* model, void* dev_buf, size_t bytes, ot_state** out);
void ot_state_release(ot_state* state);

/* Initial state. q, qd: [n_dofs]; apple_x, apple_v: [n_apples][3]; FP32; host pointers when
 * on_device == 0 (copied synchronously), device pointers otherwise (copied on `stream`).
 * NULL q / qd / apple_v mean zeros; apple_x must be given when the forest has apples.
 * Clears all flags, counters, event steps and status words. */
typedef struct ot_state_init {
  const float* q;
  const float* qd;
  const float* apple_x;
  const float* apple_v;
  int32_t on_device;
} ot_state_init;
ot_status ot_state_set(ot_state* state, const ot_state_init* init, void* stream);

/* Device views of the state arrays (for reading results; same layout as ot_state_init plus
 * int32 per-body broken flag and break step, per-apple detached flag and detach step,
 * uint32 per-world status). Any pointer may be NULL. */
typedef struct ot_state_view {
  float* q;
  float* qd;
  float* apple_x;       /* [na][3] */
  float* apple_v;       /* [na][3] */
  int32_t* broken;      /* [nb] */
  int32_t* break_step;  /* [nb] step index of the break, -1 if none */
  int32_t* detached;    /* [na] */
  int32_t* detach_step; /* [na] */
  uint32_t* status;     /* [W] OT_WORLD_* bits */
} ot_state_view;
ot_status ot_state_get_view(const ot_state* state, ot_state_view* view);

/* Per-world status words copied (device to device) into dev_status[W] on `stream`. */
ot_status ot_world_status(const ot_state* state, uint32_t* dev_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Pull schedule on apples (device pointers): force [na][3] applied during steps
 * start[a] <= step < end[a] (absolute step indices). NULL force means no pulls. */
typedef struct ot_force_schedule {
  const float* force;
  const int32_t* start;
  const int32_t* end;
} ot_force_schedule;

/* One step of every world (step index `step` for the pull schedule and the event records),
 * with ext_force [na][3] (device, may be NULL) added to the scheduled pulls. */
ot_status ot_step(ot_model* model, ot_state* state, const float* ext_force, const ot_force_schedule* pulls,
                  int32_t step, double dt, void* stream);

/* Record of a rollout (device buffers, any may be NULL):
 *   tips: [n_steps][n_tips][3] tip positions after every step;
 *   ckpt: state snapshots taken before steps 0, ckpt_every, 2 ckpt_every, ...
 *         (ot_ckpt_bytes gives the size for n_steps);
 *   tape: the adjoint's full tape (ot_tape_bytes gives the size for n_steps; 16-byte aligned):
 *         every step's start state and what the reverse of the step reads from its forward
 *         pass (joint origins, DOF axes, the solution, apple data, the snapped flags, the
 *         factors, the end velocities, and the kinematics its kinematics sweep found), so
 *         that ot_rollout_backward runs no step again and rebuilds no kinematics. It
 *         trades memory for the replay of checkpoint segments: about 59 KB per step of a
 *         200-body world (11.7 GB for 1024 such worlds over 200 steps). Its layout is internal:
 *         the caller owns the buffer, ot_rollout writes it, and ot_rollout_backward reads it
 *         for the same model and n_steps; keep it unmodified in between.
 *   tape_steps: how many of the rollout's final steps the tape covers (0: all n_steps). With
 *         0 < tape_steps < n_steps the record must hold checkpoints too: the backward reverses
 *         the taped steps straight from the tape and replays only the earlier checkpoint
 *         segments (a tape sized by ot_tape_bytes(model, tape_steps), for rollouts whose full
 *         tape does not fit in device memory).
 * A buffer too small (or a misaligned tape) fails with OT_EINVAL before any work is queued.
 * ot_ckpt_bytes / ot_tape_bytes write the byte sizes for n_steps steps (OT_EINVAL for a NULL
 * model or bytes, n_steps < 0, or ckpt_every < 1). */
typedef struct ot_record {
  float* tips;
  void* ckpt;
  size_t ckpt_bytes;
  int32_t ckpt_every;
  float* tape;
  size_t tape_bytes;
  int32_t tape_steps;
} ot_record;
ot_status ot_ckpt_bytes(const ot_model* model, int32_t n_steps, int32_t ckpt_every, size_t* bytes);
ot_status ot_tape_bytes(const ot_model* model, int32_t n_steps, size_t* bytes);

/* n_steps steps from absolute step index step0: one persistent launch per size class over a
 * cost-sorted work queue (each group of threads pops a world and runs all its steps),
 * captured once into a CUDA graph per (n_steps, record layout, schedules) with the classes as
 * independent branches (they overlap on the GPU), and replayed on `stream`. */
ot_status ot_rollout(ot_model* model, ot_state* state, int32_t n_steps, int32_t step0, double dt,
                     const ot_force_schedule* pulls, const ot_record* record, void* stream);

/* The plain form: one kernel launch per world per step (no queue, no graph, no autotune). */
ot_status ot_rollout_plain(ot_model* model, ot_state* state, int32_t n_steps, int32_t step0, double dt,
                           const ot_force_schedule* pulls, void* stream);

/* ---------------------------------------------------------------------------------------
 * Adjoint of a recorded rollout with the break and detach masks frozen as recorded (an
 * addition: the paper simulates forward only and never differentiates the step).
 * The forward must have been run by ot_rollout with the same model, n_steps, step0, dt and
 * pulls, and a record holding a tape or checkpoints (ckpt, ckpt_every); with both, the tape is
 * used. A world the forward froze on a non-finite state gets NaN gradients (tape) or whatever
 * its replay gives (checkpoints). The caller gives the cotangent
 * of the recorded tips, dL_dtips [n_steps][n_tips][3] (device); for the tip-tracking loss
 * L = sum_t sum_tips |p_t - p*_t|^2 / (n_steps n_tips_of_world) it is 2 (p - p*) / (...).
 * Gradients (device, any may be NULL): dk, dkd [nb] per joint are ACCUMULATED into; dq0,
 * dqd0 [n_dofs] (the initial state) are written. Without a tape, each segment between
 * checkpoints is recomputed forward with the forward's step code (equal to the recorded run up
 * to the last bits: it is compiled into another kernel) and then swept in reverse step by step;
 * with a tape, the steps are swept in reverse straight from it.
 * workspace: device buffer of at least ot_backward_workspace_bytes bytes (256-byte aligned),
 * queried with the record's ckpt_every, or 0 for a record with a tape (no segment buffers);
 * NULL when that size is 0. */
typedef struct ot_grads {
  float* dk;
  float* dkd;
  float* dq0;
  float* dqd0;
} ot_grads;
ot_status ot_backward_workspace_bytes(const ot_model* model, int32_t ckpt_every, size_t* bytes);
/* Backward schedules: the backward kernel's threads per world for size class c (64, 128 or 256;
 * 0 restores the default by tree size: 64 up to 96 bodies, else 256). ot_autotune_backward
 * takes ot_rollout_backward's arguments (a recorded rollout), times each candidate of each
 * class on it with CUDA events on `stream`, one class at a time, and keeps the fastest. The
 * grads then hold meaningless values (they serve as scratch); run ot_rollout_backward again
 * for the gradients. The workspace size
 * (ot_backward_workspace_bytes) fits every candidate, so it does not change with the choice. */
ot_status ot_get_backward_schedule(const ot_model* model, int32_t size_class, int32_t* threads_per_world);
ot_status ot_set_backward_schedule(ot_model* model, int32_t size_class, int32_t threads_per_world);
ot_status ot_autotune_backward(ot_model* model, ot_state* state, int32_t n_steps, int32_t step0, double dt,
                               const ot_force_schedule* pulls, const ot_record* record, const float* dL_dtips,
                               ot_grads* grads, void* workspace, size_t workspace_bytes, void* stream);
ot_status ot_rollout_backward(ot_model* model, ot_state* state, int32_t n_steps, int32_t step0, double dt,
                              const ot_force_schedule* pulls, const ot_record* record, const float* dL_dtips,
                              ot_grads* grads, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Schedules and autotuning. Size classes are formed at upload from the world sizes.
 * ot_get_schedule / ot_set_schedule read or replace the schedule of class c.
 * ot_autotune times every candidate schedule of every class on `n_steps` steps with CUDA
 * events on `stream`: each class alone, then its three fastest with all classes running
 * together as a rollout runs them; it keeps the fastest. Every timed launch starts from the
 * state as it was at the call (the call allocates one device copy of the state arrays, and
 * frees it before returning), and the state is restored at the end. Synchronous: returns after
 * the restore has completed on `stream`. */
ot_status ot_get_schedule(const ot_model* model, int32_t size_class, ot_schedule* sched);
ot_status ot_set_schedule(ot_model* model, int32_t size_class, const ot_schedule* sched);
ot_status ot_autotune(ot_model* model, ot_state* state, int32_t n_steps, double dt, void* stream);

/* ---------------------------------------------------------------------------------------
 * Allocation-free step (the paper has no counterpart; this is a library convenience).
 * ot_step_static_scratch does what ot_step does, but the per-world temporaries of the step
 * live in a fixed array compiled into the library instead of the state's scratch area, so a
 * caller that cannot allocate device memory while it steps (a control loop that must not
 * stall or fail on an allocation mid-run, or a host program with a fixed device-memory
 * budget that only holds the model and state buffers) needs nothing more. The caller still
 * passes the model, the state, the forces and the stream.
 *   - Size: OT_STATIC_SCRATCH_BYTES per GPU, held from library load until process exit. A
 *     world whose temporaries exceed it (minus 256 bytes of counters) is rejected with
 *     OT_ECAPACITY, and a state of another model or a pull schedule without its start and
 *     end arrays with OT_EINVAL; every check runs before any work is queued, so a rejected
 *     call changes nothing. A class whose schedule asks for more worlds per block than the
 *     array has slots for runs with fewer worlds per block.
 *   - The array's device address is looked up with cudaGetSymbolAddress on the first call on
 *     each device (with that device current); make that first call outside any stream capture.
 *   - Every call uses the same array and leaves its contents behind; the call clears what must
 *     start at zero. Calls that overlap on the GPU (other streams, other host threads) race:
 *     serialise them.
 *   - No device memory is allocated or freed. */
#define OT_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
ot_status ot_step_static_scratch(ot_model* model, ot_state* state, const float* ext_force,
                                 const ot_force_schedule* pulls, int32_t step, double dt, void* stream);

/* ---------------------------------------------------------------------------------------
 * Diagnostics. */
const char* ot_status_string(ot_status s);
int32_t ot_last_cuda_error(void);
/* Number of kernel launches the library issued since the last reset (graph replays count
 * each kernel node once). */
int64_t ot_launch_count(int32_t reset);
/* Phase clocks, for profiling only: available in the instrumented build of the library
 * (compiled with ORCHARD_PHASE_CLOCKS), OT_EINVAL in the product build. Copies max_classes
 * (at most 64) rows of 10 counters into out (host, [row][10]). Row k < 32: size class k's
 * rollouts, the SM cycles summed over all world-steps since the last reset for each phase of
 * the step (forward kinematics sweep, forces and apple loads, tip record, bias sweep,
 * mass-matrix rows, LDL^T, update sweep, apple update, the rest of the rollout), then the
 * world-step count. Row 32 + k: class k's backward passes (apple update reverse and hang-point
 * loads, the solve with the step's factors, the L sweep with springs and tape, the seeds, the
 * leaf-to-root chain, restoring a step's start state and record, segment replays, the final
 * seed, the rest), then the world-steps reversed. Synchronises the device; reset != 0 zeroes
 * the counters afterwards. */
ot_status ot_phase_clocks(const ot_model* model, uint64_t* out, int32_t max_classes, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* ORCHARD_H */
