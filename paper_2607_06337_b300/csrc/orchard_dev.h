// Internal device-side layout shared by the kernels and the host side of liborchard.
// (Not part of the public ABI: include/orchard.h is.)
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace orchard {

// Packed model in device memory (all pointers into the caller's model buffer).
// Bodies, DOFs, apples and tips are stored in world order; world w owns the ranges given by
// the *_off arrays. Everything inside a world is indexed world-locally.
struct DevModel {
  int W;
  const int* body_off;   // [W+1]
  const int* dof_off;    // [W+1]
  const int* apple_off;  // [W+1]
  const int* tip_off;    // [W+1]
  const int* m_off;      // [W+1] start of the world's ancestor-row storage (entries)
  const int* lvl_off;    // [W+1] start of the world's level boundaries in lvl
  const int* lvl;        // world-local first body of each level, plus one past the last
  // per body: x parent, y dof0 | ndof << 28, z child_first | child_count << 24,
  //           w apple_first | apple_count << 24
  const int4* bi;
  const float4* bp0;     // joint origin in the parent frame (xyz), mass (w)
  const float4* bp1;     // rest rotation quaternion (w, x, y, z)
  const float4* bp2;     // com in the body frame (xyz), Ixx (w)
  const float4* bp3;     // Iyy, Izz, k, kd
  const float4* bp4;     // armature, m_max, -, -
  const int4* bj;        // per body: its first DOF's row start, the second DOF's row start (-1 for
                         // a one-DOF joint), the first DOF's depth, the DOF count | 16 if the
                         // pivot is inverted in FP64 (zeros, y = -1, for a body without DOFs)
  const unsigned* anc;   // per row entry c of DOF i: its c-th ancestor DOF j | (body of j) << 16
  const int* bl_off;     // [W+1] start of the world's factorisation level boundaries in bl_bound
  const int* bl_bound;   // world-local level position of each level's first body (+ end). A level
                         // holds the bodies with DOFs whose first DOF has that depth, in
                         // depth-first preorder
  const int4* bl_info;   // per level position (world-local, at the world's body offset): the
                         // body's first DOF, its row start, the second DOF's row start (-1 for a
                         // one-DOF joint), the DOF count | 16 if the pivot is inverted in FP64
  const int* bl_fbase;   // parallel to bl_bound: each level's first entry in the fac_tgt block
  const int* fac_off;    // [W+1] start of the world's fac_tgt block
  const int2* fac_tgt;   // per level l, ancestor distance c (1..l), position p in the level:
                         // entry (c - 1) * count_l + p = {row start of the c-th ancestor of the
                         // p-th body's first DOF minus c (the factorisation's target base), that
                         // ancestor}
  const int* bl_ibase;   // parallel to bl_bound: each level's first factorisation work item
  const int* fit_off;    // [W+1] start of the world's work items in fitem
  const int4* fitem;     // per level, its work items {c, first position, end position, scan
                         // count}: the positions [first, end) of ancestor distance c, cut only
                         // between groups of positions that share their c-th ancestor, largest
                         // first
  const float4* ap0;     // hang point in the body frame (xyz), apple mass (w)
  const float4* ap1;     // k_s, c_s, f_detach, -
  const int* apple_body; // world-local body of each apple
  const int* tip_body;   // world-local body of each tip
  const int* btip;       // per body: first tip (world-local) | tip count << 24 (tips sorted by body)
  const float4* tip_local;
  const float4* gravity; // per world
  const int* queue;      // world ids sorted by (size class, cost descending)
  const long long* tape_off;  // [W+1] prefix sums of WsLayout::tape_unit over the worlds: the
                              // tape of a T-step rollout gives world w floats from (T + 1) tape_off[w]
  const int2* apre;      // per apple slot (world-local, at the world's apple offset): {apple,
                         // its body}, ordered by the body's depth-first preorder position
  const int2* arange;    // per body: the slots [x, y) in apre of the apples in its subtree
};

// State arrays in device memory (views into the caller's state buffer).
struct DevState {
  float* q;          // [NV]
  float* qd;         // [NV]
  float* ax;         // [NA*3]
  float* av;         // [NA*3]
  int* broken;       // [NB]
  int* bcnt;         // [NB]
  int* break_step;   // [NB]
  int* detached;     // [NA]
  int* pcnt;         // [NA]
  int* tcnt;         // [NA]
  int* detach_step;  // [NA]
  unsigned* status;  // [W]
  float* scratch;    // global per-step workspace for classes that do not fit in shared memory
};

// Per-launch arguments.
struct StepArgs {
  float dt;
  int alpha;            // implicit springs
  int tether_implicit;
  int n_break, n_pull, n_tension;
  float gamma, clamp;
  float ramp_inv;       // 1 / (post-break ramp time in steps), 0: no ramp (full factor at once)
  float ramp_gain;      // post-break damper factor minus one
  float cv, cv_snap;    // body damping c_v, and c_v on a snapped sub-tree (1/s)
  float cw;             // body damping c_omega (1/s)
  float rail_v;         // applied-force rails: v_lim (0: off), v_fade, 1 / (v_lim - v_fade),
  float rail_vf;        // v_lim / dt (the impulse cap per unit mass), brake c_b
  float rail_inv, rail_cap, rail_cb;
  int step0;            // absolute index of the first step of this launch
  int n_steps;
  const float* pull_force;  // [NA*3] or null
  const int* pull_start;
  const int* pull_end;
  const float* ext_force;   // [NA*3] or null (added during every step of the launch)
  float* tips;              // [n_steps][NT][3] or null
  int n_tips_total;
  unsigned* ckpt;           // snapshots or null
  int ckpt_every;
  long long ckpt_words;     // 32-bit words per snapshot
  float* tape;              // the adjoint's tape of the rollout (written by the forward, read by
                            // the backward), or null
  int tape_steps;           // the final steps the tape covers (n_steps: all; fewer: the earlier
                            // ones come from the checkpoints)
  int NB, NV, NA;           // totals (snapshot layout)
  int q_begin, q_end;       // queue range of this launch
  int* q_counter;           // next queue entry (relative to q_begin); null: one world per group
  int single_world;         // >= 0: the plain form, this world only
  long long ws_floats;      // workspace floats per group
  int global_ws;            // 1: workspace in DevState::scratch, slot = global group index
  unsigned long long* phase_clk;  // instrumented builds only (ORCHARD_PHASE_CLOCKS): this
                                  // launch's kPhaseSlots accumulators, or null
  int stage_mask;           // StageLayout parts copied into shared memory per world (0: none)
  long long stage_floats;   // shared-memory floats per group for them (the class's largest world)
  int lean;                 // 1: the lean placement (WsLayout::make_lean; never with a tape)
  long long lean_floats;    // floats per group of its global slots in DevState::scratch
};

// Parts of a world's model that a rollout can stage in shared memory (after the workspace),
// copied once when a group takes the world and read from there for all its steps.
enum StagePart {
  kStageKin = 1,     // bi, bp0, bp1: kinematics sweep (and the topology of every pass)
  kStageBias = 2,    // bp3: bias sweep (stiffness, damping)
  kStageUpd = 4,     // bj, bp4: update sweep, mass matrix (joint rows, armature, rupture moment)
  kStageAnc = 8,     // anc: ancestor ids of the mass-matrix rows (L sweep, mass matrix)
  kStageInfo = 16,   // bl_info, fitem: factorisation level records and work items
  kStageFac = 32,    // fac_tgt: factorisation targets
  kStageForce = 64,  // bp2, ap0, ap1, apple_body: forces and apples
};
// The order in which the automatic choice takes the parts, each one that still fits (measured
// on B300: the ancestor walks of the L sweep and the mass matrix gain most, the factorisation's
// tables least, since its loads are issued one step ahead).
constexpr int kStageOrder[7] = {kStageKin, kStageAnc, kStageUpd, kStageBias, kStageForce, kStageInfo, kStageFac};

// The staged area of a world opens with a table of one pointer per model record array (kTab*):
// to the array's copy in shared memory when its part is staged, else to the world's records in
// global memory. The step reads a record through the table, so no pointer stays in a register.
enum StageTab {
  kTabBi, kTabBj, kTabInfo, kTabP0, kTabP1, kTabP2, kTabP3, kTabP4, kTabA0, kTabA1, kTabAnc, kTabFac,
  kTabItems, kTabAbody, kTabEntries
};
constexpr int kStageTableFloats = 32;  // kTabEntries 8-byte pointers, rounded up to 16 bytes
static_assert(2 * kTabEntries <= kStageTableFloats, "stage table");

// Float offsets of the staged parts of one world (each on a 16-byte boundary, after the table);
// -1: not staged. total: the whole staged area, 0 when nothing is staged.
struct StageLayout {
  int bi, bp0, bp1, bp3, bj, bp4, anc, info, items, fac, bp2, ap0, ap1, abody, total;
  __host__ __device__ static int r4(int n) { return (n + 3) & ~3; }
  __host__ __device__ static StageLayout make(int mask, int nb, int nm, int na, int nfac, int nitem) {
    StageLayout S;
    int o = mask ? kStageTableFloats : 0;
    auto take = [&](int part, int floats) {
      if (!(mask & part)) return -1;
      const int at = o;
      o += r4(floats);
      return at;
    };
    S.bi = take(kStageKin, 4 * nb);
    S.bp0 = take(kStageKin, 4 * nb);
    S.bp1 = take(kStageKin, 4 * nb);
    S.bp3 = take(kStageBias, 4 * nb);
    S.bj = take(kStageUpd, 4 * nb);
    S.bp4 = take(kStageUpd, 4 * nb);
    S.anc = take(kStageAnc, nm);
    S.info = take(kStageInfo, 4 * nb);
    S.items = take(kStageInfo, 4 * nitem);
    S.fac = take(kStageFac, 2 * nfac);
    S.bp2 = take(kStageForce, 4 * nb);
    S.ap0 = take(kStageForce, 4 * na);
    S.ap1 = take(kStageForce, 4 * na);
    S.abody = take(kStageForce, na);
    S.total = o;
    return S;
  }
};

// Phase clocks of the instrumented build (ORCHARD_PHASE_CLOCKS): per size class, SM cycles
// summed over every world-step of each phase of the step, then the world-step count.
// Phases: forward kinematics sweep, forces and apple loads, tip record, bias and composite
// inertia sweep, mass-matrix rows, LDL^T with the L^T sweep, L sweep and update sweep, apple
// update and detach tests, and the rest of the rollout (state staging, checkpoints, tape).
constexpr int kPhases = 9;
constexpr int kPhaseSlots = kPhases + 1;
constexpr int kPhaseClasses = 64;
constexpr int kBackPhaseRow = 32;  // rows kBackPhaseRow + k: the backward of class k
// Device address of the accumulators ([kPhaseClasses][kPhaseSlots]), null in the product build.
unsigned long long* phase_clock_buffer();

// Workspace layout of one world (floats), a function of its sizes only. Rotations, bias
// accelerations and forces (live in the two sweeps) share space with the mass-matrix rows
// (live from the mass matrix to the end of the step). Each body's velocity (w, v: live from the
// kinematics sweep to the force pass, and from the update sweep to the next step's kinematics)
// shares its 10-float slot with its spatial, then composite, inertia (live from the force pass
// to the mass matrix): the force pass reads a body's velocity before it writes the body's
// inertia, and no pass reads another body's velocity there. S holds the world's state for the
// whole rollout (see staged_view): the step reads and writes it there, not in global memory.
constexpr int kVel = 10;  // float stride of the body velocities (the inertia slots)
struct WsLayout {
  int X, E, IC, r, AT, V, SN, S, R, A, F, M, total;
  // every region starts on a 16-byte boundary, so whole regions move as float4
  __host__ __device__ static int r4(int n) { return (n + 3) & ~3; }
  __host__ __device__ static int state_words(int nb, int nv, int na) {
    return 2 * r4(nv) + 6 * na + 3 * nb + 4 * na + 1;  // q and qd each padded to 4 floats
  }
  // The adjoint's tape of a T-step rollout, per world: T + 1 snapshots of the staged state (before
  // every step, then the final state), then T step records, each holding what the reverse of the
  // step reads from its forward workspace: joint origins and DOF axes, the solution Delta and the
  // apple data, the snapped flags, the factors, and qd at the step's end; then (kin_offset) the
  // step's kinematics as its kinematics sweep found them, kKin floats per body: R (3 columns),
  // x_b, w, v at x_b, and the velocity-product accelerations alpha, a (gravity as a base
  // acceleration, no joint acceleration).
  static constexpr int kKin = 24;
  __host__ __device__ static int snap_words(int nb, int nv, int na) { return r4(state_words(nb, nv, na)); }
  __host__ __device__ static long long kin_offset(int nb, int nv, int nm, int na) {
    const WsLayout L = make(nb, nv, nm, na);
    return (long long)r4(L.E - L.X + 3 * nv) + r4(L.AT - L.r + 10 * na) + r4(nb) + r4(nm) + r4(nv);
  }
  __host__ __device__ static long long record_words(int nb, int nv, int nm, int na) {
    return kin_offset(nb, nv, nm, na) + (long long)kKin * nb;
  }
  __host__ __device__ static long long tape_unit(int nb, int nv, int nm, int na) {
    return snap_words(nb, nv, na) + record_words(nb, nv, nm, na);
  }
  // The regions a step's reverse reads, packed (the adjoint without a step to replay): joint
  // origins and DOF axes, the solution and the apple data, the snapped flags, the staged state
  // and the factors. The sweep temporaries and the inertias (IC, V, R, A, F) are absent (-1).
  __host__ __device__ static WsLayout make_reverse(int nb, int nv, int nm, int na) {
    WsLayout L;
    L.X = 0;
    L.E = L.X + r4(3 * nb);
    L.r = L.E + r4(3 * nv);
    L.AT = L.r + r4(nv);
    L.SN = L.AT + r4(10 * na);
    L.S = L.SN + r4(nb);
    L.M = L.S + r4(state_words(nb, nv, na));
    L.total = L.M + r4(nm);
    L.IC = L.V = L.R = L.A = L.F = -1;
    return L;
  }
  // The lean placement of the step's temporaries: the regions the sweeps, the mass matrix and
  // the factorisation use (X, E, IC with V, r, and the shared region) in shared memory; the
  // state stays in the world's state arrays in global memory, and the apple records (AT) and
  // the snapped flags (SN) go to the group's slot of global memory (lean_slot_floats floats:
  // AT at 0, SN at lean_sn). Offsets AT, SN and S are -1. No tape is written in this placement.
  __host__ __device__ static WsLayout make_lean(int nb, int nv, int nm, int na) {
    WsLayout L;
    L.X = 0;
    L.E = L.X + r4(3 * nb);
    L.IC = L.E + r4(3 * nv);
    L.r = L.IC + r4(10 * nb);
    L.V = L.IC;
    L.AT = L.SN = L.S = -1;
    const int u = L.r + r4(nv);
    L.R = u;
    L.A = L.R + r4(9 * nb);
    L.F = L.A + r4(6 * nb);
    L.M = u;
    const int end_sweeps = L.F + r4(6 * nb), end_m = L.M + r4(nm);
    L.total = end_sweeps > end_m ? end_sweeps : end_m;
    return L;
  }
  __host__ __device__ static int lean_sn(int na) { return r4(10 * na); }
  __host__ __device__ static int lean_slot_floats(int nb, int na) { return r4(10 * na) + r4(nb); }
  __host__ __device__ static WsLayout make(int nb, int nv, int nm, int na) {
    WsLayout L;
    L.X = 0;                         // joint origins
    L.E = L.X + r4(3 * nb);          // DOF axes
    L.IC = L.E + r4(3 * nv);         // spatial (then composite) inertias about x_b
    L.r = L.IC + r4(10 * nb);        // right-hand side, then the solution
    L.AT = L.r + r4(nv);             // per apple: velocity with the hang point frozen, beta,
                                     // tension, pull, hang offset r_h (10 floats)
    L.V = L.IC;                      // body velocities (start of step, then end of step), in
                                     // the first 6 floats of each inertia slot (kVel)
    L.SN = L.AT + r4(10 * na);       // 1 on a snapped sub-tree
    L.S = L.SN + r4(nb);             // the staged state
    const int u = L.S + r4(state_words(nb, nv, na));  // shared region
    L.R = u;
    L.A = L.R + r4(9 * nb);
    L.F = L.A + r4(6 * nb);
    L.M = u;
    const int end_sweeps = L.F + r4(6 * nb), end_m = L.M + r4(nm);
    L.total = end_sweeps > end_m ? end_sweeps : end_m;
    return L;
  }
};

constexpr size_t kSmemLimitBytes = 226 * 1024;  // dynamic shared memory per block we use at most
constexpr int kMaxDepth = 255;  // DOF depth limit

}  // namespace orchard

struct ot_model;
struct ot_state;
struct ot_force_schedule;

namespace orchard {

// The static-scratch entry's one-step launches, the workspace in a caller-held area of
// scratch_floats floats. static_step_plan validates everything a launch could reject (the
// state's model, the pull schedule, a world too large for the area, the kernel attributes) and
// fills every class's shape before anything is queued; static_step_class then launches class
// k with its shape.
struct StaticShape {
  int worlds_per_block;  // the class's schedule, capped at the area's slot count
  int blocks;
};
int static_step_plan(ot_model* m, const ot_state* s, const ot_force_schedule* pulls, size_t scratch_floats,
                     int max_classes, int* n_classes, StaticShape* shapes);
int static_step_class(ot_model* m, ot_state* s, int k, const StaticShape& sh, const float* ext_force,
                      const ot_force_schedule* pulls, int step, double dt, float* scratch, int* counter, void* stream);

// Outputs and inputs of a backward pass beyond the forward's StepArgs.
struct BackArgs {
  const float* dtips;  // [n_steps][n_tips_total][3]
  float* dk;           // [NB] accumulated
  float* dkd;          // [NB] accumulated
  float* dq0;          // [NV] written
  float* dqd0;         // [NV] written
};
// Where a backward group keeps its temporaries (see adjoint_kernel.cu): mode 0 all in its
// global slot, 1 the forward step's in shared memory, 2 the forward's and the backward's in
// shared memory, 3 the forward's and the backward's but the C slots in shared memory; the
// checkpoint segment's snapshots always in the global slot.
struct BackShape {
  int mode;
  long long fwd_floats;     // forward temporaries of the class's largest world (WsLayout, or
                            // WsLayout::make_reverse for the tape-only backward)
  long long adj_floats;     // backward temporaries (AdjLayout)
  long long small_floats;   // the part of them before the tape T (AdjLayout::small)
  long long head_floats;    // the part of them before the C slots (AdjLayout::head)
  long long t_floats;       // the tape T (36 per body)
  long long c_floats;       // the C slots (44 per body)
  long long smem_floats;    // per group in shared memory
  long long global_floats;  // per slot of the workspace
};
// Threads per block of the backward kernel at most (two such blocks per SM: 128 registers per
// thread, which the reverse sweep needs without spilling; measured faster on B300 than 512).
constexpr int kBackMaxThreads = 256;
void launch_backward(int tpw, int groups_per_block, int blocks, cudaStream_t st, const DevModel& m,
                     const StepArgs& a, const BackArgs& ba, float* work, const BackShape& sh);
cudaError_t backward_attributes(int tpw, int mode, int groups_per_block, size_t smem_bytes, int* blocks_per_sm);
long long backward_adj_floats(int nb, int nv, int na);
long long backward_adj_head_floats(int nb, int nv, int na);
long long backward_adj_small_floats(int nb, int nv, int na);
long long backward_reverse_ws_floats(int nb, int nv, int nm, int na);
long long backward_seg_floats(int nb, int nv, int nm, int na, int ckpt_every);

void launch_rollout(int tpw, int groups_per_block, int blocks, size_t smem_bytes, cudaStream_t s,
                    const DevModel& m, const DevState& st, const StepArgs& a);
// Occupancy of the rollout kernel for tpw threads per world, the staged instantiation or not,
// the lean one (128-512 threads) or not.
cudaError_t kernel_attributes(int tpw, bool staged, bool lean, int groups_per_block, size_t smem_bytes,
                              int* blocks_per_sm);

}  // namespace orchard
