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
  const int4* dinfo;     // per DOF: row start (world-local), body, depth d_i, -
  const unsigned short* anc;  // per row entry c of DOF i: world-local DOF id of its c-th ancestor
  const float4* ap0;     // hang point in the body frame (xyz), apple mass (w)
  const float4* ap1;     // k_s, c_s, f_detach, -
  const int* apple_body; // world-local body of each apple
  const int* tip_body;   // world-local body of each tip
  const float4* tip_local;
  const float4* gravity; // per world
  const int* queue;      // world ids sorted by (size class, cost descending)
  const unsigned char* pairs;  // (c, c2) pairs 1 <= c <= c2 <= d, ordered by c2 then c
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
  int NB, NV, NA;           // totals (snapshot layout)
  int q_begin, q_end;       // queue range of this launch
  int* q_counter;           // next queue entry (relative to q_begin); null: one world per group
  int single_world;         // >= 0: the plain form, this world only
  long long ws_floats;      // workspace floats per group
  int global_ws;            // 1: workspace in DevState::scratch, slot = global group index
};

// Workspace layout of one world (floats), a function of its sizes only.
struct WsLayout {
  int R, X, V, A, F, IC, E, M, r, AT, SN, total;
  __host__ __device__ static WsLayout make(int nb, int nv, int nm, int na) {
    WsLayout L;
    L.R = 0;
    L.X = L.R + 9 * nb;
    L.V = L.X + 3 * nb;
    L.A = L.V + 6 * nb;
    L.F = L.A + 6 * nb;
    L.IC = L.F + 6 * nb;
    L.E = L.IC + 10 * nb;
    L.M = L.E + 3 * nv;
    L.r = L.M + nm;
    L.AT = L.r + nv;
    L.SN = L.AT + 8 * na;  // per body: 1 when on a snapped sub-tree
    L.total = L.SN + nb;
    return L;
  }
};

constexpr size_t kSmemLimitBytes = 226 * 1024;  // dynamic shared memory per block we use at most
constexpr int kMaxDepth = 63;  // DOF depth limit (pair table size)
constexpr int kPairCount = (kMaxDepth + 1) * (kMaxDepth + 2) / 2;

void launch_rollout(int tpw, int groups_per_block, int blocks, size_t smem_bytes, cudaStream_t s,
                    const DevModel& m, const DevState& st, const StepArgs& a);
cudaError_t kernel_attributes(int tpw, int groups_per_block, size_t smem_bytes, int* blocks_per_sm);

}  // namespace orchard
