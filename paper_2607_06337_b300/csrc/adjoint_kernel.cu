// Backward (adjoint) kernel of a recorded rollout for sm_103a: a persistent grid whose thread
// groups pop worlds from the cost-sorted queue and run backward_world (adjoint_device.cuh).
// Each group owns one slot of the caller's workspace (the snapshots of one checkpoint
// segment, none when the forward kept its full tape, plus whatever of its temporaries is not
// in shared memory). The checkpoint, tape and hybrid forms (MODE 0, 1, 2) are separate
// instantiations. BackShape::mode says which temporaries live in the block's shared memory:
//   0: none (forward and backward temporaries in the global slot),
//   1: the forward step's temporaries (WsLayout),
//   2: the forward step's and the backward's (WsLayout, then AdjLayout),
//   3: the forward step's and the backward's up to the C slots, which open the global slot,
//   4: the forward step's and the backward's up to the tape T; T, then the C slots, open the
//      global slot.
#include "adjoint_device.cuh"

namespace orchard {
namespace {

template <int TPW, int MODE>
__global__ void __launch_bounds__(kBackMaxThreads, 2) backward_kernel(DevModel m, StepArgs a, BackArgs ba, float* work,
                                                       BackShape sh) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int frozen[16];
  __shared__ int next[16];
  Group<TPW> g;
  g.lane = threadIdx.x % TPW;
  g.id = threadIdx.x / TPW;
  g.flag = &frozen[g.id];
  const int groups = blockDim.x / TPW;
  float* slot = work + (long long)(blockIdx.x * groups + g.id) * sh.global_floats;
  float* local = smem + (long long)g.id * sh.smem_floats;
  float *ws, *wa, *seg, *wt = nullptr, *wc = nullptr;
  if (sh.mode == 4) {
    ws = local;
    wa = local + sh.fwd_floats;
    wt = slot;
    wc = slot + sh.t_floats;
    seg = wc + sh.c_floats;
  } else if (sh.mode == 3) {
    ws = local;
    wa = local + sh.fwd_floats;
    wc = slot;
    seg = slot + sh.c_floats;
  } else if (sh.mode == 2) {
    ws = local;
    wa = local + sh.fwd_floats;
    seg = slot;
  } else if (sh.mode == 1) {
    ws = local;
    wa = slot;
    seg = slot + sh.adj_floats;
  } else {
    ws = slot;
    wa = slot + sh.fwd_floats;
    seg = wa + sh.adj_floats;
  }
  for (;;) {
    if (g.lane == 0) next[g.id] = atomicAdd(a.q_counter, 1);
    g.sync();
    const int qi = next[g.id];
    g.sync();
    if (qi >= a.q_end - a.q_begin) break;
    backward_world<TPW, MODE>(m, a, ba, m.queue[a.q_begin + qi], ws, wa, wt, wc, seg, g);
  }
}

template <int TPW>
const void* backward_fn(int mode) {
  return mode == 1 ? (const void*)backward_kernel<TPW, 1>
                   : mode == 2 ? (const void*)backward_kernel<TPW, 2> : (const void*)backward_kernel<TPW, 0>;
}

const void* backward_fn_of(int tpw, int mode) {
  switch (tpw) {
    case 32: return backward_fn<32>(mode);
    case 64: return backward_fn<64>(mode);
    case 128: return backward_fn<128>(mode);
    case 256: return backward_fn<256>(mode);
    default: return nullptr;
  }
}

// 0: checkpoints, 1: the full tape, 2: the tape for the last steps, checkpoints before
inline int back_mode(const StepArgs& a) { return !a.tape ? 0 : a.tape_steps < a.n_steps ? 2 : 1; }

template <int TPW>
void launch_of(int blocks, int threads, size_t smem, cudaStream_t st, const DevModel& m, const StepArgs& a,
               const BackArgs& ba, float* work, const BackShape& sh) {
  switch (back_mode(a)) {
    case 1: backward_kernel<TPW, 1><<<blocks, threads, smem, st>>>(m, a, ba, work, sh); break;
    case 2: backward_kernel<TPW, 2><<<blocks, threads, smem, st>>>(m, a, ba, work, sh); break;
    default: backward_kernel<TPW, 0><<<blocks, threads, smem, st>>>(m, a, ba, work, sh); break;
  }
}

}  // namespace

void launch_backward(int tpw, int groups_per_block, int blocks, cudaStream_t st, const DevModel& m,
                     const StepArgs& a, const BackArgs& ba, float* work, const BackShape& sh) {
  const int threads = tpw * groups_per_block;
  const size_t smem = (size_t)sh.smem_floats * 4 * groups_per_block;
  switch (tpw) {
    case 32: launch_of<32>(blocks, threads, smem, st, m, a, ba, work, sh); break;
    case 64: launch_of<64>(blocks, threads, smem, st, m, a, ba, work, sh); break;
    case 128: launch_of<128>(blocks, threads, smem, st, m, a, ba, work, sh); break;
    case 256: launch_of<256>(blocks, threads, smem, st, m, a, ba, work, sh); break;
    default: break;
  }
}

cudaError_t backward_attributes(int tpw, int mode, int groups_per_block, size_t smem_bytes, int* blocks_per_sm) {
  const void* fn = backward_fn_of(tpw, mode);
  if (!fn) return cudaErrorInvalidValue;
  if (smem_bytes > kSmemLimitBytes) return cudaErrorInvalidValue;
  // the attribute belongs to the instantiation, shared by every class using it: always the limit
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimitBytes);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, tpw * groups_per_block, smem_bytes);
}

long long backward_adj_floats(int nb, int nv, int na) { return AdjLayout::make(nb, nv, na).total; }
long long backward_adj_head_floats(int nb, int nv, int na) { return AdjLayout::make(nb, nv, na).head; }
long long backward_adj_small_floats(int nb, int nv, int na) { return AdjLayout::make(nb, nv, na).small; }
long long backward_reverse_ws_floats(int nb, int nv, int nm, int na) {
  return WsLayout::make_reverse(nb, nv, nm, na).total;
}

long long backward_seg_floats(int nb, int nv, int nm, int na, int ckpt_every) {
  return (long long)ckpt_every * WsLayout::tape_unit(nb, nv, nm, na);
}

}  // namespace orchard
