// Backward (adjoint) kernel of a recorded rollout for sm_103a: a persistent grid whose thread
// groups pop worlds from the cost-sorted queue and run backward_world (adjoint_device.cuh),
// each in its own slot of the caller's workspace.
#include "adjoint_device.cuh"

namespace orchard {
namespace {

template <int TPW>
__global__ void __launch_bounds__(512) backward_kernel(DevModel m, StepArgs a, BackArgs ba, float* work,
                                                       long long ws_floats) {
  __shared__ int frozen[16];
  __shared__ int next[16];
  Group<TPW> g;
  g.lane = threadIdx.x % TPW;
  g.id = threadIdx.x / TPW;
  g.flag = &frozen[g.id];
  const int groups = blockDim.x / TPW;
  float* ws = work + (long long)(blockIdx.x * groups + g.id) * ws_floats;
  for (;;) {
    if (g.lane == 0) next[g.id] = atomicAdd(a.q_counter, 1);
    g.sync();
    const int qi = next[g.id];
    g.sync();
    if (qi >= a.q_end - a.q_begin) break;
    backward_world<TPW>(m, a, ba, m.queue[a.q_begin + qi], ws, g);
  }
}

}  // namespace

void launch_backward(int tpw, int groups_per_block, int blocks, cudaStream_t st, const DevModel& m,
                     const StepArgs& a, const BackArgs& ba, float* work, long long ws_floats) {
  const int threads = tpw * groups_per_block;
  switch (tpw) {
    case 32: backward_kernel<32><<<blocks, threads, 0, st>>>(m, a, ba, work, ws_floats); break;
    case 64: backward_kernel<64><<<blocks, threads, 0, st>>>(m, a, ba, work, ws_floats); break;
    case 128: backward_kernel<128><<<blocks, threads, 0, st>>>(m, a, ba, work, ws_floats); break;
    case 256: backward_kernel<256><<<blocks, threads, 0, st>>>(m, a, ba, work, ws_floats); break;
    default: break;
  }
}

cudaError_t backward_attributes(int tpw, int groups_per_block, int* blocks_per_sm) {
  const void* fn = nullptr;
  switch (tpw) {
    case 32: fn = (const void*)backward_kernel<32>; break;
    case 64: fn = (const void*)backward_kernel<64>; break;
    case 128: fn = (const void*)backward_kernel<128>; break;
    case 256: fn = (const void*)backward_kernel<256>; break;
    default: return cudaErrorInvalidValue;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, tpw * groups_per_block, 0);
}

// Floats of one world's backward workspace for the given sizes (forward part included).
long long backward_ws_floats(int nb, int nv, int nm, int na, int ckpt_every) {
  const WsLayout L = WsLayout::make(nb, nv, nm, na);
  return AdjLayout::make(L.total, nb, nv, na, ckpt_every).total;
}

}  // namespace orchard
