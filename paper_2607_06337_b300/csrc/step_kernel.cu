// Batched compliant-tree forward rollout kernel for sm_103a (the per-world step is in
// step_device.cuh): a persistent grid whose thread groups pop worlds from a cost-sorted queue
// and run all their steps.
#include "step_device.cuh"

namespace orchard {
namespace {

// ST: the instantiation that reads the model records a class stages in shared memory (the
// other one reads them from the model in global memory and holds no pointers for them).
// LN: the lean placement (WsLayout::make_lean), instantiated for 128-512 threads per world.
template <int TPW, bool ST, bool LN>
__global__ void __launch_bounds__(512) rollout_kernel(DevModel m, DevState s, StepArgs a) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int frozen[16];
  Group<TPW> g;
  g.lane = threadIdx.x % TPW;
  g.id = threadIdx.x / TPW;
  g.flag = &frozen[g.id];
  const int groups = blockDim.x / TPW;
  float* ws = a.global_ws ? s.scratch + (long long)(blockIdx.x * groups + g.id) * a.ws_floats
                          : smem + (long long)g.id * (a.ws_floats + a.stage_floats);
  // the lean placement's global slot of this group (apple records, snapped flags)
  float* lslot = LN ? s.scratch + (long long)(blockIdx.x * groups + g.id) * a.lean_floats : nullptr;
  if (a.single_world >= 0) {
    run_world<TPW, ST>(m, s, a, a.single_world, ws, lslot, g);
    return;
  }
  __shared__ int next[16];
  for (;;) {
    int qi;
    if (a.q_counter) {
      if (g.lane == 0) next[g.id] = atomicAdd(a.q_counter, 1);
      g.sync();
      qi = next[g.id];
      g.sync();
    } else {
      qi = blockIdx.x * groups + g.id;
    }
    if (qi >= a.q_end - a.q_begin) break;
    run_world<TPW, ST>(m, s, a, m.queue[a.q_begin + qi], ws, lslot, g);
    if (!a.q_counter) break;
  }
}

#ifdef ORCHARD_PHASE_CLOCKS
__device__ unsigned long long g_phase_clk[kPhaseClasses * kPhaseSlots];
#endif

}  // namespace

unsigned long long* phase_clock_buffer() {
#ifdef ORCHARD_PHASE_CLOCKS
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_phase_clk) != cudaSuccess) return nullptr;
  return (unsigned long long*)p;
#else
  return nullptr;
#endif
}

template <bool ST, bool LN>
const void* rollout_fn(int tpw) {
  switch (tpw) {
    case 32: return LN ? nullptr : (const void*)rollout_kernel<32, ST, false>;
    case 64: return LN ? nullptr : (const void*)rollout_kernel<64, ST, false>;
    case 128: return (const void*)rollout_kernel<128, ST, LN>;
    case 256: return (const void*)rollout_kernel<256, ST, LN>;
    case 512: return (const void*)rollout_kernel<512, ST, LN>;
    default: return nullptr;
  }
}

template <bool ST, bool LN>
void launch_rollout_t(int tpw, int threads, int blocks, size_t smem_bytes, cudaStream_t st, const DevModel& m,
                      const DevState& s, const StepArgs& a) {
  switch (tpw) {
    case 32: if (!LN) rollout_kernel<32, ST, false><<<blocks, threads, smem_bytes, st>>>(m, s, a); break;
    case 64: if (!LN) rollout_kernel<64, ST, false><<<blocks, threads, smem_bytes, st>>>(m, s, a); break;
    case 128: rollout_kernel<128, ST, LN><<<blocks, threads, smem_bytes, st>>>(m, s, a); break;
    case 256: rollout_kernel<256, ST, LN><<<blocks, threads, smem_bytes, st>>>(m, s, a); break;
    case 512: rollout_kernel<512, ST, LN><<<blocks, threads, smem_bytes, st>>>(m, s, a); break;
    default: break;
  }
}

void launch_rollout(int tpw, int groups_per_block, int blocks, size_t smem_bytes, cudaStream_t st,
                    const DevModel& m, const DevState& s, const StepArgs& a) {
  const int threads = tpw * groups_per_block;
  // the staged instantiation keeps the world's records and their table after its workspace
  const bool staged = a.stage_mask && !a.global_ws;
  if (a.lean) {
    if (staged) launch_rollout_t<true, true>(tpw, threads, blocks, smem_bytes, st, m, s, a);
    else launch_rollout_t<false, true>(tpw, threads, blocks, smem_bytes, st, m, s, a);
  } else {
    if (staged) launch_rollout_t<true, false>(tpw, threads, blocks, smem_bytes, st, m, s, a);
    else launch_rollout_t<false, false>(tpw, threads, blocks, smem_bytes, st, m, s, a);
  }
}

cudaError_t kernel_attributes(int tpw, bool staged, bool lean, int groups_per_block, size_t smem_bytes,
                              int* blocks_per_sm) {
  const void* fn = lean ? (staged ? rollout_fn<true, true>(tpw) : rollout_fn<false, true>(tpw))
                        : (staged ? rollout_fn<true, false>(tpw) : rollout_fn<false, false>(tpw));
  if (!fn) return cudaErrorInvalidValue;
  if (smem_bytes > kSmemLimitBytes) return cudaErrorInvalidValue;
  // the attribute belongs to the instantiation, shared by every class using it: always the limit
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimitBytes);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, tpw * groups_per_block, smem_bytes);
}

}  // namespace orchard
