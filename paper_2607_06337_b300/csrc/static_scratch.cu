// ot_step_static_scratch: one step of every world with the per-world temporaries held in a
// fixed array that lives inside this library, so the call needs no scratch area from the
// caller and allocates nothing.
//
// Who needs it: callers that cannot allocate device memory when they step, for example a
// control loop that must not block or fail on an allocation in the middle of a run, or a
// host program that owns a fixed device-memory budget and hands the library only the model
// and state buffers it already holds.
//
// How it works: the rollout kernel runs with its workspace in global memory, pointed at
// g_static_scratch instead of the state's scratch area. In host code the array's name is not
// a device address, so the address is fetched once per device with cudaGetSymbolAddress
// (with that device current) and cached. The queue counters sit in the first 256 bytes of the
// array and are cleared on every call; the rest is fully written before it is read.
//
// Limits: OT_STATIC_SCRATCH_BYTES in total (every GPU that loads the library holds it until
// the process exits). A world whose temporaries do not fit in it, or any other argument a
// launch would reject, is reported before anything is queued (OT_ECAPACITY, OT_EINVAL). A
// block holds at most as many worlds as the array has slots, whatever the class's schedule.
// All calls share the array, so calls that overlap on the GPU (on different streams, or from
// different threads) race with each other: serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/orchard.h"
#include "orchard_dev.h"

namespace {

constexpr size_t kFloats = OT_STATIC_SCRATCH_BYTES / sizeof(float);
constexpr size_t kCounterFloats = 64;  // first 256 bytes: one queue counter per size class
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_static_scratch[kFloats];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array for the current device (looked up once per device).
cudaError_t scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = (float*)g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ot_status ot_step_static_scratch(ot_model* model, ot_state* state, const float* ext_force,
                                            const ot_force_schedule* pulls, int32_t step, double dt, void* stream) {
  if (!model || !state || !(dt > 0)) return OT_EINVAL;
  // validate and shape every class before queuing anything: a rejection leaves no work behind
  int n_classes = 0;
  orchard::StaticShape shapes[kCounterFloats];
  ot_status st = orchard::static_step_plan(model, state, pulls, kFloats - kCounterFloats, (int)kCounterFloats,
                                           &n_classes, shapes);
  if (st != OT_OK) return st;
  float* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return OT_ECUDA;
  int* counters = (int*)base;
  if (cudaMemsetAsync(counters, 0, kCounterFloats * sizeof(float), (cudaStream_t)stream) != cudaSuccess)
    return OT_ECUDA;
  for (int k = 0; k < n_classes; ++k) {
    st = orchard::static_step_class(model, state, k, shapes[k], ext_force, pulls, step, dt, base + kCounterFloats,
                                    counters + k, stream);
    if (st != OT_OK) return st;
  }
  return OT_OK;
}
