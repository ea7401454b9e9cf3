"""Thin Python binding of liborchard (include/orchard.h): argument marshalling only.

Every step of the path runs in the CUDA library. Torch supplies the device buffers (the
library never allocates device memory) and the CUDA stream. The functions keep the C names
(tree_model_upload, world_state_alloc, step, rollout, rollout_backward, ...). Importing this
module loads the in-tree ``_lib/liborchard.so`` and raises if it is missing: there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liborchard.so")
# ORCHARD_LIB_VARIANT=phase loads the profiling build with the step's phase clocks instead
if os.environ.get("ORCHARD_LIB_VARIANT", "") == "phase":
    LIB_PATH = os.path.join(HERE, "_lib", "liborchard_phase.so")

OT_OK = 0
OT_EINVAL = -1
OT_ETOPO = -2
OT_ENONFINITE = -3
OT_ECAPACITY = -4
OT_ECUDA = -5
OT_ESTATE = -6
OT_WORLD_NONFINITE = 1

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)
_f32p = C.POINTER(C.c_float)


class OrchardError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().ot_status_string(status).decode()
        extra = f" (cuda error {lib().ot_last_cuda_error()})" if status == OT_ECUDA else ""
        super().__init__(f"{where}: {msg} [{status}]{extra}")
        self.status = status


class TreeDesc(C.Structure):
    _fields_ = [("n_worlds", C.c_int32),
                ("body_off", _i32p), ("apple_off", _i32p), ("tip_off", _i32p),
                ("parent", _i32p), ("ndof", _i32p),
                ("jpos", _f64p), ("qrel", _f64p), ("com", _f64p), ("mass", _f64p), ("inertia", _f64p),
                ("k", _f64p), ("kd", _f64p), ("armature", _f64p), ("m_max", _f64p),
                ("apple_body", _i32p), ("hang_local", _f64p), ("apple_mass", _f64p), ("k_s", _f64p),
                ("c_s", _f64p), ("f_detach", _f64p),
                ("tip_body", _i32p), ("tip_local", _f64p), ("gravity", _f64p), ("diam", _f64p),
                ("length", _f64p), ("rho", _f64p), ("youngs", _f64p), ("sigma_r", _f64p)]


class ModelFlags(C.Structure):
    _fields_ = [("alpha_implicit_spring", C.c_int32), ("tether_implicit", C.c_int32),
                ("n_break", C.c_int32), ("n_pull", C.c_int32), ("n_tension", C.c_int32),
                ("gamma_tension", C.c_double), ("clamp_factor", C.c_double),
                ("break_ramp_s", C.c_double), ("break_ramp_factor", C.c_double),
                ("fp64_twig_diam", C.c_double), ("lin_damping", C.c_double), ("ang_damping", C.c_double),
                ("snapped_lin_damping", C.c_double), ("rail_speed", C.c_double), ("rail_fade_speed", C.c_double),
                ("rail_brake", C.c_double)]


class Schedule(C.Structure):
    _fields_ = [("threads_per_world", C.c_int32), ("worlds_per_block", C.c_int32), ("blocks", C.c_int32),
                ("global_workspace", C.c_int32), ("stage", C.c_int32)]


class StateInit(C.Structure):
    _fields_ = [("q", C.c_void_p), ("qd", C.c_void_p), ("apple_x", C.c_void_p), ("apple_v", C.c_void_p),
                ("on_device", C.c_int32)]


class StateView(C.Structure):
    _fields_ = [("q", C.c_void_p), ("qd", C.c_void_p), ("apple_x", C.c_void_p), ("apple_v", C.c_void_p),
                ("broken", C.c_void_p), ("break_step", C.c_void_p), ("detached", C.c_void_p),
                ("detach_step", C.c_void_p), ("status", C.c_void_p)]


class ForceSchedule(C.Structure):
    _fields_ = [("force", C.c_void_p), ("start", C.c_void_p), ("end", C.c_void_p)]


class Record(C.Structure):
    _fields_ = [("tips", C.c_void_p), ("ckpt", C.c_void_p), ("ckpt_bytes", C.c_size_t), ("ckpt_every", C.c_int32),
                ("tape", C.c_void_p), ("tape_bytes", C.c_size_t), ("tape_steps", C.c_int32)]


class Grads(C.Structure):
    _fields_ = [("dk", C.c_void_p), ("dkd", C.c_void_p), ("dq0", C.c_void_p), ("dqd0", C.c_void_p)]


# function name -> (restype, argtypes): one entry per declaration of include/orchard.h
_SIGS = {
    "ot_model_bytes": (C.c_int, [C.POINTER(TreeDesc), C.POINTER(C.c_size_t)]),
    "ot_tree_model_upload": (C.c_int, [C.POINTER(TreeDesc), C.POINTER(ModelFlags), C.c_void_p, C.c_size_t,
                                       C.c_void_p, C.POINTER(C.c_void_p)]),
    "ot_model_release": (None, [C.c_void_p]),
    "ot_model_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "ot_model_set_gains": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ot_model_randomize": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ot_state_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "ot_world_state_alloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]),
    "ot_state_release": (None, [C.c_void_p]),
    "ot_state_set": (C.c_int, [C.c_void_p, C.POINTER(StateInit), C.c_void_p]),
    "ot_state_get_view": (C.c_int, [C.c_void_p, C.POINTER(StateView)]),
    "ot_world_status": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ot_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(ForceSchedule), C.c_int32, C.c_double,
                          C.c_void_p]),
    "ot_ckpt_bytes": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    "ot_tape_bytes": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_size_t)]),
    "ot_rollout": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.POINTER(ForceSchedule),
                             C.POINTER(Record), C.c_void_p]),
    "ot_rollout_plain": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_double,
                                   C.POINTER(ForceSchedule), C.c_void_p]),
    "ot_backward_workspace_bytes": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_size_t)]),
    "ot_rollout_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_double,
                                      C.POINTER(ForceSchedule), C.POINTER(Record), C.c_void_p, C.POINTER(Grads),
                                      C.c_void_p, C.c_size_t, C.c_void_p]),
    "ot_autotune_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_double,
                                       C.POINTER(ForceSchedule), C.POINTER(Record), C.c_void_p, C.POINTER(Grads),
                                       C.c_void_p, C.c_size_t, C.c_void_p]),
    "ot_get_backward_schedule": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "ot_set_backward_schedule": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "ot_get_schedule": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Schedule)]),
    "ot_set_schedule": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Schedule)]),
    "ot_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p]),
    "ot_step_static_scratch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(ForceSchedule), C.c_int32,
                                         C.c_double, C.c_void_p]),
    "ot_status_string": (C.c_char_p, [C.c_int]),
    "ot_last_cuda_error": (C.c_int32, []),
    "ot_launch_count": (C.c_int64, [C.c_int32]),
    "ot_phase_clocks": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.c_int32, C.c_int32]),
    "ot_class_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
}

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run paper_2607_06337_b300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != OT_OK:
        raise OrchardError(status, where)


def _stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class _Keep:
    def __init__(self):
        self.refs = []

    def f64(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.refs.append(a)
        return a.ctypes.data_as(_f64p)

    def i32(self, a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        self.refs.append(a)
        return a.ctypes.data_as(_i32p)


def make_desc(forest, keep: _Keep) -> TreeDesc:
    f = forest
    return TreeDesc(
        f.n_worlds, keep.i32(f.body_off), keep.i32(f.apple_off), keep.i32(f.tip_off),
        keep.i32(f.parent), keep.i32(f.ndof), keep.f64(f.jpos), keep.f64(f.qrel), keep.f64(f.com),
        keep.f64(f.mass), keep.f64(f.inertia), keep.f64(f.k), keep.f64(f.kd), keep.f64(f.armature),
        keep.f64(f.m_max), keep.i32(f.apple_body), keep.f64(f.hang_local), keep.f64(f.apple_mass),
        keep.f64(f.k_s), keep.f64(f.c_s), keep.f64(f.f_detach), keep.i32(f.tip_body), keep.f64(f.tip_local),
        keep.f64(f.gravity), keep.f64(f.diam) if getattr(f, "diam", None) is not None else None,
        *(keep.f64(getattr(f, key)) if getattr(f, key, None) is not None else None
          for key in ("length", "rho", "youngs", "sigma_r")))


def make_flags(flags) -> ModelFlags:
    return ModelFlags(int(flags.alpha_implicit_spring), int(flags.tether_implicit), int(flags.n_break),
                      int(flags.n_pull), int(flags.n_tension), float(flags.gamma_tension), float(flags.clamp_factor),
                      float(flags.break_ramp_s), float(flags.break_ramp_factor),
                      float(getattr(flags, "fp64_twig_diam", 0.0)), float(getattr(flags, "lin_damping", 0.0)),
                      float(getattr(flags, "ang_damping", 0.0)), float(getattr(flags, "snapped_lin_damping", 0.1)),
                      float(getattr(flags, "rail_speed", 0.0)), float(getattr(flags, "rail_fade_speed", 0.0)),
                      float(getattr(flags, "rail_brake", 0.0)))


# ------------------------------------------------------------------------------------------
# C-named entry points
# ------------------------------------------------------------------------------------------
def model_bytes(forest) -> int:
    keep = _Keep()
    d = make_desc(forest, keep)
    n = C.c_size_t(0)
    _check(lib().ot_model_bytes(C.byref(d), C.byref(n)), "ot_model_bytes")
    return n.value


def tree_model_upload(forest, flags, dev_buf, stream=None):
    """Upload a forest into the torch uint8 tensor dev_buf; returns the model handle."""
    keep = _Keep()
    d = make_desc(forest, keep)
    fl = make_flags(flags)
    h = C.c_void_p()
    _check(lib().ot_tree_model_upload(C.byref(d), C.byref(fl), _ptr(dev_buf), dev_buf.numel(),
                                      _stream_handle(stream), C.byref(h)), "ot_tree_model_upload")
    return h


def model_set_gains(model, k=None, kd=None, stream=None):
    """Write per-body k and kd (float32 device tensors [nb], either may be None) into the model."""
    for t in (k, kd):
        if t is not None and (t.dtype.itemsize != 4 or not t.is_cuda or not t.is_contiguous()):
            raise ValueError("gains must be contiguous float32 CUDA tensors")
    _check(lib().ot_model_set_gains(model, _ptr(k), _ptr(kd), _stream_handle(stream)), "ot_model_set_gains")


def model_randomize(model, factors, capsule_links=False, stream=None):
    """Domain randomisation on the device: factors, a float32 CUDA tensor [worlds, 6] of
    (s_len, s_diam, s_rho, s_E, s_sigma, c_d) per world (see include/orchard.h)."""
    if factors.dtype.itemsize != 4 or not factors.is_cuda or not factors.is_contiguous() or factors.dim() != 2 \
            or factors.shape[1] != 6:
        raise ValueError("factors must be a contiguous float32 CUDA tensor [worlds, 6]")
    _check(lib().ot_model_randomize(model, _ptr(factors), int(bool(capsule_links)), _stream_handle(stream)),
           "ot_model_randomize")


def state_bytes(model) -> int:
    n = C.c_size_t(0)
    _check(lib().ot_state_bytes(model, C.byref(n)), "ot_state_bytes")
    return n.value


def world_state_alloc(model, dev_buf):
    h = C.c_void_p()
    _check(lib().ot_world_state_alloc(model, _ptr(dev_buf), dev_buf.numel(), C.byref(h)), "ot_world_state_alloc")
    return h


def step(model, state, ext_force=None, pulls=None, step_index=0, dt=2e-3, stream=None):
    fs = pulls if pulls is not None else ForceSchedule(None, None, None)
    _check(lib().ot_step(model, state, _ptr(ext_force), C.byref(fs), int(step_index), float(dt),
                         _stream_handle(stream)), "ot_step")


def rollout(model, state, n_steps, step0=0, dt=2e-3, pulls=None, record=None, stream=None):
    fs = pulls if pulls is not None else ForceSchedule(None, None, None)
    rec = record if record is not None else Record(None, None, 0, 0)
    _check(lib().ot_rollout(model, state, int(n_steps), int(step0), float(dt), C.byref(fs), C.byref(rec),
                            _stream_handle(stream)), "ot_rollout")


def rollout_plain(model, state, n_steps, step0=0, dt=2e-3, pulls=None, stream=None):
    fs = pulls if pulls is not None else ForceSchedule(None, None, None)
    _check(lib().ot_rollout_plain(model, state, int(n_steps), int(step0), float(dt), C.byref(fs),
                                  _stream_handle(stream)), "ot_rollout_plain")


def backward_workspace_bytes(model, ckpt_every) -> int:
    n = C.c_size_t(0)
    _check(lib().ot_backward_workspace_bytes(model, int(ckpt_every), C.byref(n)), "ot_backward_workspace_bytes")
    return n.value


def rollout_backward(model, state, n_steps, step0, dt, pulls, record, dL_dtips, grads, workspace, stream=None):
    fs = pulls if pulls is not None else ForceSchedule(None, None, None)
    _check(lib().ot_rollout_backward(model, state, int(n_steps), int(step0), float(dt), C.byref(fs),
                                     C.byref(record), _ptr(dL_dtips), C.byref(grads), _ptr(workspace),
                                     workspace.numel() * workspace.element_size(), _stream_handle(stream)),
           "ot_rollout_backward")


def autotune_backward(model, state, n_steps, step0, dt, pulls, record, dL_dtips, grads, workspace, stream=None):
    fs = pulls if pulls is not None else ForceSchedule(None, None, None)
    _check(lib().ot_autotune_backward(model, state, int(n_steps), int(step0), float(dt), C.byref(fs),
                                      C.byref(record), _ptr(dL_dtips), C.byref(grads), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), _stream_handle(stream)),
           "ot_autotune_backward")


def get_backward_schedule(model, k) -> int:
    t = C.c_int32(0)
    _check(lib().ot_get_backward_schedule(model, int(k), C.byref(t)), "ot_get_backward_schedule")
    return int(t.value)


def set_backward_schedule(model, k, threads_per_world):
    _check(lib().ot_set_backward_schedule(model, int(k), int(threads_per_world)), "ot_set_backward_schedule")


def ckpt_bytes(model, n_steps, ckpt_every) -> int:
    n = C.c_size_t(0)
    _check(lib().ot_ckpt_bytes(model, int(n_steps), int(ckpt_every), C.byref(n)), "ot_ckpt_bytes")
    return n.value


def tape_bytes(model, n_steps) -> int:
    n = C.c_size_t(0)
    _check(lib().ot_tape_bytes(model, int(n_steps), C.byref(n)), "ot_tape_bytes")
    return n.value


def get_schedule(model, k) -> Schedule:
    s = Schedule()
    _check(lib().ot_get_schedule(model, int(k), C.byref(s)), "ot_get_schedule")
    return s


def set_schedule(model, k, sched: Schedule):
    _check(lib().ot_set_schedule(model, int(k), C.byref(sched)), "ot_set_schedule")


CLASS_INFO = ("worlds", "max_bodies", "workspace_bytes", "stage_mask", "stage_bytes", "smem_per_block",
              "blocks_per_sm", "blocks")


def class_info(model, k) -> dict:
    """What size class k resolves to under its schedule (ot_class_info)."""
    out = (C.c_int64 * 8)()
    _check(lib().ot_class_info(model, int(k), out), "ot_class_info")
    return dict(zip(CLASS_INFO, (int(x) for x in out)))


def autotune(model, state, n_steps, dt=2e-3, stream=None):
    _check(lib().ot_autotune(model, state, int(n_steps), float(dt), _stream_handle(stream)), "ot_autotune")


def launch_count(reset=False) -> int:
    return int(lib().ot_launch_count(1 if reset else 0))


PHASES = ("kinematics", "forces", "tips", "bias_sweep", "mass_matrix", "ldlt", "update_sweep", "apples", "other")
BACK_PHASES = ("apples_hang", "solve", "lsweep_springs_tape", "seeds", "chain", "restore", "replay", "final",
               "other")
BACK_ROW = 32


def phase_clocks(model, n_classes, reset=True, backward=False):
    """Per size class, SM cycles per world-step of each phase (the profiling build only):
    a list of dicts {phase: cycles, "world_steps": n}; backward=True: the backward passes'."""
    n = len(PHASES) + 1
    rows = BACK_ROW + n_classes if backward else n_classes
    buf = (C.c_uint64 * (n * rows))()
    _check(lib().ot_phase_clocks(model, buf, int(rows), 1 if reset else 0), "ot_phase_clocks")
    names = BACK_PHASES if backward else PHASES
    out = []
    for k in range(BACK_ROW if backward else 0, rows):
        row = list(buf[k * n:(k + 1) * n])
        steps = row[-1]
        d = {p: (row[i] / steps if steps else 0.0) for i, p in enumerate(names)}
        d["world_steps"] = steps
        out.append(d)
    return out


# ------------------------------------------------------------------------------------------
# Convenience wrapper owning the torch buffers
# ------------------------------------------------------------------------------------------
@dataclass
class Counts:
    worlds: int
    bodies: int
    dofs: int
    apples: int
    tips: int
    classes: int


class Simulator:
    """A forest uploaded to the GPU with its state; torch tensors own all device memory."""

    def __init__(self, forest, flags, device="cuda", stream=None):
        import torch
        self.forest = forest
        self.flags = flags
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.model_buf = torch.empty(model_bytes(forest), dtype=torch.uint8, device=self.device)
        self.model = tree_model_upload(forest, flags, self.model_buf, stream)
        cnt = (C.c_int64 * 6)()
        _check(lib().ot_model_counts(self.model, cnt), "ot_model_counts")
        self.counts = Counts(*[int(x) for x in cnt])
        self.state_buf = torch.empty(state_bytes(self.model), dtype=torch.uint8, device=self.device)
        self.state = world_state_alloc(self.model, self.state_buf)
        v = StateView()
        _check(lib().ot_state_get_view(self.state, C.byref(v)), "ot_state_get_view")
        base = self.state_buf.data_ptr()
        c = self.counts

        def sl(ptr, n, dtype):
            off = ptr - base
            nbytes = n * 4
            return self.state_buf[off:off + nbytes].view(dtype)

        self.q = sl(v.q, c.dofs, torch.float32)
        self.qd = sl(v.qd, c.dofs, torch.float32)
        self.apple_x = sl(v.apple_x, 3 * c.apples, torch.float32).view(c.apples, 3)
        self.apple_v = sl(v.apple_v, 3 * c.apples, torch.float32).view(c.apples, 3)
        self.broken = sl(v.broken, c.bodies, torch.int32)
        self.break_step = sl(v.break_step, c.bodies, torch.int32)
        self.detached = sl(v.detached, c.apples, torch.int32)
        self.detach_step = sl(v.detach_step, c.apples, torch.int32)
        self.status = sl(v.status, c.worlds, torch.int32)
        self._pull_tensors = None
        self.pulls = ForceSchedule(None, None, None)
        if forest.pull_force is not None and forest.n_apples > 0 and (forest.pull_start < (1 << 29)).any():
            self.set_pulls(forest.pull_force, forest.pull_start, forest.pull_end)

    def set_pulls(self, force, start, end):
        import torch
        f = torch.as_tensor(np.asarray(force, np.float32).reshape(-1, 3), device=self.device).contiguous()
        s = torch.as_tensor(np.asarray(start, np.int32), device=self.device).contiguous()
        e = torch.as_tensor(np.asarray(end, np.int32), device=self.device).contiguous()
        self._pull_tensors = (f, s, e)
        self.pulls = ForceSchedule(f.data_ptr(), s.data_ptr(), e.data_ptr())

    def reset(self, q=None, qd=None, apple_x=None, apple_v=None, stream=None):
        """Initial state from host arrays (defaults: the forest's q0, qd0, apple_x0, apple_v0)."""
        f = self.forest
        arrs = [np.ascontiguousarray(a, np.float32) for a in (
            f.q0 if q is None else q, f.qd0 if qd is None else qd,
            f.apple_x0 if apple_x is None else apple_x, f.apple_v0 if apple_v is None else apple_v)]
        ptrs = [a.ctypes.data if a.size else None for a in arrs]
        init = StateInit(ptrs[0], ptrs[1], ptrs[2], ptrs[3], 0)
        _check(lib().ot_state_set(self.state, C.byref(init), _stream_handle(stream)), "ot_state_set")

    def reset_from_device(self, q, qd, apple_x, apple_v, stream=None):
        init = StateInit(q.data_ptr(), qd.data_ptr(), apple_x.data_ptr() if apple_x.numel() else None,
                         apple_v.data_ptr() if apple_v.numel() else None, 1)
        _check(lib().ot_state_set(self.state, C.byref(init), _stream_handle(stream)), "ot_state_set")

    def rollout(self, n_steps, step0=0, dt=None, record=None, stream=None):
        rollout(self.model, self.state, n_steps, step0, self.flags.dt if dt is None else dt, self.pulls, record,
                stream)

    def rollout_plain(self, n_steps, step0=0, dt=None, stream=None):
        rollout_plain(self.model, self.state, n_steps, step0, self.flags.dt if dt is None else dt, self.pulls,
                      stream)

    def step(self, step_index=0, ext_force=None, dt=None, stream=None):
        step(self.model, self.state, ext_force, self.pulls, step_index, self.flags.dt if dt is None else dt,
             stream)

    def set_gains(self, k=None, kd=None, stream=None):
        """Per-body joint stiffness and damping from float32 device tensors [bodies]."""
        model_set_gains(self.model, k, kd, stream)

    def randomize(self, factors, capsule_links=None, stream=None):
        """Per-world domain randomisation on the device (factors [worlds, 6], float32 CUDA)."""
        if capsule_links is None:
            capsule_links = bool(self.forest.meta.get("capsule", False))
        model_randomize(self.model, factors, capsule_links, stream)

    def record_buffers(self, n_steps, ckpt_every, tips=True, tape_steps=0):
        """Device buffers for a recorded rollout: tips [n_steps, n_tips, 3], and checkpoints every
        ``ckpt_every`` steps, or with ``ckpt_every`` 0 the adjoint's full tape (ot_tape_bytes:
        the backward then replays no step). With ``ckpt_every`` > 0 and 0 < ``tape_steps`` <
        ``n_steps``, both: a tape of the final ``tape_steps`` steps and checkpoints for the
        earlier ones. Returns (tips, buffer, record); buffer is (checkpoints, tape) for both."""
        import torch
        t = torch.empty((n_steps, self.counts.tips, 3), dtype=torch.float32, device=self.device) if tips else None
        tp = None if t is None else t.data_ptr()
        if ckpt_every == 0:
            nb = tape_bytes(self.model, n_steps)
            buf = torch.empty(nb, dtype=torch.uint8, device=self.device)
            return t, buf, Record(tp, None, 0, 0, buf.data_ptr(), nb, 0)
        nb = ckpt_bytes(self.model, n_steps, ckpt_every)
        buf = torch.empty(nb, dtype=torch.uint8, device=self.device)
        if 0 < tape_steps < n_steps:
            nt = tape_bytes(self.model, tape_steps)
            tbuf = torch.empty(nt, dtype=torch.uint8, device=self.device)
            return t, (buf, tbuf), Record(tp, buf.data_ptr(), nb, ckpt_every, tbuf.data_ptr(), nt, tape_steps)
        return t, buf, Record(tp, buf.data_ptr(), nb, ckpt_every, None, 0, 0)

    def backward(self, n_steps, record, dL_dtips, step0=0, dt=None, grads=None, workspace=None, stream=None):
        """Adjoint of a recorded rollout. Returns (dk, dkd, dq0, dqd0) as float32 device tensors.

        dk and dkd are accumulated into when given in ``grads``; fresh zeroed ones otherwise."""
        import torch
        c = self.counts
        if grads is None:
            grads = tuple(torch.zeros(n, dtype=torch.float32, device=self.device)
                          for n in (c.bodies, c.bodies, c.dofs, c.dofs))
        if workspace is None:
            workspace = torch.empty(backward_workspace_bytes(self.model, record.ckpt_every), dtype=torch.uint8,
                                    device=self.device)
        g = Grads(*[t.data_ptr() if t.numel() else None for t in grads])
        rollout_backward(self.model, self.state, n_steps, step0, self.flags.dt if dt is None else dt, self.pulls,
                         record, dL_dtips.contiguous(), g, workspace, stream)
        return grads

    def schedules(self):
        return [get_schedule(self.model, k) for k in range(self.counts.classes)]

    def backward_schedules(self):
        """The backward's threads per world of each size class."""
        return [get_backward_schedule(self.model, k) for k in range(self.counts.classes)]

    def autotune_backward(self, n_steps, record, dL_dtips, step0=0, dt=None, workspace=None, stream=None):
        """Pick every class's fastest backward threads per world on a recorded rollout (the
        gradients it produces meanwhile are discarded)."""
        import torch
        c = self.counts
        grads = tuple(torch.zeros(n, dtype=torch.float32, device=self.device)
                      for n in (c.bodies, c.bodies, c.dofs, c.dofs))
        if workspace is None:
            workspace = torch.empty(backward_workspace_bytes(self.model, record.ckpt_every), dtype=torch.uint8,
                                    device=self.device)
        g = Grads(*[t.data_ptr() if t.numel() else None for t in grads])
        autotune_backward(self.model, self.state, n_steps, step0, self.flags.dt if dt is None else dt, self.pulls,
                          record, dL_dtips.contiguous(), g, workspace, stream)

    def class_infos(self):
        """Per size class: its schedule and what it resolves to (class_info)."""
        out = []
        for k, sc in enumerate(self.schedules()):
            d = dict(threads_per_world=sc.threads_per_world, worlds_per_block=sc.worlds_per_block,
                     global_workspace=sc.global_workspace, stage=sc.stage)
            d.update(class_info(self.model, k))
            out.append(d)
        return out

    def autotune(self, n_steps=20, dt=None, stream=None):
        """Pick every class's fastest schedule, every candidate timed from the current state
        (ot_autotune restores it); then reset to the forest's initial state."""
        autotune(self.model, self.state, n_steps, self.flags.dt if dt is None else dt, stream)
        self.reset(stream=stream)

    def close(self):
        if getattr(self, "state", None):
            lib().ot_state_release(self.state)
            self.state = None
        if getattr(self, "model", None):
            lib().ot_model_release(self.model)
            self.model = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
