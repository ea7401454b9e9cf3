"""Python access to the FP64 CPU oracle (oracle/oracle.cpp) through ctypes.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package; the product path never does. It imports nothing from
the CUDA package; the seeded inputs reach it as plain numpy arrays of a ``Forest``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liboracle.so")
SRC = os.path.join(HERE, "oracle.cpp")

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (in-tree, oracle/_build/liboracle.so)."""
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread", "-o", LIB_PATH, SRC]
        subprocess.run(cmd, check=True)
    return LIB_PATH


class OForest(C.Structure):
    _fields_ = [("n_worlds", C.c_int32),
                ("body_off", _i32p), ("apple_off", _i32p), ("tip_off", _i32p),
                ("parent", _i32p), ("ndof", _i32p),
                ("jpos", _f64p), ("qrel", _f64p), ("com", _f64p), ("mass", _f64p), ("inertia", _f64p),
                ("k", _f64p), ("kd", _f64p), ("armature", _f64p), ("m_max", _f64p),
                ("apple_body", _i32p),
                ("hang_local", _f64p), ("apple_mass", _f64p), ("k_s", _f64p), ("c_s", _f64p),
                ("f_detach", _f64p),
                ("tip_body", _i32p), ("tip_local", _f64p), ("gravity", _f64p)]


class OFlags(C.Structure):
    _fields_ = [("dt", C.c_double), ("alpha_implicit_spring", C.c_int32), ("tether_implicit", C.c_int32),
                ("n_break", C.c_int32), ("n_pull", C.c_int32), ("n_tension", C.c_int32),
                ("gamma_tension", C.c_double), ("clamp_factor", C.c_double), ("dense_limit", C.c_int32),
                ("break_ramp_s", C.c_double), ("break_ramp_factor", C.c_double),
                ("lin_damping", C.c_double), ("ang_damping", C.c_double), ("snapped_lin_damping", C.c_double),
                ("rail_speed", C.c_double), ("rail_fade_speed", C.c_double), ("rail_brake", C.c_double)]


class OState(C.Structure):
    _fields_ = [("q", _f64p), ("qd", _f64p), ("ax", _f64p), ("av", _f64p),
                ("broken", _i32p), ("bcnt", _i32p), ("break_step", _i32p),
                ("detached", _i32p), ("pcnt", _i32p), ("tcnt", _i32p), ("detach_step", _i32p),
                ("status", _i32p)]


class OPulls(C.Structure):
    _fields_ = [("force", _f64p), ("start", _i32p), ("end", _i32p)]


class ORecord(C.Structure):
    _fields_ = [("tips", _f64p), ("q", _f64p), ("near", _i32p), ("near_margin", _f64p),
                ("near_cap", C.c_int32), ("near_count", _i32p), ("near_eps", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_rollout.argtypes = [C.POINTER(OForest), C.POINTER(OFlags), C.POINTER(OState),
                                        C.POINTER(OPulls), C.c_int, C.c_int, C.POINTER(ORecord), C.c_int]
        _lib.oracle_eval.argtypes = [C.POINTER(OForest), C.POINTER(OFlags), C.c_int, _f64p, _f64p, _f64p,
                                     _f64p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        _lib.oracle_solve.argtypes = [C.c_int, _i32p, _f64p, _f64p, C.c_int]
        _lib.oracle_grad.argtypes = [C.POINTER(OForest), C.POINTER(OFlags), C.POINTER(OState), C.POINTER(OPulls),
                                     C.c_int, C.c_int, C.c_int, _f64p, C.c_int, _i32p, _i32p, _f64p, C.c_int,
                                     _f64p, _f64p, C.c_int]
        _lib.oracle_grad_full.argtypes = [C.POINTER(OForest), C.POINTER(OFlags), C.POINTER(OState),
                                          C.POINTER(OPulls), C.c_int, C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p,
                                          _f64p, _f64p, C.c_longlong]
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


class _Keep:
    """Holds contiguous copies alive while a ctypes struct points at them."""

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


def _forest_struct(f, keep: _Keep) -> OForest:
    return OForest(
        f.n_worlds, keep.i32(f.body_off), keep.i32(f.apple_off), keep.i32(f.tip_off),
        keep.i32(f.parent), keep.i32(f.ndof), keep.f64(f.jpos), keep.f64(f.qrel), keep.f64(f.com),
        keep.f64(f.mass), keep.f64(f.inertia), keep.f64(f.k), keep.f64(f.kd), keep.f64(f.armature),
        keep.f64(f.m_max), keep.i32(f.apple_body), keep.f64(f.hang_local),
        keep.f64(f.apple_mass), keep.f64(f.k_s), keep.f64(f.c_s), keep.f64(f.f_detach),
        keep.i32(f.tip_body), keep.f64(f.tip_local), keep.f64(f.gravity))


def _flags_struct(fl, dense_limit: int) -> OFlags:
    return OFlags(fl.dt, fl.alpha_implicit_spring, fl.tether_implicit, fl.n_break, fl.n_pull, fl.n_tension,
                  fl.gamma_tension, fl.clamp_factor, dense_limit, fl.break_ramp_s, fl.break_ramp_factor,
                  getattr(fl, "lin_damping", 0.0), getattr(fl, "ang_damping", 0.0),
                  getattr(fl, "snapped_lin_damping", 0.1), getattr(fl, "rail_speed", 0.0),
                  getattr(fl, "rail_fade_speed", 0.0), getattr(fl, "rail_brake", 0.0))


@dataclass
class OracleState:
    q: np.ndarray
    qd: np.ndarray
    ax: np.ndarray
    av: np.ndarray
    broken: np.ndarray
    bcnt: np.ndarray
    break_step: np.ndarray
    detached: np.ndarray
    pcnt: np.ndarray
    tcnt: np.ndarray
    detach_step: np.ndarray
    status: np.ndarray

    @staticmethod
    def initial(f) -> "OracleState":
        nb, na = f.n_bodies, f.n_apples
        return OracleState(
            q=np.array(f.q0, np.float64), qd=np.array(f.qd0, np.float64),
            ax=np.array(f.apple_x0, np.float64).reshape(na, 3).copy(),
            av=np.array(f.apple_v0, np.float64).reshape(na, 3).copy(),
            broken=np.zeros(nb, np.int32), bcnt=np.zeros(nb, np.int32), break_step=np.full(nb, -1, np.int32),
            detached=np.zeros(na, np.int32), pcnt=np.zeros(na, np.int32), tcnt=np.zeros(na, np.int32),
            detach_step=np.full(na, -1, np.int32), status=np.zeros(f.n_worlds, np.int32))

    def copy(self) -> "OracleState":
        return OracleState(**{k: v.copy() for k, v in self.__dict__.items()})

    def struct(self) -> OState:
        for k, v in self.__dict__.items():
            assert v.flags["C_CONTIGUOUS"], k
        return OState(_p(self.q, _f64p), _p(self.qd, _f64p), _p(self.ax, _f64p), _p(self.av, _f64p),
                      _p(self.broken, _i32p), _p(self.bcnt, _i32p), _p(self.break_step, _i32p),
                      _p(self.detached, _i32p), _p(self.pcnt, _i32p), _p(self.tcnt, _i32p),
                      _p(self.detach_step, _i32p), _p(self.status, _i32p))


def _pulls_struct(f, keep: _Keep) -> OPulls:
    if f.pull_force is None:
        na = f.n_apples
        return OPulls(keep.f64(np.zeros((na, 3))), keep.i32(np.full(na, 1 << 30)), keep.i32(np.full(na, 1 << 30)))
    return OPulls(keep.f64(f.pull_force), keep.i32(f.pull_start), keep.i32(f.pull_end))


def rollout(f, flags, n_steps: int, state: OracleState | None = None, step0: int = 0, record_tips: bool = False,
            record_q: bool = False, near_eps: float = 0.0, near_cap: int = 100000, n_threads: int | None = None,
            dense_limit: int = 256):
    """Run n_steps of every world; returns (final state, dict of records)."""
    st = OracleState.initial(f) if state is None else state.copy()
    keep = _Keep()
    fs = _forest_struct(f, keep)
    fl = _flags_struct(flags, dense_limit)
    pl = _pulls_struct(f, keep)
    tips = np.zeros((n_steps, f.n_tips, 3)) if record_tips else None
    qrec = np.zeros((n_steps, f.n_dofs)) if record_q else None
    near = np.zeros((near_cap, 4), np.int32)
    near_m = np.zeros(near_cap)
    near_n = np.zeros(1, np.int32)
    rec = ORecord(_p(tips, _f64p), _p(qrec, _f64p), _p(near, _i32p), _p(near_m, _f64p), near_cap,
                  _p(near_n, _i32p), near_eps)
    nt = n_threads if n_threads is not None else min(os.cpu_count() or 1, max(1, f.n_worlds))
    s = st.struct()
    lib().oracle_rollout(C.byref(fs), C.byref(fl), C.byref(s), C.byref(pl), step0, n_steps, C.byref(rec), nt)
    n = int(min(near_n[0], near_cap))
    return st, dict(tips=tips, q=qrec, near=near[:n].copy(), near_margin=near_m[:n].copy(),
                    near_overflow=int(near_n[0]) > near_cap)


def evaluate(f, flags, w: int, q, qd, ax=None, av=None, detached=None, fext=None, dense_limit: int = 256):
    """M (dense), bias c, body frames, joint origins and centres of mass of world w at (q, qd)."""
    nb = int(f.body_off[w + 1] - f.body_off[w])
    na = int(f.apple_off[w + 1] - f.apple_off[w])
    nv = int(f.ndof[f.body_off[w]:f.body_off[w + 1]].sum())
    keep = _Keep()
    fs = _forest_struct(f, keep)
    fl = _flags_struct(flags, dense_limit)
    M = np.zeros((nv, nv))
    c = np.zeros(nv)
    R = np.zeros((nb, 3, 3))
    x = np.zeros((nb, 3))
    com = np.zeros((nb, 3))
    ten = np.zeros(na)
    fapp = np.zeros((na, 3))
    q = np.ascontiguousarray(q, np.float64)
    qd = np.ascontiguousarray(qd, np.float64)
    lib().oracle_eval(C.byref(fs), C.byref(fl), w, _p(q, _f64p), _p(qd, _f64p),
                      None if ax is None else keep.f64(ax),
                      None if av is None else keep.f64(av),
                      None if detached is None else keep.i32(detached),
                      None if fext is None else keep.f64(fext),
                      _p(M, _f64p), _p(c, _f64p), _p(R, _f64p), _p(x, _f64p), _p(com, _f64p),
                      _p(ten, _f64p), _p(fapp, _f64p))
    return dict(M=M, c=c, R=R, x=x, com=com, tension=ten, fapp=fapp)


def solve(H, lam, r, mode: int):
    """Solve H x = r densely (mode 0) or by the tree LTDL factorisation (mode 1)."""
    H = np.ascontiguousarray(H, np.float64)
    x = np.array(r, np.float64)
    lam = np.ascontiguousarray(lam, np.int32)
    lib().oracle_solve(len(x), _p(lam, _i32p), _p(H, _f64p), _p(x, _f64p), mode)
    return x


def grad(f, flags, w: int, n_steps: int, target, kinds, idx, steps, mode: int, state: OracleState | None = None,
         step0: int = 0, n_threads: int | None = None, dense_limit: int = 256):
    """Loss gradient of world w by complex step (mode 0), central differences (mode 1), or
    complex step with every operation in single precision (mode 2: the FP32 rounding floor).

    kinds: 0 = k of body idx, 1 = kd of body idx, 2 = q0[idx], 3 = qd0[idx] (world-local).
    target: (n_steps, n_tips_of_world, 3) tip positions.
    """
    st = OracleState.initial(f) if state is None else state.copy()
    keep = _Keep()
    fs = _forest_struct(f, keep)
    fl = _flags_struct(flags, dense_limit)
    pl = _pulls_struct(f, keep)
    s = st.struct()
    kinds = np.ascontiguousarray(kinds, np.int32)
    idx = np.ascontiguousarray(idx, np.int32)
    steps = np.ascontiguousarray(steps, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    g = np.zeros(len(kinds))
    loss = np.zeros(1)
    nt = n_threads if n_threads is not None else (os.cpu_count() or 1)
    lib().oracle_grad(C.byref(fs), C.byref(fl), C.byref(s), C.byref(pl), w, step0, n_steps, _p(target, _f64p),
                      len(kinds), _p(kinds, _i32p), _p(idx, _i32p), _p(steps, _f64p), mode, _p(g, _f64p),
                      _p(loss, _f64p), nt)
    return g, float(loss[0])


def grad_full(f, flags, w: int, n_steps: int, target, state: OracleState | None = None, step0: int = 0,
              max_nodes: int = 30_000_000, dense_limit: int = 256):
    """Full loss gradient of world w by the oracle's reverse-mode scalar (its own FP64 adjoint).

    Returns dict(dk, dkd [nb], dq0, dqd0 [nv] world-local, loss, nodes). The tape holds every
    scalar operation of the rollout (about 32 bytes each), so this is for small worlds and
    short rollouts; raises MemoryError past max_nodes.
    """
    st = OracleState.initial(f) if state is None else state.copy()
    keep = _Keep()
    fs = _forest_struct(f, keep)
    fl = _flags_struct(flags, dense_limit)
    pl = _pulls_struct(f, keep)
    s = st.struct()
    b0, b1 = f.body_off[w], f.body_off[w + 1]
    nb = int(b1 - b0)
    nv = int(f.dof_off[w + 1] - f.dof_off[w])
    target = np.ascontiguousarray(target, np.float64)
    out = {k: np.zeros(n) for k, n in (("dk", nb), ("dkd", nb), ("dq0", nv), ("dqd0", nv))}
    loss = np.zeros(1)
    r = lib().oracle_grad_full(C.byref(fs), C.byref(fl), C.byref(s), C.byref(pl), w, step0, n_steps,
                               _p(target, _f64p), _p(out["dk"], _f64p), _p(out["dkd"], _f64p),
                               _p(out["dq0"], _f64p), _p(out["dqd0"], _f64p), _p(loss, _f64p), int(max_nodes))
    if r < 0:
        raise MemoryError(f"reverse-mode tape of world {w} exceeds {max_nodes} nodes")
    out["loss"] = float(loss[0])
    out["nodes"] = int(r)
    return out
