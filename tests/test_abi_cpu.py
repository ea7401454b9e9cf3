"""The C-ABI library on the CPU: it loads, exports every declared symbol, and validates
descriptors (host-only calls; no compute without a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2607_06337_b300 import build as Bld
from paper_2607_06337_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def orch():
    Bld.build()
    from paper_2607_06337_b300 import orchard
    orchard.lib()
    return orchard


def declared_functions():
    text = open(os.path.join(ROOT, "include", "orchard.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ot_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(orch):
    names = declared_functions()
    assert len(names) >= 20
    L = C.CDLL(orch.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    # and the binding declares a signature for each of them
    assert set(names) == set(orch._SIGS)


def test_status_strings(orch):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert orch.lib().ot_status_string(code)


def test_model_bytes_of_a_generated_forest(orch):
    f = I.make_forest(I.PLAIN, worlds=[0, 1])
    n = orch.model_bytes(f)
    assert n > 0 and n % 256 == 0


def _status_of(orch, f):
    keep = orch._Keep()
    d = orch.make_desc(f, keep)
    n = C.c_size_t(0)
    return orch.lib().ot_model_bytes(C.byref(d), C.byref(n))


def test_validation_rejects_bad_descriptors(orch):
    good = I.make_forest(I.PLAIN, worlds=[0])
    assert _status_of(orch, good) == orch.OT_OK
    # not breadth-first: swap two parents so the parent array decreases
    f = good.subset([0])
    f.parent = f.parent.copy()
    i = int(np.nonzero(np.diff(f.parent[1:]) > 0)[0][0]) + 1
    f.parent[i], f.parent[i + 1] = f.parent[i + 1], f.parent[i]
    assert _status_of(orch, f) == orch.OT_ETOPO
    # parent out of range
    f = good.subset([0])
    f.parent = f.parent.copy()
    f.parent[5] = 40
    assert _status_of(orch, f) == orch.OT_ETOPO
    # a second root
    f = good.subset([0])
    f.parent = f.parent.copy()
    f.parent[0] = 3
    assert _status_of(orch, f) == orch.OT_ETOPO
    # ndof outside {0, 1, 2}
    f = good.subset([0])
    f.ndof = f.ndof.copy()
    f.ndof[4] = 3
    assert _status_of(orch, f) == orch.OT_ETOPO
    # apples not sorted by body
    f = good.subset([0])
    f.apple_body = f.apple_body[::-1].copy()
    assert _status_of(orch, f) == orch.OT_ETOPO
    # non-finite and non-positive values
    for name, val in (("mass", np.nan), ("k", np.inf), ("mass", 0.0), ("apple_mass", -1.0)):
        f = good.subset([0])
        a = getattr(f, name).copy()
        a[1] = val
        setattr(f, name, a)
        assert _status_of(orch, f) == orch.OT_ENONFINITE, name
    # too many DOFs in one world (more than 32767)
    n = 16400
    bodies = [dict(parent=max(i - 1, -1) if i < 2 else (i - 1) // 2, ndof=2, mass=1.0,
                   inertia=(1.0, 1.0, 1.0)) for i in range(n)]
    big = I.from_bodies(bodies)
    assert _status_of(orch, big) == orch.OT_ECAPACITY


def test_upload_rejects_bad_arguments_without_touching_the_device(orch):
    f = I.make_forest(I.PLAIN, worlds=[0])
    keep = orch._Keep()
    d = orch.make_desc(f, keep)
    fl = orch.make_flags(I.Flags())
    h = C.c_void_p()
    # null device buffer
    assert orch.lib().ot_tree_model_upload(C.byref(d), C.byref(fl), None, 0, None, C.byref(h)) == orch.OT_EINVAL
    # misaligned device pointer (checked before any CUDA call)
    assert orch.lib().ot_tree_model_upload(C.byref(d), C.byref(fl), C.c_void_p(4), 1 << 20, None,
                                           C.byref(h)) == orch.OT_EINVAL
    # invalid flags
    bad = orch.make_flags(I.Flags(n_break=0))
    assert orch.lib().ot_tree_model_upload(C.byref(d), C.byref(bad), C.c_void_p(256), 1 << 20, None,
                                           C.byref(h)) == orch.OT_EINVAL
    # FP64 twig pivots asked for without diameters, or with a bad threshold
    twig = orch.make_flags(I.Flags(fp64_twig_diam=0.005))
    d_nodiam = orch.make_desc(f, keep)
    d_nodiam.diam = None
    assert orch.lib().ot_tree_model_upload(C.byref(d_nodiam), C.byref(twig), C.c_void_p(256), 1 << 20, None,
                                           C.byref(h)) == orch.OT_EINVAL
    neg = orch.make_flags(I.Flags(fp64_twig_diam=-1.0))
    assert orch.lib().ot_tree_model_upload(C.byref(d), C.byref(neg), C.c_void_p(256), 1 << 20, None,
                                           C.byref(h)) == orch.OT_EINVAL
    # body damping coefficients must be finite and non-negative
    for kw in (dict(lin_damping=-1.0), dict(ang_damping=float("nan")), dict(snapped_lin_damping=-0.5),
               dict(lin_damping=float("inf")), dict(rail_speed=-1.0),
               dict(rail_speed=2.0, rail_fade_speed=2.0), dict(rail_speed=2.0, rail_fade_speed=-0.1),
               dict(rail_speed=2.0, rail_fade_speed=1.0, rail_brake=-1.0)):
        bad_d = orch.make_flags(I.Flags(**kw))
        assert orch.lib().ot_tree_model_upload(C.byref(d), C.byref(bad_d), C.c_void_p(256), 1 << 20, None,
                                               C.byref(h)) == orch.OT_EINVAL, kw
    assert h.value is None


def test_flop_count_scales_with_the_terms():
    from paper_2607_06337_b300 import costs
    f = I.make_forest(I.PLAIN, worlds=[0])
    nb, nv, na, E, P = costs.world_terms(f)
    assert nv[0] == 2 * (nb[0] - 1)
    depth = costs.dof_depths(f)
    assert E[0] == depth.sum() and P[0] == (depth * (depth + 1) // 2).sum()
    per_body = costs.flops_per_step(f) / costs.body_count(f)
    assert 500 < per_body < 5000  # of the order of a few kflop per body-step


def test_flop_model_against_the_executed_fp32_instructions():
    """The algorithmic flop count behind the roofline fraction (paper_2607_06337_b300/costs.py,
    a tally of the step's arithmetic: FMA 2, add, multiply, divide, square root, sine and cosine
    1) against the hardware's own count: the FP32 instructions the rollout kernel executed over
    a recorded rollout (ncu, 2 FFMA + FADD + FMUL with the predicate on, all size classes;
    profiles/rollout_fp32_ops_batch4096_600w.json). The executed count bounds the algorithmic
    one from above: the kernel also executes the redundant adds of its segmented scans, pivot
    inverses computed once per warp, and the division and square-root sequences. A model that
    overcounts, or misses a quarter of the work, fails."""
    import json
    import os

    from paper_2607_06337_b300 import costs
    from paper_2607_06337_b300 import inputs as I
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rec = json.load(open(os.path.join(root, "profiles", "rollout_fp32_ops_batch4096_600w.json")))
    f = I.make_forest(rec["workload"], n_worlds=rec["worlds"])
    algo = costs.flops_per_step(f) * rec["sim_steps"]
    ratio = algo / rec["fp32_flops_executed"]
    assert 0.75 <= ratio <= 1.0, ratio
    assert rec["fp64_flops_executed"] == 0  # no FP64 pivots in this workload


def test_adjoint_flop_model_against_the_executed_fp32_instructions():
    """The backward's flop tally (costs.adjoint_flops_per_step without the replayed forward step,
    as in the tape form) against the FP32 instructions one tape-form backward launch executed
    over a 20-step recorded rollout of 256 diff1024 trees (ncu, 2 FFMA + FADD + FMUL;
    profiles/backward_fp32_ops_diff1024_256w.json). The executed count bounds it from above (the
    scans' redundant adds, divisions and square roots expanded); within a quarter below."""
    import json
    import os

    from paper_2607_06337_b300 import costs
    from paper_2607_06337_b300 import inputs as I
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rec = json.load(open(os.path.join(root, "profiles", "backward_fp32_ops_diff1024_256w.json")))
    f = I.make_forest(rec["workload"], n_worlds=rec["worlds"])
    algo = costs.adjoint_flops_per_step(f, replay=False) * rec["sim_steps"]
    ratio = algo / rec["fp32_flops_executed"]
    assert 0.75 <= ratio <= 1.0, ratio
