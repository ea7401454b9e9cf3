"""Comparison of a GPU run with the oracle: the joint-position gate and the event-set gate.

Test infrastructure, beside the oracle: the tests and the benchmark's CPU leg use it.

q gate (per world): max |q_gpu - q_ref| <= 1e-4 * max |q_ref| + 1e-7 rad.
Event gate: the sets of (joint, break step) and (apple, detach step) are identical, except that
a mismatch is excused when the oracle logged that test within 1e-5 relative of its threshold at
some step of the hysteresis window ending at the event step; a world with an excused mismatch
is left out of the q gate (its state after the event legitimately differs).
"""
from __future__ import annotations

import numpy as np

Q_REL = 1e-4
Q_ABS = 1e-7
NEAR = 1e-5


def events(broken, break_step, detached, detach_step, f, w):
    b0, b1 = f.body_off[w], f.body_off[w + 1]
    a0, a1 = f.apple_off[w], f.apple_off[w + 1]
    br = {(int(i), int(break_step[b0 + i])) for i in np.nonzero(broken[b0:b1])[0]}
    de = {(int(i), int(detach_step[a0 + i])) for i in np.nonzero(detached[a0:a1])[0]}
    return br, de


def compare(f, flags, gpu: dict, ora_state, ora_near, worlds=None):
    """gpu: dict of numpy arrays q, broken, break_step, detached, detach_step (whole forest)."""
    worlds = range(f.n_worlds) if worlds is None else worlds
    do = f.dof_off
    near = {}
    for w, kind, idx, step in ora_near:
        near.setdefault((int(w), int(kind), int(idx)), []).append(int(step))
    rep = []
    for w in worlds:
        a, b = do[w], do[w + 1]
        dq = float(np.abs(gpu["q"][a:b] - ora_state.q[a:b]).max()) if b > a else 0.0
        sq = float(np.abs(ora_state.q[a:b]).max()) if b > a else 0.0
        gb, gd = events(gpu["broken"], gpu["break_step"], gpu["detached"], gpu["detach_step"], f, w)
        ob, od = events(ora_state.broken, ora_state.break_step, ora_state.detached, ora_state.detach_step, f, w)
        excused, unexcused = [], []
        for kinds, mism, window in (((0,), gb ^ ob, flags.n_break), ((1, 2), gd ^ od, max(flags.n_pull, flags.n_tension))):
            for idx, step in mism:
                ok = any(any(step - window < s <= step for s in near.get((w, k, idx), [])) for k in kinds)
                (excused if ok else unexcused).append((kinds[0], idx, step))
        ratio = dq / (Q_REL * sq + Q_ABS)
        rep.append(dict(world=w, dq=dq, q_scale=sq, ratio=ratio, excused=excused, unexcused=unexcused,
                        q_gated=not excused, n_events=len(ob) + len(od)))
    return rep


def assert_parity(rep):
    bad = [r for r in rep if r["unexcused"] or (r["q_gated"] and r["ratio"] > 1.0)]
    assert not bad, "parity failures: " + "; ".join(
        f"w{r['world']} ratio={r['ratio']:.3g} unexcused={r['unexcused'][:4]}" for r in bad[:8])


def summary(rep) -> dict:
    """The gates of a comparison in a few numbers (for a benchmark record)."""
    gated = [r["ratio"] for r in rep if r["q_gated"]]
    return {"worlds": len(rep), "q_gate_ratio_max": float(max(gated)) if gated else None,
            "q_gate_ratio_p50": float(np.median(gated)) if gated else None,
            "q_err_max_rad": float(max(r["dq"] for r in rep)) if rep else None,
            "events": int(sum(r["n_events"] for r in rep)),
            "event_sets_identical": not any(r["unexcused"] or r["excused"] for r in rep),
            "excused": int(sum(len(r["excused"]) for r in rep)),
            "unexcused": int(sum(len(r["unexcused"]) for r in rep)),
            "pass": not any(r["unexcused"] or (r["q_gated"] and r["ratio"] > 1.0) for r in rep)}
