"""Seeded synthetic tree forests: the input recipe consumed by both the CUDA step and the oracle.

This module holds none of the step's arithmetic (no kinematics, dynamics, factorisation or
event logic). It samples tree topologies and rest geometry and writes out the per-body and
per-apple descriptor values that the step takes as inputs:

* topology: a random-frontier growth (each expansion gives a node U{2,3} children, up to a
  depth limit and an exact body budget), children placed at a U(20 deg, 60 deg) branch angle
  and at azimuths phi + i * 137.5 deg, the golden-angle divergence of the L-system (Sec. III,
  Eq. 1);
* diameters by the pipe rule with exponent 2 (Sec. III, Eq. 2 with beta = 2):
  d_b = d_trunk * sqrt(leaves(b) / leaves(root)), which gives d_p^2 = sum d_c^2 exactly;
* solid-cylinder links of wood density rho (Sec. IV): m = rho pi d^2 l / 4,
  I_xx = I_yy = m (3 r^2 + l^2) / 12, I_zz = m r^2 / 2, centre of mass at l / 2;
* joint rest transforms (Sec. IV, Eq. 3): T = (0, 0, l_parent) * q_rel;
* Euler-Bernoulli stiffness k = E I / l with I = pi r^4 / 4 (Sec. IV-A, Eq. 4);
* damping kd = 2 zeta sqrt(k J), the inversion of the paper's zeta_eff = c_d sqrt(k) / (2 sqrt(J))
  (Sec. IV-A), J the subtree's moment of inertia about the joint axes at rest;
* rupture moment M_max = sigma_r pi r^3 / 4 (Sec. IV-B, Eq. 5);
* apples on leaf spurs (Sec. IV-C): tether hang point 3 cm below the spur tip, k_s, c_s,
  detach force, initial stem elongation at the rest sag m g / k_s (an attached apple's state
  is its elongation x - x_hang; a detached apple's is its world position);
* the external pull schedule on apples.

Model variants (ModelVariant, the defaults above unless asked for): the pipe exponent beta in
[2.0, 2.5] (Sec. III, Eq. 2), capsule links (a cylinder of the segment's length with
hemispherical caps, Sec. IV), the paper's damping law Kd = c_d Kp (Sec. IV-A, Eq. 4), and the
per-level exponential stiffness k = k_0 gamma^(depth - 1) (Sec. IV-A).

Every value is derived in float64 from a ``numpy.random.Generator(PCG64(seed))`` with
seed = 1_000_003 * (the workload's position in WORKLOADS) + world, so both sides receive
bit-identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GRAVITY = 9.81
GOLDEN_ANGLE = math.radians(137.5)


# ----------------------------------------------------------------------------------------
# Model flags (the readings of the paper that are switchable).
# ----------------------------------------------------------------------------------------
@dataclass
class Flags:
    dt: float = 2e-3
    alpha_implicit_spring: int = 1   # 1: H += dt^2 K' (implicit position actuator), 0: explicit
    tether_implicit: int = 1         # 1: tether reaction linearised at the end of the step
    n_break: int = 5                 # N_b: steps over the rupture moment before a break
    n_pull: int = 3                  # N_p: steps of pull > f_det before detach
    n_tension: int = 10              # N_t: steps of tension > gamma f_det before detach
    gamma_tension: float = 1.2       # tension threshold factor (and reaction clamp factor)
    clamp_factor: float = 1.2        # reaction clamp F_clamp = clamp_factor * f_det
    break_ramp_s: float = 1.5        # post-break friction surrogate: ramp time (s)
    break_ramp_factor: float = 5.0   # ... from kd up to this multiple of kd
    fp64_twig_diam: float = 0.0      # joints thinner than this use float64 pivots (0: none)
    lin_damping: float = 0.0         # c_v (1/s): force -c_v m v at each body's centre of mass
    ang_damping: float = 0.0         # c_omega (1/s): torque -c_omega I omega
    snapped_lin_damping: float = 0.1  # factor on c_v for a body on a snapped sub-tree
    rail_speed: float = 0.0          # v_lim (m/s) of the applied-force rails (App. B), 0: off
    rail_fade_speed: float = 0.0     # v_fade (m/s): the power fade starts here (< v_lim)
    rail_brake: float = 0.0          # c_b (1/s): speed brake above v_lim


@dataclass
class ModelVariant:
    """Switches of the generated model (defaults: the workloads' model)."""
    pipe_exponent: float = 2.0       # beta of r_parent^beta = sum r_child^beta (Eq. 2), in [2, 2.5]
    capsule: bool = False            # capsule links (cylinder + hemispherical caps) for mass, inertia
    damping_cd: float = 0.0          # > 0: Kd = c_d Kp (Eq. 4) with this c_d (s) instead of the zeta law
    level_k0: float = 0.0            # > 0: per-level stiffness k = level_k0 level_gamma^(depth - 1)
    level_gamma: float = 0.3


@dataclass
class Forest:
    """Packed-CSR batch of worlds; per-world arrays are indexed world-locally."""

    n_worlds: int
    body_off: np.ndarray      # int32 [W+1]
    apple_off: np.ndarray     # int32 [W+1]
    tip_off: np.ndarray       # int32 [W+1]
    # per body
    parent: np.ndarray        # int32 world-local parent, -1 for the root
    ndof: np.ndarray          # int32 0, 1 or 2 (Cardan x then y')
    jpos: np.ndarray          # (nb,3) joint origin in the parent frame
    qrel: np.ndarray          # (nb,4) rest rotation relative to the parent (w,x,y,z)
    length: np.ndarray        # (nb,)
    diam: np.ndarray          # (nb,)
    mass: np.ndarray          # (nb,)
    com: np.ndarray           # (nb,3) centre of mass in the body frame
    inertia: np.ndarray       # (nb,3) principal inertia about the com, body axes
    k: np.ndarray             # (nb,) joint stiffness [N m / rad]
    kd: np.ndarray            # (nb,) joint damping [N m s / rad]
    armature: np.ndarray      # (nb,)
    m_max: np.ndarray         # (nb,) rupture moment [N m]
    # per apple
    apple_body: np.ndarray    # int32 world-local body
    hang_local: np.ndarray    # (na,3) hang point in the body frame
    attach_local: np.ndarray  # (na,3) stem attach point in the body frame
    apple_mass: np.ndarray
    k_s: np.ndarray
    c_s: np.ndarray
    f_detach: np.ndarray
    # per tip (loss / record points)
    tip_body: np.ndarray      # int32 world-local
    tip_local: np.ndarray     # (nt,3)
    # per world
    gravity: np.ndarray       # (W,3)
    # initial state
    q0: np.ndarray = None     # (nv,)
    qd0: np.ndarray = None
    apple_x0: np.ndarray = None   # (na,3) stem elongation x - x_hang while attached
    apple_v0: np.ndarray = None
    # external pull schedule: force applied from pull_start (inclusive) to pull_end (exclusive)
    pull_force: np.ndarray = None  # (na,3)
    pull_start: np.ndarray = None  # int32 (na,), large = never
    pull_end: np.ndarray = None    # int32 (na,)
    # rest geometry in world coordinates (for pins and diagnostics)
    rest_x: np.ndarray = None      # (nb,3) joint origins
    rest_R: np.ndarray = None      # (nb,3,3)
    # per-body material, for domain randomisation (None: not a generated tree)
    rho: np.ndarray = None         # (nb,) wood density [kg/m^3]
    youngs: np.ndarray = None      # (nb,) Young's modulus [Pa]
    sigma_r: np.ndarray = None     # (nb,) modulus of rupture [Pa]
    meta: dict = field(default_factory=dict)

    # --------------------------------------------------------------------------------
    @property
    def n_bodies(self) -> int:
        return int(self.body_off[-1])

    @property
    def n_apples(self) -> int:
        return int(self.apple_off[-1])

    @property
    def n_tips(self) -> int:
        return int(self.tip_off[-1])

    @property
    def dof_off(self) -> np.ndarray:
        per_world = np.add.reduceat(self.ndof.astype(np.int64), self.body_off[:-1]) \
            if self.n_bodies else np.zeros(self.n_worlds, np.int64)
        per_world = np.where(np.diff(self.body_off) > 0, per_world, 0)
        return np.concatenate([[0], np.cumsum(per_world)]).astype(np.int32)

    @property
    def n_dofs(self) -> int:
        return int(self.ndof.sum())

    def world_sizes(self):
        return (np.diff(self.body_off), np.diff(self.dof_off), np.diff(self.apple_off))

    def subset(self, worlds) -> "Forest":
        """A new forest holding only the listed worlds (in the given order)."""
        worlds = [int(w) for w in worlds]
        bo, ao, to, do = self.body_off, self.apple_off, self.tip_off, self.dof_off
        bsel = np.concatenate([np.arange(bo[w], bo[w + 1]) for w in worlds]).astype(np.int64)
        asel = np.concatenate([np.arange(ao[w], ao[w + 1]) for w in worlds] + [np.zeros(0, np.int64)]).astype(np.int64)
        tsel = np.concatenate([np.arange(to[w], to[w + 1]) for w in worlds] + [np.zeros(0, np.int64)]).astype(np.int64)
        dsel = np.concatenate([np.arange(do[w], do[w + 1]) for w in worlds] + [np.zeros(0, np.int64)]).astype(np.int64)

        def off(o):
            return np.concatenate([[0], np.cumsum([o[w + 1] - o[w] for w in worlds])]).astype(np.int32)

        def opt(a, sel):
            return None if a is None else a[sel].copy()

        return Forest(
            n_worlds=len(worlds), body_off=off(bo), apple_off=off(ao), tip_off=off(to),
            parent=self.parent[bsel].copy(), ndof=self.ndof[bsel].copy(), jpos=self.jpos[bsel].copy(),
            qrel=self.qrel[bsel].copy(), length=self.length[bsel].copy(), diam=self.diam[bsel].copy(),
            mass=self.mass[bsel].copy(), com=self.com[bsel].copy(), inertia=self.inertia[bsel].copy(),
            k=self.k[bsel].copy(), kd=self.kd[bsel].copy(), armature=self.armature[bsel].copy(),
            m_max=self.m_max[bsel].copy(), apple_body=self.apple_body[asel].copy(),
            hang_local=self.hang_local[asel].copy(), attach_local=self.attach_local[asel].copy(),
            apple_mass=self.apple_mass[asel].copy(), k_s=self.k_s[asel].copy(), c_s=self.c_s[asel].copy(),
            f_detach=self.f_detach[asel].copy(), tip_body=self.tip_body[tsel].copy(),
            tip_local=self.tip_local[tsel].copy(), gravity=self.gravity[worlds].copy(),
            q0=opt(self.q0, dsel), qd0=opt(self.qd0, dsel), apple_x0=opt(self.apple_x0, asel),
            apple_v0=opt(self.apple_v0, asel), pull_force=opt(self.pull_force, asel),
            pull_start=opt(self.pull_start, asel), pull_end=opt(self.pull_end, asel),
            rest_x=opt(self.rest_x, bsel), rest_R=opt(self.rest_R, bsel),
            rho=opt(self.rho, bsel), youngs=opt(self.youngs, bsel), sigma_r=opt(self.sigma_r, bsel),
            meta=dict(self.meta, subset=worlds),
        )

    @staticmethod
    def concat(forests: list) -> "Forest":
        """One forest holding the worlds of several, in order."""
        import dataclasses
        offs = ("body_off", "apple_off", "tip_off")
        kw = {"n_worlds": sum(f.n_worlds for f in forests)}
        for name in offs:
            out = [0]
            for f in forests:
                out.extend((out[-1] + np.asarray(getattr(f, name))[1:]).tolist())
            kw[name] = np.array(out, np.int32)
        for fld in dataclasses.fields(Forest):
            if fld.name in kw or fld.name == "meta":
                continue
            parts = [getattr(f, fld.name) for f in forests]
            kw[fld.name] = None if any(p is None for p in parts) else np.concatenate(parts)
        meta = dict(forests[0].meta) if forests else {}
        for key in ("E", "sigma_r"):
            if forests and all(key in f.meta for f in forests):
                meta[key] = np.concatenate([f.meta[key] for f in forests])
        kw["meta"] = meta
        return Forest(**kw)

    def forces_at(self, step: int) -> np.ndarray:
        """External pull on every apple during simulation step ``step`` (na,3)."""
        on = (step >= self.pull_start) & (step < self.pull_end)
        return np.where(on[:, None], self.pull_force, 0.0)


# ----------------------------------------------------------------------------------------
# Quaternion / rotation helpers (input geometry only).
# ----------------------------------------------------------------------------------------
def quat_mul(a, b):
    aw, ax, ay, az = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([
        aw * bw - ax * bx - ay * by - az * bz,
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
    ], axis=-1)


def quat_to_mat(q):
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def quat_axis_angle(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    angle = np.asarray(angle, dtype=np.float64)
    h = 0.5 * angle
    s = np.sin(h)
    out = np.zeros(np.broadcast(angle, axis[..., 0]).shape + (4,))
    out[..., 0] = np.cos(h)
    out[..., 1:] = axis * s[..., None]
    return out


# ----------------------------------------------------------------------------------------
# Topology growth.
# ----------------------------------------------------------------------------------------
def _grow_topology(rng: np.random.Generator, n_b: int, depth_max: int):
    """Random-frontier growth, returned in breadth-first order.

    Repeatedly a uniformly random unexpanded node of depth < depth_max receives U{2,3}
    children (truncated at the body budget). If the frontier empties before n_b bodies exist,
    a random node of depth < depth_max with fewer than 3 children receives one more child.
    """
    parent = [-1]
    depth = [0]
    nchild = [0]
    frontier = [0] if depth_max > 0 else []
    while len(parent) < n_b:
        if frontier:
            i = int(rng.integers(len(frontier)))
            node = frontier[i]
            frontier[i] = frontier[-1]
            frontier.pop()
            c = min(int(rng.integers(2, 4)), n_b - len(parent))
        else:
            cands = [j for j in range(len(parent)) if depth[j] < depth_max and 0 < nchild[j] < 3]
            if not cands:
                break
            node = cands[int(rng.integers(len(cands)))]
            c = 1
        for _ in range(c):
            parent.append(node)
            depth.append(depth[node] + 1)
            nchild.append(0)
            nchild[node] += 1
            if depth[-1] < depth_max:
                frontier.append(len(parent) - 1)
    n = len(parent)
    children = [[] for _ in range(n)]
    for j in range(1, n):
        children[parent[j]].append(j)
    order = [0]
    head = 0
    while head < len(order):
        order.extend(children[order[head]])
        head += 1
    new = np.empty(n, np.int64)
    new[np.asarray(order)] = np.arange(n)
    par = np.full(n, -1, np.int64)
    cidx = np.zeros(n, np.int64)
    for old in range(n):
        if parent[old] >= 0:
            par[new[old]] = new[parent[old]]
    for old_p in range(n):
        for i, old_c in enumerate(children[old_p]):
            cidx[new[old_c]] = i
    dep = np.asarray(depth)[np.asarray(order)]
    return par, cidx, dep


# ----------------------------------------------------------------------------------------
# Config recipes (the five workloads).
# ----------------------------------------------------------------------------------------
@dataclass
class WorldRecipe:
    n_bodies: int
    depth: int
    n_apples: int
    pulls: str = "none"           # "none" | "random25" | "fixed5"


# The workloads, by name. The position of a name in WORKLOADS is its seed stream.
PLAIN = "plain16"        # 16 trees x 64 bodies (depth 5) x 8 apples, gravity only, 1000 steps
BATCH = "batch4096"      # 4096 uneven trees: 100-600 bodies, depth 6-8, 20-120 apples,
                         # random 0-60 N pulls on a quarter of the apples, 1000 steps
SWEEP = "sweep16384"     # 16384 trees x 300 bodies (depth 8) x 60 apples, 1000 steps
DIFF = "diff1024"        # 1024 trees x 200 bodies (depth 8) x 30 apples, a fixed 5 N pull, 200 steps
STRESS = "stress8192"    # 8192 mixed trees: half 50 bodies, 40% 400, 10% 2000 (depth 6/8/10),
                         # 10-200 apples, 500 steps
WORKLOADS = (PLAIN, BATCH, SWEEP, DIFF, STRESS)
WORKLOAD_WORLDS = {PLAIN: 16, BATCH: 4096, SWEEP: 16384, DIFF: 1024, STRESS: 8192}
WORKLOAD_STEPS = {PLAIN: 1000, BATCH: 1000, SWEEP: 1000, DIFF: 200, STRESS: 500}


def world_recipe(workload: str, w: int, n_worlds: int, rng: np.random.Generator) -> WorldRecipe:
    if workload == PLAIN:
        return WorldRecipe(64, 5, 8)
    if workload == BATCH:
        return WorldRecipe(int(rng.integers(100, 601)), int(rng.integers(6, 9)),
                           int(rng.integers(20, 121)), "random25")
    if workload == SWEEP:
        return WorldRecipe(300, 8, 60)
    if workload == DIFF:
        return WorldRecipe(200, 8, 30, "fixed5")
    if workload == STRESS:
        frac = (w + 0.5) / n_worlds
        n_a = int(rng.integers(10, 201))
        if frac < 0.5:
            return WorldRecipe(50, 6, n_a)
        if frac < 0.9:
            return WorldRecipe(400, 8, n_a)
        return WorldRecipe(2000, 10, n_a)
    raise ValueError(f"unknown workload {workload!r}")


def world_seed(workload: str, w: int, sweep: int = 0) -> int:
    return 1_000_003 * WORKLOADS.index(workload) + w + 10_000_019 * sweep


def _make_worlds(workload: str, worlds: list, full: int, sweep: int, recipe_override) -> list:
    per = []
    for w in worlds:
        rng = np.random.Generator(np.random.PCG64(world_seed(workload, w, sweep)))
        rec = recipe_override or world_recipe(workload, w, full, rng)
        per.append(_make_world(rng, rec))
    return per


def _make_packed(workload: str, worlds: list, full: int, sweep: int, recipe_override, var) -> "Forest":
    return _pack(_make_worlds(workload, worlds, full, sweep, recipe_override), var)


def make_forest(workload: str, n_worlds: int | None = None, worlds=None, sweep: int = 0,
                recipe_override: WorldRecipe | None = None, variant: ModelVariant | None = None,
                processes: int = 1) -> Forest:
    """Generate a named workload (optionally a subset of its worlds).

    ``worlds`` picks world indices of the full workload (the seeds do not change), so a subset
    holds exactly the same trees as the full batch. ``sweep`` > 0 draws fresh seeds of the
    same distribution (the world-count sweep, and one batch per rank). ``processes`` > 1
    grows the trees in that many spawned worker processes (each world has its own seed, so
    the forest is the same).
    """
    if workload not in WORKLOADS:
        raise ValueError(f"unknown workload {workload!r}; one of {WORKLOADS}")
    full = WORKLOAD_WORLDS[workload] if n_worlds is None else n_worlds
    worlds = list(range(full)) if worlds is None else [int(w) for w in worlds]
    var = variant or ModelVariant()
    if processes > 1 and len(worlds) >= 512:
        # each worker grows and packs a chunk of worlds; packing is per world, so the chunks
        # concatenate to the same forest
        import multiprocessing as mp
        chunks = [c.tolist() for c in np.array_split(np.array(worlds, np.int64), 2 * processes)]
        with mp.get_context("spawn").Pool(processes) as pool:
            parts = pool.starmap(_make_packed, [(workload, c, full, sweep, recipe_override, var) for c in chunks])
        forest = Forest.concat(parts)
    else:
        forest = _pack(_make_worlds(workload, worlds, full, sweep, recipe_override), var)
    forest.meta.update(workload=workload, n_worlds_full=full, worlds=worlds, sweep=sweep)
    return forest


def _make_world(rng: np.random.Generator, rec: WorldRecipe) -> dict:
    par, cidx, dep = _grow_topology(rng, rec.n_bodies, rec.depth)
    n = len(par)
    E = rng.uniform(6e9, 10e9)
    sigma_r = rng.uniform(50e6, 90e6)
    rho = 700.0
    zeta = 0.05
    length = rng.uniform(0.1, 0.3, n)
    phi = rng.uniform(0.0, 2 * math.pi, n)
    angle = np.radians(rng.uniform(20.0, 60.0, n))
    # apples on leaf spurs
    is_leaf = np.ones(n, bool)
    is_leaf[par[par >= 0]] = False
    leaves = np.nonzero(is_leaf)[0]
    n_a = rec.n_apples
    if n_a <= len(leaves):
        abody = rng.choice(leaves, n_a, replace=False)
    else:
        abody = rng.choice(leaves, n_a, replace=True)
    amass = rng.uniform(0.15, 0.25, n_a)
    fdet = rng.uniform(10.0, 30.0, n_a)
    pull_force = np.zeros((n_a, 3))
    pull_start = np.full(n_a, 1 << 30, np.int64)
    pull_end = np.full(n_a, 1 << 30, np.int64)
    if rec.pulls == "random25" and n_a > 0:
        n_pull = int(round(0.25 * n_a))
        sel = rng.choice(n_a, n_pull, replace=False)
        mag = rng.uniform(0.0, 60.0, n_pull)
        d = rng.standard_normal((n_pull, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pull_force[sel] = d * mag[:, None]
        pull_start[sel] = rng.integers(0, 501, n_pull)
    elif rec.pulls == "fixed5" and n_a > 0:
        pull_force[0] = 5.0 * np.array([1.0, 0.0, -1.0]) / math.sqrt(2.0)
        pull_start[0] = 0
    # apples sorted by their body (stable), so each body's apples form a contiguous range
    order = np.argsort(abody, kind="stable")
    abody, amass, fdet = abody[order], amass[order], fdet[order]
    pull_force, pull_start, pull_end = pull_force[order], pull_start[order], pull_end[order]
    return dict(par=par, cidx=cidx, dep=dep, E=E, sigma_r=sigma_r, rho=rho, zeta=zeta,
                length=length, phi=phi, angle=angle, abody=abody, amass=amass, fdet=fdet,
                pull_force=pull_force, pull_start=pull_start, pull_end=pull_end, leaves=leaves)


def _pack(per: list, var: ModelVariant) -> Forest:
    W = len(per)
    nbs = np.array([len(p["par"]) for p in per], np.int64)
    nas = np.array([len(p["abody"]) for p in per], np.int64)
    nts = np.array([len(p["leaves"]) for p in per], np.int64)
    body_off = np.concatenate([[0], np.cumsum(nbs)]).astype(np.int32)
    apple_off = np.concatenate([[0], np.cumsum(nas)]).astype(np.int32)
    tip_off = np.concatenate([[0], np.cumsum(nts)]).astype(np.int32)
    NB = int(body_off[-1])
    cat = lambda key: np.concatenate([p[key] for p in per]) if per else np.zeros(0)
    par = cat("par").astype(np.int64)
    cidx = cat("cidx").astype(np.int64)
    dep = cat("dep").astype(np.int64)
    length = cat("length")
    phi = cat("phi")
    angle = cat("angle")
    wid = np.repeat(np.arange(W), nbs)
    base = body_off[:-1].astype(np.int64)[wid]
    gpar = np.where(par >= 0, par + base, -1)
    E = np.array([p["E"] for p in per])[wid]
    sig = np.array([p["sigma_r"] for p in per])[wid]
    rho = np.array([p["rho"] for p in per])[wid]
    zeta = np.array([p["zeta"] for p in per])[wid]

    # rest rotation relative to the parent: about the parent z by the azimuth, then tilt about x
    azim = np.zeros(NB)
    nonroot = gpar >= 0
    azim[nonroot] = phi[gpar[nonroot]] + cidx[nonroot] * GOLDEN_ANGLE
    qz = quat_axis_angle(np.array([0.0, 0.0, 1.0]), azim)
    qx = quat_axis_angle(np.array([1.0, 0.0, 0.0]), angle)
    qrel = quat_mul(qz, qx)
    qrel[~nonroot] = np.array([1.0, 0.0, 0.0, 0.0])
    jpos = np.zeros((NB, 3))
    jpos[nonroot, 2] = length[gpar[nonroot]]

    # rest world frames, level by level
    Qw = np.zeros((NB, 4))
    Xw = np.zeros((NB, 3))
    maxd = int(dep.max()) if NB else 0
    for lvl in range(maxd + 1):
        idx = np.nonzero(dep == lvl)[0]
        if lvl == 0:
            Qw[idx] = qrel[idx]
            Xw[idx] = jpos[idx]
        else:
            p = gpar[idx]
            Qw[idx] = quat_mul(Qw[p], qrel[idx])
            Xw[idx] = Xw[p] + np.einsum("nij,nj->ni", quat_to_mat(Qw[p]), jpos[idx])
    Rw = quat_to_mat(Qw)

    # pipe-model diameters from leaf counts
    leaves_in = np.zeros(NB)
    is_leaf = np.ones(NB, bool)
    is_leaf[gpar[nonroot]] = False
    leaves_in[is_leaf] = 1.0
    for lvl in range(maxd, 0, -1):
        idx = np.nonzero(dep == lvl)[0]
        np.add.at(leaves_in, gpar[idx], leaves_in[idx])
    root_of = body_off[:-1].astype(np.int64)[wid]
    # d ~ leaves^(1 / beta): leaves(p) = sum leaves(c) makes d_p^beta = sum d_c^beta exactly
    diam = 0.06 * (leaves_in / leaves_in[root_of]) ** (1.0 / var.pipe_exponent)
    r = 0.5 * diam
    if var.capsule:
        mass, Ixx, Izz = capsule(diam, length, rho)
        inertia = np.stack([Ixx, Ixx, Izz], axis=1)
    else:
        mass = rho * math.pi * diam ** 2 * length / 4.0
        inertia = np.stack([mass * (3 * r ** 2 + length ** 2) / 12.0,
                            mass * (3 * r ** 2 + length ** 2) / 12.0,
                            mass * r ** 2 / 2.0], axis=1)
    com = np.zeros((NB, 3))
    com[:, 2] = 0.5 * length
    ndof = np.where(nonroot, 2, 0).astype(np.int32)
    if var.level_k0 > 0:
        k = np.where(nonroot, var.level_k0 * var.level_gamma ** np.maximum(dep - 1, 0), 0.0)
    else:
        k = np.where(nonroot, math.pi * E * r ** 4 / (4.0 * length), 0.0)
    m_max = sig * math.pi * r ** 3 / 4.0

    # subtree moment of inertia about each joint's rest x and y axes (through the joint)
    comw = Xw + np.einsum("nij,nj->ni", Rw, com)
    Ic_w = np.einsum("nij,nj,nkj->nik", Rw, inertia, Rw)
    J = np.zeros((NB, 2))
    anc = np.arange(NB)
    for _ in range(maxd + 1):
        ok = anc >= 0
        b = anc[ok]
        c = np.nonzero(ok)[0]
        for a in range(2):
            e = Rw[b, :, a]
            d = comw[c] - Xw[b]
            cr = np.cross(d, e)
            val = np.einsum("ni,nij,nj->n", e, Ic_w[c], e) + mass[c] * np.einsum("ni,ni->n", cr, cr)
            np.add.at(J[:, a], b, val)
        anc = np.where(ok, gpar[np.maximum(anc, 0)], -1)
    Jm = J.mean(axis=1)
    if var.damping_cd > 0:
        kd = np.where(nonroot, var.damping_cd * k, 0.0)
    else:
        kd = np.where(nonroot, 2.0 * zeta * np.sqrt(k * Jm), 0.0)

    # apples
    abody = cat("abody").astype(np.int64) if W else np.zeros(0, np.int64)
    awid = np.repeat(np.arange(W), nas)
    gab = abody + body_off[:-1].astype(np.int64)[awid]
    NA = int(apple_off[-1])
    attach_local = np.zeros((NA, 3))
    attach_local[:, 2] = length[gab]
    attach_w = Xw[gab] + np.einsum("nij,nj->ni", Rw[gab], attach_local)
    hang_w = attach_w - np.array([0.0, 0.0, 0.03])
    hang_local = np.einsum("nji,nj->ni", Rw[gab], hang_w - Xw[gab])
    amass = cat("amass")
    k_s = np.full(NA, 1000.0)
    c_s = 2.0 * 0.2 * np.sqrt(k_s * amass)
    # attached apples carry their stem elongation u = x - x_hang; at rest it is the sag m g / k_s
    x0 = -(amass * GRAVITY / k_s)[:, None] * np.array([0.0, 0.0, 1.0])

    # tips: the far end of every leaf segment
    tbody = cat("leaves").astype(np.int64) if W else np.zeros(0, np.int64)
    twid = np.repeat(np.arange(W), nts)
    tip_local = np.zeros((len(tbody), 3))
    tip_local[:, 2] = length[tbody + body_off[:-1].astype(np.int64)[twid]]

    NV = int(ndof.sum())
    f = Forest(
        n_worlds=W, body_off=body_off, apple_off=apple_off, tip_off=tip_off,
        parent=par.astype(np.int32), ndof=ndof, jpos=jpos, qrel=qrel, length=length, diam=diam,
        mass=mass, com=com, inertia=inertia, k=k, kd=kd, armature=np.zeros(NB), m_max=m_max,
        apple_body=abody.astype(np.int32), hang_local=hang_local, attach_local=attach_local,
        apple_mass=amass, k_s=k_s, c_s=c_s, f_detach=cat("fdet"),
        tip_body=tbody.astype(np.int32), tip_local=tip_local,
        gravity=np.tile(np.array([0.0, 0.0, -GRAVITY]), (W, 1)),
        q0=np.zeros(NV), qd0=np.zeros(NV), apple_x0=x0, apple_v0=np.zeros((NA, 3)),
        pull_force=cat("pull_force").reshape(-1, 3) if W else np.zeros((0, 3)),
        pull_start=cat("pull_start").astype(np.int32), pull_end=cat("pull_end").astype(np.int32),
        rest_x=Xw, rest_R=Rw, rho=rho.copy(), youngs=E.copy(), sigma_r=sig.copy(),
    )
    f.meta["capsule"] = bool(var.capsule)
    f.meta["E"] = np.array([p["E"] for p in per])
    f.meta["sigma_r"] = np.array([p["sigma_r"] for p in per])
    return f


def from_bodies(bodies: list, apples: list = (), tips: list = (), gravity=(0.0, 0.0, -GRAVITY)) -> Forest:
    """A one-world forest from explicit body / apple dicts (for hand-built test trees).

    body keys: parent, ndof, jpos, qrel, mass, com, inertia, k, kd, m_max, length, diam, armature
    apple keys: body, hang_local, attach_local, mass, k_s, c_s, f_detach, x0, v0
    """
    nb = len(bodies)
    g = lambda key, default=0.0: np.array([b.get(key, default) for b in bodies], dtype=np.float64)
    apples = list(apples)
    tips = list(tips)
    na = len(apples)
    ga = lambda key, default=0.0: np.array([a.get(key, default) for a in apples], dtype=np.float64).reshape(
        (na,) + np.shape(default))
    ndof = np.array([b.get("ndof", 2) for b in bodies], np.int32)
    NV = int(ndof.sum())
    f = Forest(
        n_worlds=1, body_off=np.array([0, nb], np.int32), apple_off=np.array([0, na], np.int32),
        tip_off=np.array([0, len(tips)], np.int32),
        parent=np.array([b["parent"] for b in bodies], np.int32), ndof=ndof,
        jpos=g("jpos", (0.0, 0.0, 0.0)).reshape(nb, 3),
        qrel=g("qrel", (1.0, 0.0, 0.0, 0.0)).reshape(nb, 4),
        length=g("length", 0.0), diam=g("diam", 0.0), mass=g("mass"),
        com=g("com", (0.0, 0.0, 0.0)).reshape(nb, 3), inertia=g("inertia", (0.0, 0.0, 0.0)).reshape(nb, 3),
        k=g("k"), kd=g("kd"), armature=g("armature"), m_max=g("m_max", 1e30),
        apple_body=np.array([a["body"] for a in apples], np.int32),
        hang_local=ga("hang_local", (0.0, 0.0, 0.0)), attach_local=ga("attach_local", (0.0, 0.0, 0.0)),
        apple_mass=ga("mass"), k_s=ga("k_s"), c_s=ga("c_s"), f_detach=ga("f_detach", 1e30),
        tip_body=np.array([t[0] for t in tips], np.int32),
        tip_local=np.array([t[1] for t in tips], np.float64).reshape(len(tips), 3),
        gravity=np.array([gravity], np.float64),
        q0=np.zeros(NV), qd0=np.zeros(NV),
        apple_x0=ga("x0", (0.0, 0.0, 0.0)), apple_v0=ga("v0", (0.0, 0.0, 0.0)),
        pull_force=np.zeros((na, 3)), pull_start=np.full(na, 1 << 30, np.int32),
        pull_end=np.full(na, 1 << 30, np.int32),
    )
    return f


def cylinder(diam: float, length: float, rho: float):
    """Mass, com and principal inertia of a solid cylinder link along +z."""
    r = 0.5 * diam
    m = rho * math.pi * diam ** 2 * length / 4.0
    return m, (0.0, 0.0, 0.5 * length), (m * (3 * r * r + length * length) / 12.0,
                                          m * (3 * r * r + length * length) / 12.0, m * r * r / 2.0)


DR_FACTORS = ("len", "diam", "rho", "E", "sigma", "c_d")


def randomize(forest: "Forest", factors: np.ndarray, capsule_links: bool = False) -> "Forest":
    """Host counterpart of the on-device domain-randomisation build (ot_model_randomize): per
    world, factors[w] = (s_len, s_diam, s_rho, s_E, s_sigma, c_d) scale the segment lengths (and
    every body-frame point: joint origins, centres of mass, hang and tip points), diameters,
    wood density, Young's modulus and modulus of rupture, and every derived value is rebuilt:
    mass and inertia (solid cylinder, or capsule links), k = E I / l for compliant joints, the
    rupture moment sigma_r pi r^3 / 4, and kd = c_d k (the paper's law, Eq. 4). Topology, rest
    rotations, armature and the apples' own parameters are kept."""
    if forest.rho is None or forest.youngs is None or forest.sigma_r is None:
        raise ValueError("randomize needs the per-body material of a generated forest")
    import copy
    f = copy.deepcopy(forest)
    fac = np.asarray(factors, np.float64).reshape(forest.n_worlds, len(DR_FACTORS))
    wid = np.repeat(np.arange(forest.n_worlds), np.diff(forest.body_off))
    sl, sd, sr, sE, ss, cd = (fac[wid, i] for i in range(6))
    f.length = forest.length * sl
    f.diam = forest.diam * sd
    f.rho = forest.rho * sr
    f.youngs = forest.youngs * sE
    f.sigma_r = forest.sigma_r * ss
    f.jpos = forest.jpos * sl[:, None]
    f.com = forest.com * sl[:, None]
    r = 0.5 * f.diam
    if capsule_links:
        f.mass, Ixx, Izz = capsule(f.diam, f.length, f.rho)
        f.inertia = np.stack([Ixx, Ixx, Izz], axis=1)
    else:
        f.mass = f.rho * math.pi * f.diam ** 2 * f.length / 4.0
        f.inertia = np.stack([f.mass * (3 * r ** 2 + f.length ** 2) / 12.0,
                              f.mass * (3 * r ** 2 + f.length ** 2) / 12.0, f.mass * r ** 2 / 2.0], axis=1)
    f.k = np.where(forest.ndof > 0, math.pi * f.youngs * r ** 4 / (4.0 * f.length), 0.0)
    f.kd = cd * f.k
    f.m_max = f.sigma_r * math.pi * r ** 3 / 4.0
    awid = np.repeat(np.arange(forest.n_worlds), np.diff(forest.apple_off))
    twid = np.repeat(np.arange(forest.n_worlds), np.diff(forest.tip_off))
    f.hang_local = forest.hang_local * fac[awid, 0][:, None]
    f.attach_local = forest.attach_local * fac[awid, 0][:, None]
    f.tip_local = forest.tip_local * fac[twid, 0][:, None]
    f.rest_x = None
    f.rest_R = None
    return f


def capsule(diam, length, rho):
    """Mass and principal inertia (about the centre; axis, then across) of a capsule link: a
    cylinder of radius r and length l along +z with a hemisphere of radius r on each end."""
    r = 0.5 * np.asarray(diam, np.float64)
    l = np.asarray(length, np.float64)
    mc = rho * math.pi * r ** 2 * l                 # the cylinder
    ms = rho * 4.0 / 3.0 * math.pi * r ** 3         # the two caps together
    Izz = mc * r ** 2 / 2.0 + ms * 2.0 * r ** 2 / 5.0
    # each cap: 2/5 m r^2 about the sphere's centre, which sits l/2 from the link's centre;
    # parallel-axis through the cap's own centre of mass, 3 r / 8 beyond the flat face
    Ixx = mc * (3.0 * r ** 2 + l ** 2) / 12.0 + ms * (2.0 * r ** 2 / 5.0 + l ** 2 / 4.0 + 3.0 * l * r / 8.0)
    return mc + ms, Ixx, Izz


def beam_stiffness(E: float, diam: float, length: float) -> float:
    """Euler-Bernoulli rotational stiffness k = E I / l, I = pi r^4 / 4 (Sec. IV-A, Eq. 4)."""
    r = 0.5 * diam
    return math.pi * E * r ** 4 / (4.0 * length)


def rupture_moment(sigma_r: float, diam: float) -> float:
    """Modulus of rupture times section modulus, M_max = sigma_r pi r^3 / 4 (Sec. IV-B, Eq. 5)."""
    r = 0.5 * diam
    return sigma_r * math.pi * r ** 3 / 4.0
