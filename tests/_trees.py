"""Hand-built test trees (single hinge, straight cantilever chain, small random trees)."""
import math

import numpy as np

from paper_2607_06337_b300 import inputs as I
from paper_2607_06337_b300.inputs import Forest


def single_hinge(diam=0.02, length=0.2, rho=700.0, k=50.0, kd=0.0, ndof=1, gravity=(0.0, 0.0, 0.0),
                 qrel=(1.0, 0.0, 0.0, 0.0)):
    m, com, inertia = I.cylinder(diam, length, rho)
    body = dict(parent=-1, ndof=ndof, jpos=(0.0, 0.0, 0.0), qrel=qrel, mass=m, com=com, inertia=inertia,
                k=k, kd=kd, length=length, diam=diam)
    f = I.from_bodies([body], tips=[(0, (0.0, 0.0, length))], gravity=gravity)
    J = inertia[0] + m * (0.5 * length) ** 2
    return f, J, m


def chain(n, seg_len, diam, rho, E, kd, ndof=1, apple=None, gravity=(0.0, 0.0, 0.0), m_max=1e30):
    """A straight vertical chain of n equal segments; the root joint is compliant too."""
    m, com, inertia = I.cylinder(diam, seg_len, rho)
    k = I.beam_stiffness(E, diam, seg_len)
    bodies = []
    for i in range(n):
        bodies.append(dict(parent=i - 1, ndof=ndof, jpos=(0.0, 0.0, 0.0 if i == 0 else seg_len),
                           qrel=(1.0, 0.0, 0.0, 0.0), mass=m, com=com, inertia=inertia, k=k, kd=kd,
                           length=seg_len, diam=diam, m_max=m_max))
    apples = []
    if apple is not None:
        apples.append(dict(body=n - 1, hang_local=(0.0, 0.0, seg_len), attach_local=(0.0, 0.0, seg_len),
                           x0=(0.0, 0.0, 0.0), v0=(0.0, 0.0, 0.0), **apple))
    f = I.from_bodies(bodies, apples=apples, tips=[(n - 1, (0.0, 0.0, seg_len))], gravity=gravity)
    return f, k


def small_random_tree(seed, n_b=6, depth=3, n_a=0, ndof=2, root_ndof=0):
    """A generated world of a few bodies (same recipe as the configs, smaller)."""
    rec = I.WorldRecipe(n_b, depth, n_a)
    f = I.make_forest(I.PLAIN, n_worlds=1, worlds=[0], sweep=1000 + seed, recipe_override=rec)
    if ndof != 2 or root_ndof != 0:
        nd = np.where(f.parent >= 0, ndof, root_ndof).astype(np.int32)
        f.ndof = nd
        f.q0 = np.zeros(int(nd.sum()))
        f.qd0 = np.zeros(int(nd.sum()))
        # a compliant root needs stiffness of its own
        f.k = np.where(nd > 0, np.maximum(f.k, 1.0), 0.0)
        f.kd = np.where(nd > 0, f.kd, 0.0)
    return f


def rot_x(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def rot_y(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def joint_axes(f, q, w=0):
    """World DOF axes (and their body) by a direct forward pass, for the brute-force checks."""
    b0, b1 = f.body_off[w], f.body_off[w + 1]
    nb = b1 - b0
    R = [None] * nb
    axes = []
    dof_body = []
    i = 0
    for b in range(nb):
        p = f.parent[b0 + b]
        Rp = np.eye(3) if p < 0 else R[p]
        Rj = Rp @ I.quat_to_mat(f.qrel[b0 + b])
        for j in range(f.ndof[b0 + b]):
            axes.append(Rj[:, j].copy())
            dof_body.append(b)
            Rj = Rj @ (rot_x(q[i]) if j == 0 else rot_y(q[i]))
            i += 1
        R[b] = Rj
    return np.array(axes).reshape(-1, 3), np.array(dof_body, int), R


def concat(forests):
    """Pack several one-or-more-world forests into one."""
    cat = lambda name: np.concatenate([getattr(x, name) for x in forests])

    def offs(name):
        out = [0]
        for x in forests:
            o = getattr(x, name)
            out.extend((out[-1] + o[1:]).tolist())
        return np.array(out, np.int32)

    return Forest(
        n_worlds=sum(x.n_worlds for x in forests), body_off=offs("body_off"), apple_off=offs("apple_off"),
        tip_off=offs("tip_off"), parent=cat("parent"), ndof=cat("ndof"), jpos=cat("jpos"), qrel=cat("qrel"),
        length=cat("length"), diam=cat("diam"), mass=cat("mass"), com=cat("com"), inertia=cat("inertia"),
        k=cat("k"), kd=cat("kd"), armature=cat("armature"), m_max=cat("m_max"), apple_body=cat("apple_body"),
        hang_local=cat("hang_local"), attach_local=cat("attach_local"), apple_mass=cat("apple_mass"),
        k_s=cat("k_s"), c_s=cat("c_s"), f_detach=cat("f_detach"), tip_body=cat("tip_body"),
        tip_local=cat("tip_local"), gravity=cat("gravity"), q0=cat("q0"), qd0=cat("qd0"),
        apple_x0=cat("apple_x0"), apple_v0=cat("apple_v0"), pull_force=cat("pull_force"),
        pull_start=cat("pull_start"), pull_end=cat("pull_end"))
