"""Seeded synthetic robots and knot-point states.

This module is the ONLY code shared by the CUDA path and the FP64 oracle. It
draws numbers; it holds none of the dynamics arithmetic (no spatial algebra, no
inertia assembly, no transforms). Both sides consume the raw arrays it returns:

  parent  int32 [n]       parent body index, -1 = fixed base, parent[i] < i
  jtype   int32 [n]       joint type: 0 revolute, 1 prismatic, 2 fixed (optional;
                          absent means all revolute)
  axis    float64 [n,3]   unit joint axis in the joint (child) frame (ignored
                          for a fixed joint)
  xtree   float64 [n,12]  E (3x3 row-major, maps parent coordinates to child
                          coordinates) then r (child origin in parent coords)
  inertia float64 [n,10]  m, c[3] (COM in link frame), Ixx Iyy Izz Ixy Ixz Iyz
                          (rotational inertia about the COM)
  gravity float64 [3]     gravity vector in base coordinates

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma and each output is the published 64-bit finaliser; doubles take the top
53 bits. One independent stream per (workload, purpose).

The three workload robots stand in for the paper's IIWA (7 dof), HyQ (12 dof)
and Atlas (30 dof) of Sec. V-A, whose URDFs are not available: a 7-DoF serial
chain, a 12-DoF torso with four 3-joint legs (longest path 3) and a 30-DoF
humanoid-like tree (longest path 8, matching the path lengths quoted in Sec. V-C).
"""
from __future__ import annotations

import dataclasses
import zlib

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
G_STD = 9.81


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(workload: int, purpose: str) -> int:
    """Seed of the stream for one (workload id, purpose) pair."""
    key = np.array([(workload * 0x100000001B3) ^ zlib.crc32(purpose.encode())],
                   dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(_mix(key + GAMMA)[0])


class Stream:
    """Counter-based splitmix64 stream: output k is mix(seed + (k+1)*gamma)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.count = 0

    def u64(self, k: int) -> np.ndarray:
        idx = np.arange(self.count + 1, self.count + k + 1, dtype=np.uint64)
        self.count += k
        with np.errstate(over="ignore"):
            return _mix(self.seed + idx * GAMMA)

    def unit(self, size) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        size = tuple(np.atleast_1d(size))
        k = int(np.prod(size))
        return ((self.u64(k) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53).reshape(size)

    def uniform(self, lo, hi, size) -> np.ndarray:
        return lo + (hi - lo) * self.unit(size)

    def normal(self, size) -> np.ndarray:
        """Standard normals by the Box-Muller transform."""
        size = tuple(np.atleast_1d(size))
        k = int(np.prod(size))
        u1 = 1.0 - self.unit(k)          # (0, 1]
        u2 = self.unit(k)
        return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(size)


REVOLUTE, PRISMATIC, FIXED = 0, 1, 2


@dataclasses.dataclass
class Robot:
    name: str
    parent: np.ndarray
    axis: np.ndarray
    xtree: np.ndarray
    inertia: np.ndarray
    gravity: np.ndarray
    jtype: np.ndarray | None = None   # per body: REVOLUTE, PRISMATIC or FIXED (None: all revolute)

    @property
    def n(self) -> int:
        """Bodies (equal to the degrees of freedom when no joint is fixed)."""
        return int(self.parent.shape[0])

    @property
    def nd(self) -> int:
        """Degrees of freedom: the moving (non-fixed) joints."""
        return self.n if self.jtype is None else int(np.count_nonzero(self.jtype != FIXED))

    def jtypes(self) -> np.ndarray:
        jt = np.zeros(self.n, dtype=np.int32) if self.jtype is None else self.jtype
        return np.ascontiguousarray(jt, dtype=np.int32)

    def arrays(self):
        return (np.ascontiguousarray(self.parent, dtype=np.int32),
                np.ascontiguousarray(self.axis, dtype=np.float64),
                np.ascontiguousarray(self.xtree, dtype=np.float64),
                np.ascontiguousarray(self.inertia, dtype=np.float64),
                np.ascontiguousarray(self.gravity, dtype=np.float64))

    def permuted(self, perm) -> "Robot":
        """Same robot with bodies renumbered: new body k is old body perm[k].
        perm must keep parents before children."""
        perm = np.asarray(perm)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(len(perm))
        par = np.array([-1 if self.parent[p] < 0 else inv[self.parent[p]] for p in perm],
                       dtype=np.int32)
        return Robot(self.name + "-perm", par, self.axis[perm].copy(), self.xtree[perm].copy(),
                     self.inertia[perm].copy(), self.gravity.copy(),
                     None if self.jtype is None else self.jtype[perm].copy())


_AX = {"x": (1.0, 0.0, 0.0), "y": (0.0, 1.0, 0.0), "z": (0.0, 0.0, 1.0)}


def _haar_rotation(s: Stream) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    w, x, y, z = s.normal(4)
    nrm = np.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / nrm, x / nrm, y / nrm, z / nrm
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _link_inertia(s: Stream, mlo: float, mhi: float) -> np.ndarray:
    """m ~ U[mlo, mhi]; COM uniform in the 0.1 m ball; I_c = R diag(l) R^T
    with l ~ U[0.005, 0.05] and R Haar-random."""
    m = s.uniform(mlo, mhi, 1)[0]
    while True:
        c = s.uniform(-0.1, 0.1, 3)
        if c @ c <= 0.01:
            break
    lam = s.uniform(0.005, 0.05, 3)
    R = _haar_rotation(s)
    Ic = R @ np.diag(lam) @ R.T
    return np.array([m, c[0], c[1], c[2], Ic[0, 0], Ic[1, 1], Ic[2, 2],
                     Ic[0, 1], Ic[0, 2], Ic[1, 2]])


def _xtree(E: np.ndarray, r) -> np.ndarray:
    return np.concatenate([np.asarray(E, dtype=np.float64).reshape(9),
                           np.asarray(r, dtype=np.float64)])


def _rpy_E(roll, pitch, yaw) -> np.ndarray:
    """E = R^T for the URDF rotation R = Rz(yaw) Ry(pitch) Rx(roll)."""
    cr, sr, cp, sp, cy, sy = (np.cos(roll), np.sin(roll), np.cos(pitch), np.sin(pitch),
                              np.cos(yaw), np.sin(yaw))
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    return (Rz @ Ry @ Rx).T


def _assemble(name, parent, axes, offsets, s_inertia, mlo, mhi, E=None) -> Robot:
    n = len(parent)
    axis = np.array([_AX[a] if isinstance(a, str) else a for a in axes], dtype=np.float64)
    xtree = np.stack([_xtree(np.eye(3) if E is None else E[i], offsets[i]) for i in range(n)])
    inertia = np.stack([_link_inertia(s_inertia, mlo, mhi) for _ in range(n)])
    return Robot(name, np.asarray(parent, dtype=np.int32), axis, xtree, inertia,
                 np.array([0.0, 0.0, -G_STD]))


def chain7(workload: int = 1) -> Robot:
    """7-DoF fixed-base serial chain: axes z,y,z,y,z,y,z; offsets (0,0,L),
    L ~ U[0.1, 0.4]; mass U[1,4] kg."""
    s_geo = Stream(stream_seed(workload, "chain7/geometry"))
    s_in = Stream(stream_seed(workload, "chain7/inertia"))
    n = 7
    L = s_geo.uniform(0.1, 0.4, n)
    offsets = [(0.0, 0.0, L[i]) for i in range(n)]
    return _assemble("chain7", [-1] + list(range(n - 1)), list("zyzyzyz"), offsets,
                     s_in, 1.0, 4.0)


def tree12(workload: int = 2) -> Robot:
    """12-DoF torso (fixed base) with four 3-joint legs, axes x,y,y, hips at
    (+-0.3, +-0.15, 0), knee/foot offsets (0,0,-L), L ~ U[0.1,0.4]; DFS order."""
    s_geo = Stream(stream_seed(workload, "tree12/geometry"))
    s_in = Stream(stream_seed(workload, "tree12/inertia"))
    parent, axes, offsets = [], [], []
    hips = [(0.3, 0.15, 0.0), (0.3, -0.15, 0.0), (-0.3, 0.15, 0.0), (-0.3, -0.15, 0.0)]
    for h in hips:
        b = len(parent)
        parent += [-1, b, b + 1]
        axes += ["x", "y", "y"]
        L = s_geo.uniform(0.1, 0.4, 2)
        offsets += [h, (0.0, 0.0, -L[0]), (0.0, 0.0, -L[1])]
    return _assemble("tree12", parent, axes, offsets, s_in, 1.0, 4.0)


def tree30(workload: int = 3) -> Robot:
    """30-DoF humanoid-like tree: 6-joint torso/neck chain from the base
    (axes z,y,x,z,y,x, offsets (0,0,L)); two 7-joint arms whose first parent is
    torso joint 0, attached at (0,+-0.2,0.3) (axes y,x,z,y,x,z,y, then offsets
    (0,0,-L)); two 5-joint legs from the base at (0,+-0.1,-0.1) (axes z,x,y,y,x,
    then offsets (0,0,-L)). Mass U[0.5, 8] kg. DFS numbering; longest path 8."""
    s_geo = Stream(stream_seed(workload, "tree30/geometry"))
    s_in = Stream(stream_seed(workload, "tree30/inertia"))
    parent, axes, offsets = [], [], []
    # torso / neck chain 0..5
    L = s_geo.uniform(0.1, 0.4, 6)
    for k, a in enumerate("zyxzyx"):
        parent.append(-1 if k == 0 else k - 1)
        axes.append(a)
        offsets.append((0.0, 0.0, L[k]))
    for side in (1.0, -1.0):                      # arms off torso joint 0
        L = s_geo.uniform(0.1, 0.4, 6)
        b = len(parent)
        for k, a in enumerate("yxzyxzy"):
            parent.append(0 if k == 0 else b + k - 1)
            axes.append(a)
            offsets.append((0.0, 0.2 * side, 0.3) if k == 0 else (0.0, 0.0, -L[k - 1]))
    for side in (1.0, -1.0):                      # legs off the base
        L = s_geo.uniform(0.1, 0.4, 4)
        b = len(parent)
        for k, a in enumerate("zxyyx"):
            parent.append(-1 if k == 0 else b + k - 1)
            axes.append(a)
            offsets.append((0.0, 0.1 * side, -0.1) if k == 0 else (0.0, 0.0, -L[k - 1]))
    return _assemble("tree30", parent, axes, offsets, s_in, 0.5, 8.0)


def random_tree(n: int, seed: int, general: bool = True, max_children: int = 3) -> Robot:
    """Small random tree for unit tests: parent[i] ~ U{-1..i-1} (base attaches
    allowed), general unit axes, E_T from rpy ~ U[-pi/4, pi/4], offsets in
    [-0.3, 0.3]^3. With general=False axes are x/y/z and E_T = I."""
    s = Stream(stream_seed(10_000 + n, f"random_tree/{seed}"))
    parent, kids = [], {}
    for i in range(n):
        while True:
            p = int(np.floor(s.unit(1)[0] * (i + 1))) - 1
            if kids.get(p, 0) < max_children:
                break
        kids[p] = kids.get(p, 0) + 1
        parent.append(p)
    if general:
        axes = []
        for _ in range(n):
            a = s.normal(3)
            axes.append(tuple(a / np.linalg.norm(a)))
        E = [_rpy_E(*s.uniform(-np.pi / 4, np.pi / 4, 3)) for _ in range(n)]
    else:
        axes = [("x", "y", "z")[int(s.unit(1)[0] * 3)] for _ in range(n)]
        E = None
    offsets = [tuple(s.uniform(-0.3, 0.3, 3)) for _ in range(n)]
    return _assemble(f"rand{n}-{seed}", parent, axes, offsets, s, 1.0, 4.0, E=E)


def random_mixed(n: int, seed: int, p_prismatic: float = 0.3, p_fixed: float = 0.2,
                 max_children: int = 3) -> Robot:
    """random_tree(n, seed) with a joint type drawn per body: fixed with
    probability p_fixed, prismatic with p_prismatic, else revolute (at least
    one joint moves)."""
    r = random_tree(n, seed, general=True, max_children=max_children)
    u = Stream(stream_seed(20_000 + n, f"random_mixed/{seed}")).unit(n)
    jt = np.where(u < p_fixed, FIXED, np.where(u < p_fixed + p_prismatic, PRISMATIC, REVOLUTE))
    jt = jt.astype(np.int32)
    if np.all(jt == FIXED):
        jt[-1] = REVOLUTE
    return dataclasses.replace(r, name=f"mixed{n}-{seed}", jtype=jt)


def chain7_tool(workload: int = 1) -> Robot:
    """The 7-DoF chain with a fixed tool body after joint 7 (offset (0,0,0.1),
    rotated by rpy (0.3,-0.2,0.5)) and a fixed sensor body between joints 3 and 4
    (joint 4 then hangs from the sensor): 9 bodies, 7 degrees of freedom."""
    base = chain7(workload)
    s_in = Stream(stream_seed(workload, "chain7_tool/inertia"))
    body = list(range(7))
    parent, axis, xtree, inertia, jt = [], [], [], [], []
    for i in body:
        if i == 3:                                  # sensor: fixed, hangs from body 2
            parent.append(2)
            axis.append((0.0, 0.0, 1.0))
            xtree.append(_xtree(np.eye(3), (0.0, 0.0, 0.05)))
            inertia.append(_link_inertia(s_in, 0.2, 0.5))
            jt.append(FIXED)
        parent.append(-1 if i == 0 else (len(parent) - 1))
        axis.append(tuple(base.axis[i]))
        xtree.append(base.xtree[i])
        inertia.append(base.inertia[i])
        jt.append(REVOLUTE)
    parent.append(len(parent) - 1)                  # tool
    axis.append((0.0, 0.0, 1.0))
    xtree.append(_xtree(_rpy_E(0.3, -0.2, 0.5), (0.0, 0.0, 0.1)))
    inertia.append(_link_inertia(s_in, 0.3, 1.0))
    jt.append(FIXED)
    return Robot("chain7_tool", np.asarray(parent, dtype=np.int32), np.asarray(axis, dtype=np.float64),
                 np.stack(xtree), np.stack(inertia), base.gravity.copy(), np.asarray(jt, dtype=np.int32))


def slider(m: float = 1.7, axis=(0.0, 0.0, 1.0), com=(0.05, -0.02, 0.1)) -> Robot:
    """Single prismatic joint at the base with unit axis `axis`, mass m with its
    COM at `com` and a small rotational inertia; gravity -z."""
    a = np.asarray(axis, dtype=np.float64)
    return Robot("slider", np.array([-1], dtype=np.int32), (a / np.linalg.norm(a))[None, :],
                 _xtree(np.eye(3), (0.1, 0.2, 0.3))[None, :],
                 np.array([[m, *com, 0.02, 0.03, 0.04, 0.001, 0.002, 0.003]]),
                 np.array([0.0, 0.0, -G_STD]), np.array([PRISMATIC], dtype=np.int32))


def cartpole(mc: float = 1.3, mp: float = 0.4, l: float = 0.6) -> Robot:
    """Cart on a prismatic joint along x (mass mc at its origin, no rotational
    inertia) carrying a pole on a revolute joint about y: a point mass mp at
    (0, 0, l) in the pole frame. Gravity -z."""
    return Robot("cartpole", np.array([-1, 0], dtype=np.int32),
                 np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]),
                 np.stack([_xtree(np.eye(3), (0.0, 0.0, 0.0))] * 2),
                 np.array([[mc, 0, 0, 0, 0, 0, 0, 0, 0, 0], [mp, 0, 0, l, 0, 0, 0, 0, 0, 0]], dtype=np.float64),
                 np.array([0.0, 0.0, -G_STD]), np.array([PRISMATIC, REVOLUTE], dtype=np.int32))


def pendulum(m: float = 2.0, l: float = 0.5) -> Robot:
    """Single pendulum: revolute axis x at the base, point mass m at c=(0,l,0),
    zero rotational inertia, gravity -z."""
    return Robot("pendulum", np.array([-1], dtype=np.int32), np.array([[1.0, 0.0, 0.0]]),
                 _xtree(np.eye(3), (0.0, 0.0, 0.0))[None, :],
                 np.array([[m, 0.0, l, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]]),
                 np.array([0.0, 0.0, -G_STD]))


def double_pendulum(m1=1.5, m2=1.0, l1=0.6, l2=0.4, lc1=0.3, lc2=0.2, i1=0.02, i2=0.01) -> Robot:
    """Planar acrobot in the y-z plane: two revolute joints about x, link k has
    mass m_k with COM at distance lc_k along the link (+y of its frame) and
    rotational inertia i_k about the x axis through its COM."""
    inertia = np.array([[m1, 0.0, lc1, 0.0, i1, i1, i1, 0.0, 0.0, 0.0],
                        [m2, 0.0, lc2, 0.0, i2, i2, i2, 0.0, 0.0, 0.0]])
    xtree = np.stack([_xtree(np.eye(3), (0.0, 0.0, 0.0)), _xtree(np.eye(3), (0.0, l1, 0.0))])
    return Robot("acrobot", np.array([-1, 0], dtype=np.int32),
                 np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]), xtree, inertia,
                 np.array([0.0, 0.0, -G_STD]))


WORKLOAD_ROBOTS = {"chain7": chain7, "tree12": tree12, "tree30": tree30}


def robot(name: str) -> Robot:
    return WORKLOAD_ROBOTS[name]()


def states(n: int, N: int, seed: int, dtype=np.float64):
    """Knot-point states, knot-major [N, n]: q ~ U[-pi, pi], qd ~ U[-1, 1],
    tau ~ U[-5, 5]."""
    s = Stream(stream_seed(seed, "states"))
    q = s.uniform(-np.pi, np.pi, (N, n))
    qd = s.uniform(-1.0, 1.0, (N, n))
    tau = s.uniform(-5.0, 5.0, (N, n))
    return q.astype(dtype), qd.astype(dtype), tau.astype(dtype)


def upstream(n: int, N: int, seed: int, dtype=np.float64):
    """Upstream gradients for the VJP, N(0, 1), [N, n]."""
    s = Stream(stream_seed(seed, "upstream"))
    return s.normal((N, n)).astype(dtype)


def workload_seed(workload: int, N: int) -> int:
    """State seed 1000*workload + N."""
    return 1000 * workload + N
