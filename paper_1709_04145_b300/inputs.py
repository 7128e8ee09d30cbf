"""Seeded synthetic workloads for the position-based articulated dynamics path.

This module only draws random numbers and assembles plain descriptions of
articulated bodies (topology, link lengths, masses, radii, initial poses and
torques). It holds none of the method's arithmetic: mass moments, kinematics,
objectives and solvers live on each side (the CUDA library and the CPU oracle)
separately, and both consume the same description.

Every generator takes a seed; ``numpy.random.default_rng(seed)`` (PCG64) is
the only source of randomness. The workloads mirror the paper's chain-swinging
benchmark (Section 6.1, Fig. SWING/OPTProf/CPUGPU) and its articulated
characters (Section 6.2): serial chains of rods or capsules, and branching
trees with hinge and ball joints, always with a fixed root.

Geometry conventions: a link's frame origin is its joint; the link body runs
along its local -z axis from 0 to -L; a child's joint sits at its parent's tip
unless an explicit attachment point is given; hinge axes are local +y.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HINGE = 0
BALL = 1
TRANSLATION = 2  # three prismatic coordinates along the joint frame's axes
ROD = 0
CAPSULE = 1

GRAVITY = np.array([0.0, 0.0, -9.81])


@dataclass
class BodySpec:
    """Plain description of ``count`` instances sharing one topology.

    Attributes (N links, B = count instances):
        parent:   (N,) int32, parent[l] < l, -1 = world.
        jtype:    (N,) int32, 0 hinge / 1 ball / 2 translation.
        axis:     (N, 3) hinge axes in the joint frame (ignored for balls).
        rest_rot: (N, 3, 3) rotation of the joint frame in the parent frame.
        attach:   (B, N, 3) joint position in the parent link frame.
        length:   (B, N) link lengths.
        mass:     (B, N) link masses.
        radius:   (B, N) capsule radii (0 for rods).
        shape:    (N,) int32, 0 rod / 1 capsule.
        gravity:  (3,).
    """

    parent: np.ndarray
    jtype: np.ndarray
    axis: np.ndarray
    rest_rot: np.ndarray
    attach: np.ndarray
    length: np.ndarray
    mass: np.ndarray
    radius: np.ndarray
    shape: np.ndarray
    gravity: np.ndarray = field(default_factory=lambda: GRAVITY.copy())
    name: str = ""

    @property
    def n_links(self) -> int:
        return int(self.parent.shape[0])

    @property
    def count(self) -> int:
        return int(self.length.shape[0])

    @property
    def n_dof(self) -> int:
        return int(np.sum(np.where(self.jtype == HINGE, 1, 3)))

    def dof_slices(self):
        off = 0
        out = []
        for t in self.jtype:
            k = 1 if t == HINGE else 3
            out.append(slice(off, off + k))
            off += k
        return out

    def select(self, idx) -> "BodySpec":
        """Sub-batch with the given instance indices."""
        idx = np.asarray(idx)
        return BodySpec(self.parent, self.jtype, self.axis, self.rest_rot,
                        self.attach[idx], self.length[idx], self.mass[idx],
                        self.radius[idx], self.shape, self.gravity, self.name)


def _chain_topology(n_links: int, joint: int):
    parent = np.arange(-1, n_links - 1, dtype=np.int32)
    jtype = np.full(n_links, joint, dtype=np.int32)
    axis = np.tile(np.array([0.0, 1.0, 0.0]), (n_links, 1))
    rest_rot = np.tile(np.eye(3), (n_links, 1, 1))
    return parent, jtype, axis, rest_rot


def _chain_attach(length: np.ndarray) -> np.ndarray:
    B, N = length.shape
    attach = np.zeros((B, N, 3))
    attach[:, 1:, 2] = -length[:, :-1]
    return attach


def rod_chain(count: int, n_links: int, length: float = 1.0, mass: float = 1.0,
              name: str = "") -> BodySpec:
    """Planar serial chain of uniform rods with hinge joints (paper Fig. SWING
    chains; the 3-link pendulum and the hinge chains of the scaling study)."""
    parent, jtype, axis, rest_rot = _chain_topology(n_links, HINGE)
    L = np.full((count, n_links), float(length))
    M = np.full((count, n_links), float(mass))
    return BodySpec(parent, jtype, axis, rest_rot, _chain_attach(L), L, M,
                    np.zeros((count, n_links)), np.full(n_links, ROD, np.int32),
                    name=name or f"rod_chain{n_links}")


def ball_chain(count: int, n_links: int, seed: int, radius: float = 0.05,
               name: str = "") -> BodySpec:
    """3D serial chains of capsules with ball joints; per-instance lengths
    U[0.5, 1.5] and masses lognormal(0, 0.3)."""
    rng = np.random.default_rng(seed)
    parent, jtype, axis, rest_rot = _chain_topology(n_links, BALL)
    L = rng.uniform(0.5, 1.5, size=(count, n_links))
    M = rng.lognormal(0.0, 0.3, size=(count, n_links))
    return BodySpec(parent, jtype, axis, rest_rot, _chain_attach(L), L, M,
                    np.full((count, n_links), radius),
                    np.full(n_links, CAPSULE, np.int32),
                    name=name or f"ball_chain{n_links}")


def humanoid(count: int, seed: int, name: str = "humanoid20") -> BodySpec:
    """Branching humanoid-like tree with 20 links and 34 DOFs: a torso on a
    ball joint at the world origin; four limbs (ball, hinge, hinge, hinge);
    a spine/head of (ball, ball, hinge) pointing up. Capsules (torso radius
    0.1, others 0.05), lengths U[0.25, 0.45], masses lognormal(0, 0.3)."""
    rng = np.random.default_rng(seed)
    parent, jtype, attach_pts, flips = [], [], [], []
    parent.append(-1); jtype.append(BALL); attach_pts.append(("fixed", (0, 0, 0))); flips.append(False)
    limb_attach = [(0.15, 0.0, "top"), (-0.15, 0.0, "top"), (0.1, 0.0, "bottom"), (-0.1, 0.0, "bottom")]
    for ax, ay, where in limb_attach:
        for k, jt in enumerate([BALL, HINGE, HINGE, HINGE]):
            if k == 0:
                parent.append(0)
                attach_pts.append((where, (ax, ay)))
            else:
                parent.append(len(parent) - 1)
                attach_pts.append(("tip", None))
            jtype.append(jt)
            flips.append(False)
    for k, jt in enumerate([BALL, BALL, HINGE]):
        if k == 0:
            parent.append(0)
            attach_pts.append(("top", (0.0, 0.0)))
            flips.append(True)
        else:
            parent.append(len(parent) - 1)
            attach_pts.append(("tip", None))
            flips.append(False)
        jtype.append(jt)
    N = len(parent)
    parent = np.array(parent, np.int32)
    jtype = np.array(jtype, np.int32)
    axis = np.tile(np.array([0.0, 1.0, 0.0]), (N, 1))
    rest_rot = np.tile(np.eye(3), (N, 1, 1))
    for l in range(N):
        if flips[l]:  # rotate by pi about x: the link points up
            rest_rot[l] = np.diag([1.0, -1.0, -1.0])
    L = rng.uniform(0.25, 0.45, size=(count, N))
    M = rng.lognormal(0.0, 0.3, size=(count, N))
    R = np.full((count, N), 0.05)
    R[:, 0] = 0.1
    attach = np.zeros((count, N, 3))
    for l in range(N):
        kind, val = attach_pts[l]
        if kind == "top":
            attach[:, l, 0], attach[:, l, 1] = val
        elif kind == "bottom":
            attach[:, l, 0], attach[:, l, 1] = val
            attach[:, l, 2] = -L[:, parent[l]]
        elif kind == "tip":
            attach[:, l, 2] = -L[:, parent[l]]
    return BodySpec(parent, jtype, axis, rest_rot, attach, L, M, R,
                    np.full(N, CAPSULE, np.int32), name=name)


def random_state(spec: BodySpec, seed: int, pose_scale: float = np.pi / 8,
                 vel_sigma: float = 0.5, hinge_scale: float | None = None):
    """Initial poses and velocities: exp-map / hinge coordinates uniform in
    [-pose_scale, pose_scale] (hinges use hinge_scale if given) and velocities
    N(0, vel_sigma^2). Returns (q0, qdot0), each (B, n)."""
    rng = np.random.default_rng(seed)
    B, n = spec.count, spec.n_dof
    q0 = rng.uniform(-pose_scale, pose_scale, size=(B, n))
    if hinge_scale is not None:
        for l, sl in enumerate(spec.dof_slices()):
            if spec.jtype[l] == HINGE:
                q0[:, sl] = rng.uniform(-hinge_scale, hinge_scale, size=(B, 1))
    qd0 = rng.normal(0.0, vel_sigma, size=(B, n)) if vel_sigma > 0 else np.zeros((B, n))
    return q0, qd0


def torques(spec: BodySpec, n_steps: int, seed: int, sigma: float = 0.1):
    """Per-step generalised joint torques, Gaussian N(0, sigma^2):
    (n_steps, B, n). sigma = 0 gives zeros."""
    if sigma == 0:
        return np.zeros((n_steps, spec.count, spec.n_dof))
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, size=(n_steps, spec.count, spec.n_dof))


def target_points(count: int, center: np.ndarray, seed: int, radius: float = 1.0):
    """Targets uniform in a ball of the given radius around center: (B, 3)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    rad = radius * rng.uniform(0, 1, size=(count, 1)) ** (1.0 / 3.0)
    return center + v * rad


# --------------------------------------------------------------------------
# The workloads (seed = 1000 * workload + stream)
# --------------------------------------------------------------------------

def pendulum3(seed_base: int = 1000):
    """3-link planar rod pendulum (L = 1, m = 1), q0 ~ U[-pi/4, pi/4], zero
    velocity, dt = 0.01, one stage (K = 2), L-BFGS history 5, tol 1e-10,
    200 steps."""
    spec = rod_chain(1, 3, name="pendulum3")
    rng = np.random.default_rng(seed_base + 1)
    q0 = rng.uniform(-np.pi / 4, np.pi / 4, size=(1, 3))
    return dict(spec=spec, q0=q0, qd0=np.zeros((1, 3)), dt=0.01, stages=1,
                history=5, tol=1e-10, n_steps=200, solver="lbfgs")


def ball_chains(count: int = 4096, n_links: int = 10, seed_base: int = 2000,
                n_steps: int = 100, radius: float = 0.15):
    """Batched 3D ball-joint capsule chains (capsule radius 0.15 m): dt =
    0.033, three stages (K = 4), L-BFGS history 8, 100 steps."""
    spec = ball_chain(count, n_links, seed_base + 1, radius=radius)
    q0, qd0 = random_state(spec, seed_base + 2)
    return dict(spec=spec, q0=q0, qd0=qd0, dt=0.033, stages=3, history=8,
                tol=1e-8, n_steps=n_steps, solver="lbfgs")


def uneven_batch(seed_base: int = 3000, n_steps: int = 10):
    """One launch over three buckets: 1024 humanoid trees (Newton), 1024
    chains of 50 hinge rods and 2048 chains of 5 hinge rods (L-BFGS m = 8);
    torques N(0, 0.1^2) per DOF per step, dt = 0.05, two stages."""
    specs = [humanoid(1024, seed_base + 1), rod_chain(1024, 50, name="rod_chain50"),
             rod_chain(2048, 5, name="rod_chain5")]
    states = [random_state(s, seed_base + 10 + k) for k, s in enumerate(specs)]
    taus = [torques(s, n_steps, seed_base + 20 + k, sigma=0.1) for k, s in enumerate(specs)]
    return dict(specs=specs, states=states, taus=taus, dt=0.05, stages=2, history=8,
                solvers=("newton", "lbfgs", "lbfgs"), n_steps=n_steps, tol=1e-8)


def swimmers(count: int = 4096, n_links: int = 4, seed_base: int = 6000, n_steps: int = 20,
             drag: float = 0.5):
    """Swimmer-like chains for the drag potential (Section 6.2): chains of
    n_links hinge rods (L = 1, m = 1) with a fixed root, immersed (no
    gravity: buoyancy cancels it), drag coefficient c per unit mass, dt = 0.05
    (the paper's swimmer step), one stage (Eq. EQ), L-BFGS history 8; poses
    U[-pi/4, pi/4], joint velocities N(0, 1)."""
    spec = rod_chain(count, n_links, name=f"swimmer{n_links}")
    spec.gravity = np.zeros(3)
    q0, qd0 = random_state(spec, seed_base + 1, pose_scale=np.pi / 4, vel_sigma=1.0)
    return dict(spec=spec, q0=q0, qd0=qd0, dt=0.05, stages=1, history=8, tol=1e-10,
                n_steps=n_steps, drag=drag, solver="lbfgs")


def free_chain(count: int, n_links: int, length: float = 1.0, mass: float = 1.0,
               name: str = "") -> BodySpec:
    """Chain of n_links uniform rods whose root moves freely: a massless
    link 0 with a translation joint at the world origin, then the first rod
    on a ball joint at the same point (the 6-DOF rigid root of Section 6.2's
    swimmer), then n_links - 1 rods on hinge joints (axis local +y). n_links
    + 1 links in the model, 6 + (n_links - 1) DOFs."""
    N = n_links + 1
    parent = np.arange(-1, N - 1, dtype=np.int32)
    jtype = np.array([TRANSLATION, BALL] + [HINGE] * (n_links - 1), np.int32)
    axis = np.tile(np.array([0.0, 1.0, 0.0]), (N, 1))
    rest_rot = np.tile(np.eye(3), (N, 1, 1))
    L = np.full((count, N), float(length))
    M = np.full((count, N), float(mass))
    L[:, 0] = 0.0
    M[:, 0] = 0.0
    return BodySpec(parent, jtype, axis, rest_rot, _chain_attach(L), L, M, np.zeros((count, N)),
                    np.full(N, ROD, np.int32), name=name or f"free_chain{n_links}")


def swimmers_free(count: int = 4096, seed_base: int = 6100, n_steps: int = 20, drag: float = 0.5):
    """Section 6.2's swimmer body: a 4-link chain with a free 6-DOF root and
    3 hinge joints (9 DOFs), immersed (no gravity), drag c per unit mass,
    dt = 0.05, one stage, L-BFGS history 8; root at the origin with random
    orientation U[-pi/4, pi/4] per exp-map coordinate, hinge angles
    U[-pi/4, pi/4], velocities N(0, 1) per coordinate."""
    spec = free_chain(count, 4, name="swimmer_free4")
    spec.gravity = np.zeros(3)
    q0, qd0 = random_state(spec, seed_base + 1, pose_scale=np.pi / 4, vel_sigma=1.0)
    q0[:, 0:3] = 0.0  # root position at the origin
    return dict(spec=spec, q0=q0, qd0=qd0, dt=0.05, stages=1, history=8, tol=1e-10,
                n_steps=n_steps, drag=drag, solver="lbfgs")


def spiders(count: int = 4096, seed_base: int = 6200, n_steps: int = 20):
    """Section 6.2's spider body on the ground: a torso rod (L = 0.4 m,
    m = 1 kg) on a free 6-DOF root and four legs, each an upper rod on a
    ball hip and a lower rod on a hinge knee (L = 0.3 m, m = 0.2 kg); the
    front pair is attached at the torso's joint, the rear pair at its tip.
    6 + 4 x (3 + 1) = 22 DOFs (the paper counts 18 for its spider). Contact
    points (Eq. FRI): the four feet and both torso ends against the ground
    z < 0, D1 = 2000, D2 = 100; drag 0.05 (settling); dt = 0.02, one stage,
    L-BFGS history 8. Initial state: torso horizontal 0.35 m above the
    ground, legs down with every angle perturbed U[-0.2, 0.2], velocities
    N(0, 0.3^2)."""
    rng = np.random.default_rng(seed_base + 1)
    # links: 0 carrier (translation), 1 torso (ball), then legs (hip ball, knee hinge) x 4
    parent = [-1, 0]
    jtype = [TRANSLATION, BALL]
    attach_z = [0.0, 0.0]
    length = [0.0, 0.4]
    mass = [0.0, 1.0]
    for k in range(4):
        parent += [1, len(parent)]
        jtype += [BALL, HINGE]
        attach_z += [0.0 if k < 2 else -0.4, -0.3]
        length += [0.3, 0.3]
        mass += [0.2, 0.2]
    N = len(parent)
    parent = np.array(parent, np.int32)
    jtype = np.array(jtype, np.int32)
    axis = np.tile(np.array([0.0, 1.0, 0.0]), (N, 1))
    rest_rot = np.tile(np.eye(3), (N, 1, 1))
    attach = np.zeros((count, N, 3))
    attach[:, :, 2] = np.array(attach_z)
    # front legs splay in +-y at the torso joint, rear legs at the tip
    for k in range(4):
        attach[:, 2 + 2 * k, 1] = 0.1 if k % 2 == 0 else -0.1
    L = np.tile(np.array(length), (count, 1))
    M = np.tile(np.array(mass), (count, 1))
    spec = BodySpec(parent, jtype, axis, rest_rot, attach, L, M, np.zeros((count, N)),
                    np.full(N, ROD, np.int32), name="spider")
    n = spec.n_dof
    q0 = np.zeros((count, n))
    sl = spec.dof_slices()
    q0[:, sl[0]] = [0.0, 0.0, 0.35]
    q0[:, sl[1]] = [0.0, np.pi / 2, 0.0]  # torso axis (local -z) along world -x
    for k in range(4):
        q0[:, sl[2 + 2 * k]] = [0.0, -np.pi / 2, 0.0]  # upper leg back to world -z
    q0[:, 3:] += rng.uniform(-0.2, 0.2, size=(count, n - 3))
    qd0 = rng.normal(0.0, 0.3, size=(count, n))
    feet = [3 + 2 * k for k in range(4)]
    contact = dict(link=feet + [1, 1], point=[[0, 0, -0.3]] * 4 + [[0, 0, 0.0], [0, 0, -0.4]],
                   z0=0.0, d1=2000.0, d2=100.0)
    return dict(spec=spec, q0=q0, qd0=qd0, contact=contact, drag=0.05, dt=0.02, stages=1,
                history=8, tol=1e-8, n_steps=n_steps, solver="lbfgs")


def humanoid_adjoint(count: int = 1024, seed_base: int = 4000, n_steps: int = 64):
    """Differentiation workload: humanoids, 64 steps at dt = 0.033 with two
    stages; loss = squared distance of the end effector (tip of limb 1's last
    link) to a target in a 1 m ball around its rest position at the final
    step; states checkpointed every 8 steps."""
    spec = humanoid(count, seed_base + 1)
    q0, qd0 = random_state(spec, seed_base + 2, pose_scale=np.pi / 8, vel_sigma=0.5)
    tau = torques(spec, n_steps, seed_base + 3, sigma=0.1)
    link = 4
    tip = np.zeros((count, 3))
    tip[:, 2] = -spec.length[:, link]
    return dict(spec=spec, q0=q0, qd0=qd0, tau=tau, dt=0.033, stages=2, n_steps=n_steps,
                checkpoint_every=8, ee_link=link, ee_point=tip, target_seed=seed_base + 4,
                tol=1e-8)


def scaling_chains(n_links: int, count: int = 256, seed_base: int = 5000, n_steps: int = 50):
    """Scaling study: hinge rod chains of n_links links, batch 256, dt = 0.1,
    four stages; L-BFGS (m = 8) against Newton on the same inputs."""
    spec = rod_chain(count, n_links, name=f"rod_chain{n_links}")
    q0, qd0 = random_state(spec, seed_base + n_links)
    return dict(spec=spec, q0=q0, qd0=qd0, dt=0.1, stages=4, history=8, n_steps=n_steps,
                tol=1e-8)
