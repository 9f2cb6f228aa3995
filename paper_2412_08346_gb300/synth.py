"""Seeded synthetic inputs for AS-ICP grasp matching.

This module produces the *inputs* of the method and nothing else: the gripper's
contact-surface cloud S for each preshape, the gripper's signed distance field
(SDF) sampled on a grid, and object clouds R.  It holds none of the method's
arithmetic (no rotation, matching, cost, collision or Stein step); both the
CUDA path and the FP64 oracle receive the arrays it returns, so they see
identical FP32 inputs.

The paper's gripper meshes (Franka, Barrett, KG3) and its scanned objects (KIT,
Google Scanned Objects, RealSense captures) are not available, so procedural
stand-ins with the paper's orders of magnitude are used (Section IV-A names the
inputs; Table I gives the point counts: objects of 1100-1900 points at 5 mm
voxels, a few preshapes, about 30 initialisations each):

* gripper: a palm plate of 8 x 8 x 1 cm (z in [-1, 0] cm) and three
  1.5 x 1.5 x 6 cm finger boxes centred at radius 3.25 cm, azimuth 0/120/240
  degrees, spanning z in [0, 6] cm.  Preshape p tilts every finger inward by
  ``tilt_deg[p]`` about the tangent axis through its base.  The approach axis
  is the gripper's +z.
* contact cloud S: points uniform by area on the inward-facing surfaces (the
  palm's top face outside the fingers and each finger's face toward the axis).
* SDF: the exact signed distance to the union of the four boxes, negated so it
  is positive inside the gripper (the paper's collision sign, Section IV-C),
  sampled on a node-centred grid over the cube [-10, 10]^3 cm, x fastest.
* objects: a box surface (the small case) or a shape drawn from box / cylinder /
  ellipsoid / superquadric with extents U[3, 15] cm and superquadric exponents
  U[0.3, 2]; single-view partial clouds keep points whose outward normal faces
  a random camera direction; Gaussian noise sigma = 1 mm.  Superquadric and
  ellipsoid points are sampled parametrically (not area-uniform).

All geometry is generated in float64 and rounded once to float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 241208346

PALM_HALF = np.array([0.04, 0.04, 0.005])       # palm plate half extents (m)
PALM_CENTER = np.array([0.0, 0.0, -0.005])
FINGER_HALF = np.array([0.0075, 0.0075, 0.03])  # radial, tangent, axial half extents
FINGER_RADIUS = 0.0325
FINGER_AZIMUTHS_DEG = (0.0, 120.0, 240.0)
SDF_HALF_WIDTH = 0.10                            # grid covers [-0.1, 0.1]^3 m
DEFAULT_TILTS_DEG = (0.0, 10.0, 20.0)   # 40 degrees would make the fingertips intersect


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# Gripper geometry (boxes as centre + orthonormal frame + half extents)
# --------------------------------------------------------------------------
@dataclass
class Box:
    center: np.ndarray   # (3,)
    axes: np.ndarray     # (3,3) rows are the box's local unit axes in gripper frame
    half: np.ndarray     # (3,) half extents along those axes


def gripper_boxes(tilt_deg: float) -> list[Box]:
    """Palm plate plus three finger boxes for one preshape."""
    boxes = [Box(PALM_CENTER.copy(), np.eye(3), PALM_HALF.copy())]
    b = math.radians(tilt_deg)
    for az in FINGER_AZIMUTHS_DEG:
        a = math.radians(az)
        u = np.array([math.cos(a), math.sin(a), 0.0])      # radial (outward)
        v = np.array([-math.sin(a), math.cos(a), 0.0])     # tangent
        z = np.array([0.0, 0.0, 1.0])
        base = FINGER_RADIUS * u                           # base centre on the palm top
        # tilt inward about the tangent axis: the finger axis leans toward -u
        axial = math.cos(b) * z - math.sin(b) * u
        radial = math.cos(b) * u + math.sin(b) * z
        center = base + FINGER_HALF[2] * axial
        boxes.append(Box(center, np.stack([radial, v, axial]), FINGER_HALF.copy()))
    return boxes


def box_sdf(points: np.ndarray, box: Box) -> np.ndarray:
    """Exact signed distance to an oriented box (negative inside)."""
    local = (points - box.center) @ box.axes.T
    q = np.abs(local) - box.half
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(np.max(q, axis=-1), 0.0)
    return outside + inside


def gripper_sdf_value(points: np.ndarray, tilt_deg: float) -> np.ndarray:
    """Gripper SDF at arbitrary points, positive inside the gripper."""
    d = np.min(np.stack([box_sdf(points, bx) for bx in gripper_boxes(tilt_deg)]), axis=0)
    return -d


def sdf_grid(tilt_deg: float, n: int):
    """Node-centred SDF grid over [-0.1, 0.1]^3 m, x fastest.

    Returns (grid float32 of shape (n, n, n) indexed [z, y, x], origin (3,), voxel).
    """
    voxel = 2.0 * SDF_HALF_WIDTH / (n - 1)
    origin = np.full(3, -SDF_HALF_WIDTH)
    ax = origin[0] + voxel * np.arange(n)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    pts = np.stack([xx, yy, zz], axis=-1).reshape(-1, 3)
    phi = gripper_sdf_value(pts, tilt_deg).reshape(n, n, n)
    return phi.astype(np.float32), origin.astype(np.float32), np.float32(voxel)


def _inside_any(points: np.ndarray, boxes: list[Box], margin: float = 0.0) -> np.ndarray:
    hit = np.zeros(len(points), dtype=bool)
    for bx in boxes:
        local = (points - bx.center) @ bx.axes.T
        hit |= np.all(np.abs(local) <= bx.half + margin, axis=-1)
    return hit


def gripper_contact_cloud(n: int, tilt_deg: float, seed: int) -> np.ndarray:
    """N points uniform by area on the inward-facing surfaces (float32, (n, 3))."""
    g = rng(seed)
    boxes = gripper_boxes(tilt_deg)
    fingers = boxes[1:]
    palm_area = (2 * PALM_HALF[0]) * (2 * PALM_HALF[1])
    face_area = (2 * FINGER_HALF[1]) * (2 * FINGER_HALF[2])
    total = palm_area + 3 * face_area
    n_f = int(round(n * face_area / total))
    n_palm = n - 3 * n_f
    # palm top face z = 0, rejecting the finger footprints
    palm = np.empty((0, 3))
    while len(palm) < n_palm:
        cand = np.column_stack([
            g.uniform(-PALM_HALF[0], PALM_HALF[0], 4 * n_palm),
            g.uniform(-PALM_HALF[1], PALM_HALF[1], 4 * n_palm),
            np.zeros(4 * n_palm)])
        probe = cand + np.array([0.0, 0.0, 1e-4])
        palm = np.concatenate([palm, cand[~_inside_any(probe, fingers)]])
    parts = [palm[:n_palm]]
    for bx in fingers:
        # the inward face of a tilted finger dips into the palm at its base: keep z >= 0
        face = np.empty((0, 3))
        while len(face) < n_f:
            tang = g.uniform(-bx.half[1], bx.half[1], 2 * n_f)
            axl = g.uniform(-bx.half[2], bx.half[2], 2 * n_f)
            pts = (bx.center - bx.half[0] * bx.axes[0]) + tang[:, None] * bx.axes[1] + axl[:, None] * bx.axes[2]
            face = np.concatenate([face, pts[pts[:, 2] >= 0.0]])
        parts.append(face[:n_f])
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------------------
# Objects
# --------------------------------------------------------------------------
def _spow(x, e):
    return np.sign(x) * np.abs(x) ** e


def _box_surface(g, half, n):
    areas = np.array([half[1] * half[2], half[0] * half[2], half[0] * half[1]]) * 4.0
    probs = np.repeat(areas, 2) / (2 * areas.sum())
    face = g.choice(6, size=n, p=probs)
    axis = face // 2
    sign = np.where(face % 2 == 0, 1.0, -1.0)
    pts = g.uniform(-1.0, 1.0, (n, 3)) * half
    pts[np.arange(n), axis] = sign * half[axis]
    nrm = np.zeros((n, 3))
    nrm[np.arange(n), axis] = sign
    return pts, nrm


def _cylinder_surface(g, half, n):
    a, b, h = half
    side = 2 * math.pi * math.sqrt((a * a + b * b) / 2) * 2 * h
    cap = math.pi * a * b
    kind = g.choice(3, size=n, p=np.array([side, cap, cap]) / (side + 2 * cap))
    th = g.uniform(-math.pi, math.pi, n)
    pts = np.empty((n, 3))
    nrm = np.empty((n, 3))
    s = kind == 0
    pts[s] = np.column_stack([a * np.cos(th[s]), b * np.sin(th[s]), g.uniform(-h, h, s.sum())])
    nrm[s] = np.column_stack([np.cos(th[s]) / a, np.sin(th[s]) / b, np.zeros(s.sum())])
    for k, zsgn in ((1, 1.0), (2, -1.0)):
        c = kind == k
        rr = np.sqrt(g.uniform(0.0, 1.0, c.sum()))
        pts[c] = np.column_stack([a * rr * np.cos(th[c]), b * rr * np.sin(th[c]), np.full(c.sum(), zsgn * h)])
        nrm[c] = np.column_stack([np.zeros(c.sum()), np.zeros(c.sum()), np.full(c.sum(), zsgn)])
    return pts, nrm


def _superquadric_surface(g, half, e1, e2, n):
    eta = g.uniform(-math.pi / 2, math.pi / 2, n)
    om = g.uniform(-math.pi, math.pi, n)
    ce, se, co, so = np.cos(eta), np.sin(eta), np.cos(om), np.sin(om)
    pts = np.column_stack([half[0] * _spow(ce, e1) * _spow(co, e2),
                           half[1] * _spow(ce, e1) * _spow(so, e2),
                           half[2] * _spow(se, e1)])
    nrm = np.column_stack([_spow(ce, 2 - e1) * _spow(co, 2 - e2) / half[0],
                           _spow(ce, 2 - e1) * _spow(so, 2 - e2) / half[1],
                           _spow(se, 2 - e1) / half[2]])
    return pts, nrm


@dataclass
class ObjectCloud:
    points: np.ndarray          # (M, 3) float32
    kind: str
    half_extents: np.ndarray
    camera: np.ndarray | None
    exponents: tuple = field(default_factory=tuple)


def box_object(m: int, seed: int, size=(0.06, 0.04, 0.10), noise=0.001) -> ObjectCloud:
    """Full box surface, uniform by area, centred at the origin, plus noise."""
    g = rng(seed)
    half = np.asarray(size, dtype=np.float64) / 2
    pts, _ = _box_surface(g, half, m)
    pts = pts + g.normal(0.0, noise, pts.shape)
    return ObjectCloud(pts.astype(np.float32), "box", half, None)


def partial_object(m: int, seed: int, kind: str | None = None, noise=0.001,
                   oversample: int = 8) -> ObjectCloud:
    """Single-view partial cloud of a seeded procedural shape, centred at the origin."""
    g = rng(seed)
    kinds = ("box", "cylinder", "ellipsoid", "superquadric")
    if kind is None:
        kind = kinds[int(g.integers(0, 4))]
    half = g.uniform(0.03, 0.15, 3) / 2
    exps = ()
    cam = g.normal(size=3)
    cam /= np.linalg.norm(cam)
    keep = np.empty((0, 3))
    while len(keep) < m:
        n = oversample * m
        if kind == "box":
            pts, nrm = _box_surface(g, half, n)
        elif kind == "cylinder":
            pts, nrm = _cylinder_surface(g, half, n)
        elif kind == "ellipsoid":
            pts, nrm = _superquadric_surface(g, half, 1.0, 1.0, n)
        else:
            if not exps:
                exps = (float(g.uniform(0.3, 2.0)), float(g.uniform(0.3, 2.0)))
            pts, nrm = _superquadric_surface(g, half, exps[0], exps[1], n)
        keep = np.concatenate([keep, pts[nrm @ cam > 0.0]])
    pts = keep[:m] + g.normal(0.0, noise, (m, 3))
    return ObjectCloud(pts.astype(np.float32), kind, half, cam, exps)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
@dataclass
class Preshape:
    S: np.ndarray           # (N, 3) float32 contact cloud
    sdf: np.ndarray         # (n, n, n) float32, [z, y, x]
    origin: np.ndarray      # (3,) float32
    voxel: np.float32
    tilt_deg: float


@dataclass
class Workload:
    name: str
    preshapes: list
    objects: list           # list[ObjectCloud]
    K: int
    k_max: int
    k_stein: int
    schedule: int           # 0 = cyclic annealing, 1 = linear
    g0: float = 0.1
    g1: float = 1.0
    C_cycles: float = 5.0
    p_exp: float = 2.0


def make_preshapes(P: int, N: int, grid: int, seed: int, tilts=DEFAULT_TILTS_DEG) -> list:
    out = []
    for p in range(P):
        sdf, origin, voxel = sdf_grid(tilts[p], grid)
        S = gripper_contact_cloud(N, tilts[p], seed + 17 * p)
        out.append(Preshape(S, sdf, origin, voxel, tilts[p]))
    return out


def k_stein_for(k_max: int) -> int:
    """15 SVGD : 25 SGD iterations (Table I) scaled to k_max."""
    return int(round(0.375 * k_max))


def small_box_case(seed: int = BASE_SEED + 1) -> Workload:
    """1 preshape, N=256, 32^3 SDF, 512-point noisy 6x4x10 cm box, K=32, 50 linear-annealed SVGD iterations."""
    pre = make_preshapes(1, 256, 32, seed)
    obj = box_object(512, seed + 1000)
    return Workload("box-P1-K32-N256-M512-sdf32-it50", pre, [obj], K=32, k_max=50, k_stein=50,
                    schedule=1, g0=0.1, g1=1.0)


def paper_scale_case(seed: int = BASE_SEED + 2, n_objects: int = 1) -> Workload:
    """3 preshapes x 256 particles, N=2048, M=8192 partial views, 64^3 SDF, 100 iterations."""
    pre = make_preshapes(3, 2048, 64, seed)
    objs = [partial_object(8192, seed + 1000 * (o + 1)) for o in range(n_objects)]
    return Workload("partial-P3-K256-N2048-M8192-sdf64-it100", pre, objs, K=256, k_max=100,
                    k_stein=k_stein_for(100), schedule=0)


def custom_case(P: int, K: int, N: int, M: int, grid: int, k_max: int, seed: int,
                kind: str | None = None, k_stein: int | None = None, schedule: int = 0) -> Workload:
    pre = make_preshapes(P, N, grid, seed)
    obj = partial_object(M, seed + 1000, kind=kind)
    return Workload(f"partial-P{P}-K{K}-N{N}-M{M}-sdf{grid}-it{k_max}", pre, [obj], K=K, k_max=k_max,
                    k_stein=k_stein_for(k_max) if k_stein is None else k_stein, schedule=schedule)


def batched_case(n_objects: int = 64, seed: int = BASE_SEED + 3, k_max: int = 100):
    """Many objects optimised together: point counts log-uniform in [1024, 32768], particles per
    (object, preshape) drawn from {128, 256, 512}; 3 preshapes, N=2048, 64^3 SDF.

    Returns (workload, K) with K an int32 array [n_objects, 3] of particle counts (object-major)."""
    g = rng(seed)
    Ms = np.exp(g.uniform(np.log(1024.0), np.log(32768.0), n_objects)).astype(int)
    K = g.choice(np.array([128, 256, 512], np.int32), size=(n_objects, 3)).astype(np.int32)
    pre = make_preshapes(3, 2048, 64, seed)
    objs = [partial_object(int(Ms[o]), seed + 1000 * (o + 1)) for o in range(n_objects)]
    w = Workload(f"batched-{n_objects}obj-M1k-32k-K128-512-P3-N2048-sdf64-it{k_max}", pre, objs, K=int(K.max()),
                 k_max=k_max, k_stein=k_stein_for(k_max), schedule=0)
    return w, K


def proposal_params(P: int, seed: int) -> np.ndarray:
    """Seeded initial weights of the proposal network (flat float32, layout of
    include/asicp_proposal.h): He-normal matrices, zero biases, the output layer scaled by 0.1."""
    g = rng(seed)
    dims = [(64, 3), (128, 64), (256, 128), (256, 256), (P * 16 * 10, 256)]
    parts = []
    for li, (o, i) in enumerate(dims):
        W = g.normal(0.0, np.sqrt(2.0 / i), (o, i)) * (0.1 if li == 4 else 1.0)
        parts += [W.ravel(), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


def table_points(n: int, obj_points: np.ndarray, seed: int, extent: float = 0.30, gap: float = 0.002,
                 noise: float = 0.001) -> np.ndarray:
    """A table under the object (the collision cloud C of Section IV-C holds the object and the
    table): n points uniform on a square of side `extent` centred under the object's centroid,
    `gap` below its lowest point, with normal noise."""
    g = rng(seed)
    c = obj_points.mean(0)
    z = obj_points[:, 2].min() - gap
    xy = c[:2] + g.uniform(-extent / 2, extent / 2, (n, 2))
    pts = np.concatenate([xy, np.full((n, 1), z)], 1) + g.normal(0.0, noise, (n, 3))
    return pts.astype(np.float32)


def minibatch_ramp(M: int, k_max: int, seed: int):
    """Mini-batches of the object cloud per iteration (Table I's ramp): m_k = ceil(M min(k, 2 k_max/3)
    / (2 k_max/3)), at least 1, drawn without replacement (seeded) and sorted ascending.
    Returns (offsets [k_max + 1], indices [offsets[-1]]) int32."""
    g = rng(seed)
    ramp = 2.0 * k_max / 3.0
    offs, idx = [0], []
    for k in range(k_max):
        m = int(np.ceil(M * min(k, ramp) / ramp)) if ramp > 0 else M
        m = min(max(m, 1), M)
        sel = np.sort(g.choice(M, m, replace=False)) if m < M else np.arange(M)
        idx.append(sel)
        offs.append(offs[-1] + m)
    return np.asarray(offs, np.int32), np.concatenate(idx).astype(np.int32)


def large_case(seed: int = BASE_SEED + 4, k_max: int = 10) -> Workload:
    """The largest single-object workload: 3 preshapes x 1024 particles, N=4096, M=65536 points of a
    superquadric partial view, 128^3 SDF."""
    pre = make_preshapes(3, 4096, 128, seed)
    obj = partial_object(65536, seed + 1000, kind="superquadric")
    return Workload(f"partial-P3-K1024-N4096-M65536-sdf128-it{k_max}", pre, [obj], K=1024, k_max=k_max,
                    k_stein=k_stein_for(k_max), schedule=0)
