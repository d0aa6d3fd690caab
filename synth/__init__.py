"""Seeded synthetic meshes and rigid poses.

These generators are the only code shared by the CUDA path's tests, the benchmark and the
FP64 oracle.  They hold none of the method's arithmetic (no bounding volumes, no
quantisation, no traversal, no triangle tests): they only draw meshes and poses from a
seeded NumPy PCG64 stream, computing in FP64 and rounding the results to FP32.

The paper measures on the OpenCollBench models (ds9 station, hand, robots; Sec. IV and
Fig. 2), which are not available here.  Displaced icospheres, a fractal heightfield,
random boxes and a DH serial arm stand in for them, at the sizes of the five workloads
generated by C1 to C5 below.

Pose convention: a pose is 12 FP32 numbers, the row-major 3x3 rotation R followed by the
translation t, and maps a point of mesh B into the frame of mesh A: x_A = R x_B + t.
"""
from __future__ import annotations

import functools
import math

import numpy as np

__all__ = [
    "icosphere", "heightfield", "ValueNoise2D", "box_mesh", "capsule", "shoemake_rotations",
    "poses_box", "poses_terrain", "dh_link_poses", "merge_meshes", "transform_mesh",
    "scene_diameter", "C1", "C2", "C3", "C4", "C5", "clutter", "arm_links", "self_pairs", "relative_poses",
]

_PHI = (1.0 + math.sqrt(5.0)) / 2.0
_ICO_V = np.array([
    (-1, _PHI, 0), (1, _PHI, 0), (-1, -_PHI, 0), (1, -_PHI, 0),
    (0, -1, _PHI), (0, 1, _PHI), (0, -1, -_PHI), (0, 1, -_PHI),
    (_PHI, 0, -1), (_PHI, 0, 1), (-_PHI, 0, -1), (-_PHI, 0, 1),
], dtype=np.float64)
_ICO_F = np.array([
    (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
    (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
    (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
    (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
], dtype=np.int64)


@functools.lru_cache(maxsize=8)
def _unit_icosphere_cached(level: int):
    v, f = _unit_icosphere_build(level)
    v.setflags(write=False)
    f.setflags(write=False)
    return v, f


def _unit_icosphere(level: int):
    """Unit icosphere: the icosahedron with each face split into 4, `level` times."""
    v, f = _unit_icosphere_cached(level)
    return v.copy(), f.copy()


def _unit_icosphere_build(level: int):
    v = list(_ICO_V / np.linalg.norm(_ICO_V, axis=1, keepdims=True))
    f = _ICO_F.copy()
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                p = v[a] + v[b]
                v.append(p / np.linalg.norm(p))
                idx = len(v) - 1
                cache[key] = idx
            return idx

        nf = np.empty((len(f) * 4, 3), dtype=np.int64)
        for i, (a, b, c) in enumerate(f):
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf[4 * i + 0] = (a, ab, ca)
            nf[4 * i + 1] = (b, bc, ab)
            nf[4 * i + 2] = (c, ca, bc)
            nf[4 * i + 3] = (ab, bc, ca)
        f = nf
    return np.asarray(v, dtype=np.float64), f


class _Noise3:
    """Smooth 3-D value noise on an integer lattice (hash values drawn from a seeded stream)."""

    def __init__(self, rng: np.random.Generator, size: int = 64):
        self.size = size
        self.table = rng.uniform(-1.0, 1.0, size=(size, size, size))

    def __call__(self, p: np.ndarray) -> np.ndarray:
        s = self.size
        i0 = np.floor(p).astype(np.int64)
        f = p - i0
        w = f * f * (3.0 - 2.0 * f)
        out = np.zeros(p.shape[0])
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    wt = ((w[:, 0] if dx else 1 - w[:, 0]) * (w[:, 1] if dy else 1 - w[:, 1])
                          * (w[:, 2] if dz else 1 - w[:, 2]))
                    out += wt * self.table[(i0[:, 0] + dx) % s, (i0[:, 1] + dy) % s, (i0[:, 2] + dz) % s]
        return out


def icosphere(level: int, radius: float = 1.0, disp: float = 0.15, seed: int = 0,
              fractal: bool = False, octaves: int = 4):
    """Radially displaced icosphere with 20 * 4**level triangles.

    With ``fractal=False`` every vertex is scaled by (1 + U(-disp, disp)) (an independent
    seeded draw per vertex).  With ``fractal=True`` the factor is 1 + disp * n(x), where n is
    a sum of ``octaves`` octaves of smooth value noise evaluated at the unit direction, so
    that fine meshes stay smooth.  Returns (verts float32 (V, 3), tris int32 (T, 3)).
    """
    v, f = _unit_icosphere(level)
    rng = np.random.default_rng(seed)
    if fractal:
        noise = _Noise3(rng)
        n = np.zeros(len(v))
        amp, tot = 1.0, 0.0
        for o in range(octaves):
            n += amp * noise(v * (2.0 * 2 ** o) + 17.0 * o + 32.0)
            tot += amp
            amp *= 0.5
        fac = 1.0 + disp * n / tot
    else:
        fac = 1.0 + rng.uniform(-disp, disp, size=len(v))
    verts = v * (radius * fac)[:, None]
    return verts.astype(np.float32), f.astype(np.int32)


class ValueNoise2D:
    """Fractal 2-D value noise over the square [-extent/2, extent/2]^2.

    Octave o uses a (base * 2**o + 1)^2 lattice of U(-1, 1) values drawn from the seeded
    stream, smoothstep-interpolated; octaves are summed with weights 0.5**o and normalised
    by the sum of the weights, then scaled by ``amplitude``.
    """

    def __init__(self, seed: int, extent: float = 4.0, amplitude: float = 0.4,
                 octaves: int = 4, base: int = 4):
        rng = np.random.default_rng(seed)
        self.extent, self.amplitude = float(extent), float(amplitude)
        self.freqs = [base * 2 ** o for o in range(octaves)]
        self.weights = [0.5 ** o for o in range(octaves)]
        self.tables = [rng.uniform(-1.0, 1.0, size=(f + 1, f + 1)) for f in self.freqs]

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        u = np.clip((x / self.extent) + 0.5, 0.0, 1.0)
        v = np.clip((y / self.extent) + 0.5, 0.0, 1.0)
        out = np.zeros(np.broadcast(u, v).shape)
        for f, wgt, tab in zip(self.freqs, self.weights, self.tables):
            gx, gy = u * f, v * f
            i = np.minimum(np.floor(gx).astype(np.int64), f - 1)
            j = np.minimum(np.floor(gy).astype(np.int64), f - 1)
            fx, fy = gx - i, gy - j
            sx, sy = fx * fx * (3 - 2 * fx), fy * fy * (3 - 2 * fy)
            a = tab[i, j] * (1 - sx) + tab[i + 1, j] * sx
            b = tab[i, j + 1] * (1 - sx) + tab[i + 1, j + 1] * sx
            out += wgt * (a * (1 - sy) + b * sy)
        return self.amplitude * out / sum(self.weights)


def heightfield(cells: int = 512, extent: float = 4.0, seed: int = 0, octaves: int = 4,
                amplitude_frac: float = 0.1):
    """Terrain: (cells+1)^2 vertices over [-extent/2, extent/2]^2, 2 * cells^2 triangles.

    Heights come from :class:`ValueNoise2D` with amplitude ``amplitude_frac * extent``.
    Returns (verts float32, tris int32, height function).
    """
    h = ValueNoise2D(seed, extent=extent, amplitude=amplitude_frac * extent, octaves=octaves)
    g = np.linspace(-extent / 2, extent / 2, cells + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    Z = h(X, Y)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(cells), np.arange(cells), indexing="ij")
    v00 = (i * (cells + 1) + j).ravel()
    v10 = v00 + (cells + 1)
    v01 = v00 + 1
    v11 = v10 + 1
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tris = np.empty((2 * len(v00), 3), dtype=np.int64)
    tris[0::2], tris[1::2] = t1, t2
    return verts.astype(np.float32), tris.astype(np.int32), h


def box_mesh(size=(1.0, 1.0, 1.0)):
    """Axis-aligned box centred at the origin: 8 vertices, 12 triangles."""
    sx, sy, sz = (0.5 * float(s) for s in size)
    v = np.array([[x, y, z] for x in (-sx, sx) for y in (-sy, sy) for z in (-sz, sz)])
    # vertex index = 4*ix + 2*iy + iz
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    f = []
    for a, b, c, d in quads:
        f.append((a, b, c))
        f.append((a, c, d))
    return v.astype(np.float32), np.array(f, dtype=np.int32)


def capsule(length: float, radius: float, n_tris_target: int, disp: float = 0.05, seed: int = 0):
    """Displaced capsule along +x from 0 to ``length``: a UV-sphere split at its equator with a
    cylinder inserted; the ring/segment counts are chosen so that the triangle count is close
    to ``n_tris_target``.  Returns (verts float32, tris int32)."""
    seg = max(8, int(round(math.sqrt(n_tris_target / 2.0))))
    rings = max(4, int(round(n_tris_target / (2.0 * seg))))
    rings += rings % 2
    rng = np.random.default_rng(seed)
    verts, ring_ids = [], []
    # rings of the UV sphere, with the two hemispheres pushed apart along x
    for r in range(rings + 1):
        th = math.pi * r / rings - math.pi / 2  # -pi/2 .. pi/2 along x
        x0 = radius * math.sin(th) + (length if th > 0 else 0.0)
        rr = radius * math.cos(th)
        ids = []
        count = 1 if r in (0, rings) else seg
        for s in range(count):
            ph = 2 * math.pi * s / seg
            verts.append((x0, rr * math.cos(ph), rr * math.sin(ph)))
            ids.append(len(verts) - 1)
        ring_ids.append(ids)
    tris = []
    for r in range(rings):
        a, b = ring_ids[r], ring_ids[r + 1]
        for s in range(seg):
            s1 = (s + 1) % seg
            if len(a) == 1:
                tris.append((a[0], b[s1], b[s]))
            elif len(b) == 1:
                tris.append((a[s], a[s1], b[0]))
            else:
                tris.append((a[s], a[s1], b[s1]))
                tris.append((a[s], b[s1], b[s]))
    v = np.asarray(verts, dtype=np.float64)
    axis = np.clip(v[:, 0], 0.0, length)
    rad = v - np.stack([axis, np.zeros_like(axis), np.zeros_like(axis)], axis=1)
    v = v + rad * rng.uniform(-disp, disp, size=(len(v), 1))
    return v.astype(np.float32), np.asarray(tris, dtype=np.int32)


def shoemake_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n rotation matrices uniform on SO(3), from Shoemake's uniform random unit quaternion
    (Graphics Gems III, 1992), computed in FP64.  Returns float64 (n, 3, 3)."""
    u1, u2, u3 = rng.uniform(size=(3, n))
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    x, y = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    z, w = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _pack(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    P = np.empty((len(R), 12), dtype=np.float64)
    P[:, :9] = R.reshape(len(R), 9)
    P[:, 9:] = t
    return P.astype(np.float32)


def poses_box(n: int, seed: int, lo=-2.0, hi=2.0) -> np.ndarray:
    """n poses: uniform rotation, translation uniform in [lo, hi]^3.  float32 (n, 12)."""
    rng = np.random.default_rng(seed)
    R = shoemake_rotations(rng, n)
    t = rng.uniform(lo, hi, size=(n, 3))
    return _pack(R, t)


def poses_terrain(n: int, seed: int, height_fn, extent: float = 4.0, radius: float = 1.0,
                  gap: float = 0.3) -> np.ndarray:
    """n poses of a sphere of ``radius`` over a terrain: (x, y) uniform over the footprint,
    centre z = H(x, y) + radius + U(0, gap), rotation uniform.  float32 (n, 12)."""
    rng = np.random.default_rng(seed)
    R = shoemake_rotations(rng, n)
    xy = rng.uniform(-extent / 2, extent / 2, size=(n, 2))
    z = height_fn(xy[:, 0], xy[:, 1]) + radius + rng.uniform(0.0, gap, size=n)
    return _pack(R, np.concatenate([xy, z[:, None]], axis=1))


def dh_link_poses(q: np.ndarray, a: float = 0.3, d: float = 0.0) -> np.ndarray:
    """Forward kinematics of a serial arm with standard DH parameters
    (Rz(theta) Tz(d) Tx(a) Rx(alpha)), alpha alternating +pi/2, -pi/2, base at the origin.
    q: (n, L) joint angles.  Returns float32 (n, L, 12): the pose of every link frame."""
    q = np.asarray(q, dtype=np.float64)
    n, L = q.shape
    T = np.tile(np.eye(4), (n, 1, 1))
    out = np.empty((n, L, 12), dtype=np.float64)
    for i in range(L):
        al = math.pi / 2 if i % 2 == 0 else -math.pi / 2
        ct, st = np.cos(q[:, i]), np.sin(q[:, i])
        ca, sa = math.cos(al), math.sin(al)
        A = np.zeros((n, 4, 4))
        A[:, 0, 0], A[:, 0, 1], A[:, 0, 2], A[:, 0, 3] = ct, -st * ca, st * sa, a * ct
        A[:, 1, 0], A[:, 1, 1], A[:, 1, 2], A[:, 1, 3] = st, ct * ca, -ct * sa, a * st
        A[:, 2, 1], A[:, 2, 2], A[:, 2, 3] = sa, ca, d
        A[:, 3, 3] = 1.0
        T = T @ A
        out[:, i, :9] = T[:, :3, :3].reshape(n, 9)
        out[:, i, 9:] = T[:, :3, 3]
    return out.astype(np.float32)


def transform_mesh(verts: np.ndarray, R: np.ndarray, t: np.ndarray) -> np.ndarray:
    return (np.asarray(verts, np.float64) @ np.asarray(R, np.float64).T + t).astype(np.float32)


def merge_meshes(parts):
    """Concatenate (verts, tris) meshes into one."""
    vs, ts, off = [], [], 0
    for v, t in parts:
        vs.append(np.asarray(v, np.float32))
        ts.append(np.asarray(t, np.int64) + off)
        off += len(v)
    return np.concatenate(vs), np.concatenate(ts).astype(np.int32)


def scene_diameter(va: np.ndarray, vb: np.ndarray) -> float:
    """D = diag(AABB(A)) + diag(AABB(B)), each in its own frame (independent of the pose)."""
    def diag(v):
        v = np.asarray(v, np.float64)
        return float(np.linalg.norm(v.max(0) - v.min(0)))
    return diag(va) + diag(vb)


# ---------------------------------------------------------------- named workloads
def C1(n_poses: int = 256):
    """Small case: two displaced level-3 icospheres (1,280 triangles each, radius 1,
    displacement U(-0.15, 0.15)); 18-DOP, branching 4, 16-bit deltas, 4 KB treelets;
    poses with uniform rotation and translation in [-2, 2]^3.  Mesh seeds 1001/1011, pose
    seed 2001."""
    A = icosphere(3, 1.0, 0.15, seed=1001)
    B = icosphere(3, 1.0, 0.15, seed=1011)
    P = poses_box(n_poses, seed=2001)
    return dict(A=A, B=B, poses=P, k=18, m=4, bits=16, treelet=4096)


def C2(n_poses: int = 10000, cells: int = 512):
    """Terrain against a sphere: A (static) = 512 x 512 fractal heightfield (524,288
    triangles, 4 x 4 footprint, amplitude 0.4); B (posed) = displaced level-5 icosphere
    (20,480 triangles).  24-DOP, branching 8, 8-bit deltas, 16 KB treelets.  Poses: (x, y)
    over the footprint, sphere centre 1 + U(0, 0.3) above the terrain height, uniform
    rotation.  Mesh seeds 1002/1012, pose seed 2002."""
    va, ta, H = heightfield(cells, 4.0, seed=1002)
    B = icosphere(5, 1.0, 0.15, seed=1012)
    P = poses_terrain(n_poses, seed=2002, height_fn=H)
    return dict(A=(va, ta), B=B, poses=P, k=24, m=8, bits=8, treelet=16384, height=H)


def clutter(n_boxes: int = 200, n_spheres: int = 200, seed: int = 1003, level: int = 4, half: float = 2.0):
    """Static clutter scene: boxes (side U(0.05, 0.4)) and displaced level-`level` spheres
    (radius U(0.05, 0.3)), placed uniformly in [-half, half]^3 with uniform rotations."""
    rng = np.random.default_rng(seed)
    parts = []
    for k in range(n_boxes):
        v, t = box_mesh(rng.uniform(0.05, 0.4, size=3))
        R = shoemake_rotations(rng, 1)[0]
        parts.append((transform_mesh(v, R, rng.uniform(-half, half, size=3)), t))
    for k in range(n_spheres):
        v, t = icosphere(level, rng.uniform(0.05, 0.3), 0.15, seed=seed * 7 + k)
        R = shoemake_rotations(rng, 1)[0]
        parts.append((transform_mesh(v, R, rng.uniform(-half, half, size=3)), t))
    return merge_meshes(parts)


def arm_links(a: float = 0.3, seed: int = 1013, sizes=(5120, 10000, 20480, 40000, 10000, 5120)):
    """The six link meshes of a serial arm, each in its own DH link frame, spanning x in
    [-a, 0] (from the previous joint to the frame origin): level-4 and level-5 displaced
    icospheres for the 5,120 and 20,480 sizes, displaced capsules for the others."""
    links = []
    for i, n in enumerate(sizes):
        if n in (5120, 20480):
            v, t = icosphere(4 if n == 5120 else 5, a / 2, 0.1, seed=seed + i)
            v = v + np.array([-a / 2, 0, 0], np.float32)
        else:
            v, t = capsule(a * 0.8, 0.05, n, disp=0.05, seed=seed + i)
            v = v + np.array([-a * 0.9, 0, 0], np.float32)
        links.append((v.astype(np.float32), t))
    return links


def C3(n_configs: int = 200000, n_boxes: int = 200, n_spheres: int = 200):
    """Motion-planning sweep: a 6-link DH arm (a = 0.3, alternating alpha = +-pi/2) against a
    static clutter scene of boxes and spheres in a 4 m cube; joint angles U[-pi, pi]^6.
    Returns the clutter (A), the links (B_i) and per-link poses (n, 6, 12).  Seeds 1003,
    1013 (meshes), 2003 (configurations)."""
    A = clutter(n_boxes, n_spheres)
    links = arm_links()
    rng = np.random.default_rng(2003)
    q = rng.uniform(-np.pi, np.pi, size=(n_configs, 6))
    return dict(A=A, links=links, link_poses=dh_link_poses(q), q=q, k=24, m=8, bits=8, treelet=16384)


def C5(n_poses: int = 1_000_000, n_spheres: int = 32, level: int = 7, probe_level: int = 6,
       half: float = 10.0):
    """Scale workload: an environment of `n_spheres` fractal-displaced level-`level` icospheres
    (radius U(0.5, 2), 4-octave noise, amplitude 0.15, uniform rotation) with centres uniform in
    [-half, half]^3 -- 32 level-7 spheres make 10,485,760 triangles -- probed by a displaced
    level-6 icosphere (81,920 triangles, radius 1) at poses with uniform rotation and translation
    uniform in the cube.  Seeds 1005 (environment), 1015 (probe), 2005 (poses)."""
    rng = np.random.default_rng(1005)
    parts = []
    for k in range(n_spheres):
        r = rng.uniform(0.5, 2.0)
        v, t = icosphere(level, r, 0.15, seed=1005 * 7 + k, fractal=True)
        R = shoemake_rotations(rng, 1)[0]
        parts.append((transform_mesh(v, R, rng.uniform(-half, half, size=3)), t))
    A = merge_meshes(parts)
    B = icosphere(probe_level, 1.0, 0.15, seed=1015)
    P = poses_box(n_poses, seed=2005, lo=-half, hi=half)
    return dict(A=A, B=B, poses=P, k=18, m=4, bits=8, treelet=16384)


def C4(rate: float, seconds: float, height_fn, seed: int = 2004, max_poses: int = 4096):
    """Serving workload: open-loop Poisson arrivals at ``rate`` requests/s for ``seconds``.
    Each request independently draws an environment (terrain or clutter), a robot (the 6-link
    arm, the level-5 sphere or the level-3 sphere), a kind (collision or distance, 1:1) and a
    size log-uniform in [1, max_poses] configurations.  Poses follow the workloads the models
    come from: spheres over the terrain as in the terrain workload (``height_fn``), spheres in
    the clutter uniform in its 4 m cube, the arm in the clutter at the origin with joint
    angles U[-pi, pi]^6, the arm on the terrain with its base 0.2 above a uniform point of the
    footprint.  Returns (gaps (s), requests [(env, robot, kind, poses)]); arm poses are
    (n, 6, 12), sphere poses (n, 12)."""
    rng = np.random.default_rng(seed)
    n_req = max(1, int(round(rate * seconds)))
    gaps = rng.exponential(1.0 / rate, size=n_req)
    reqs = []
    for _ in range(n_req):
        env = ("terrain", "clutter")[int(rng.integers(2))]
        robot = ("arm", "sphere5", "sphere3")[int(rng.integers(3))]
        kind = ("collide", "distance")[int(rng.integers(2))]
        n = min(max_poses, int(math.ceil(math.exp(rng.uniform(0.0, math.log(max_poses))))))
        sub = int(rng.integers(1 << 30))
        if robot == "arm":
            r2 = np.random.default_rng(sub)
            P = dh_link_poses(r2.uniform(-np.pi, np.pi, size=(n, 6)))
            if env == "terrain":
                xy = r2.uniform(-2.0, 2.0, size=(n, 2))
                base = np.concatenate([xy, (height_fn(xy[:, 0], xy[:, 1]) + 0.2)[:, None]], axis=1)
                P = P.copy()
                P[:, :, 9:] = (P[:, :, 9:].astype(np.float64) + base[:, None, :]).astype(np.float32)
        elif env == "terrain":
            P = poses_terrain(n, seed=sub, height_fn=height_fn)
        else:
            P = poses_box(n, seed=sub, lo=-2.0, hi=2.0)
        reqs.append((env, robot, kind, P))
    return gaps, reqs


def self_pairs(n_links: int = 6, gap: int = 2):
    """Link pairs checked for self-collision: (i, j) with j >= i + gap (neighbours share a
    joint and are allowed to touch)."""
    return [(i, j) for i in range(n_links) for j in range(i + gap, n_links)]


def relative_poses(link_poses: np.ndarray, i: int, j: int) -> np.ndarray:
    """Pose of link j in link i's frame for every configuration: T_i^-1 T_j, in FP64 and
    rounded to FP32.  link_poses: (n, L, 12) with x_world = R x_link + t."""
    P = np.asarray(link_poses, dtype=np.float64)
    Ri, ti = P[:, i, :9].reshape(-1, 3, 3), P[:, i, 9:]
    Rj, tj = P[:, j, :9].reshape(-1, 3, 3), P[:, j, 9:]
    RiT = np.transpose(Ri, (0, 2, 1))
    R = RiT @ Rj
    t = np.einsum("nab,nb->na", RiT, tj - ti)
    out = np.empty((len(P), 12))
    out[:, :9] = R.reshape(-1, 9)
    out[:, 9:] = t
    return out.astype(np.float32)
