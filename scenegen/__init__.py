"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module only *produces* inputs: triangle meshes, rigid instances placed in
the intersection frame of the paper's Sec. 3.1 (Table 1), and FMCW radar
profiles.  It holds none of the scattering / echo arithmetic of the method;
both the CUDA library and the oracle consume the arrays it returns.

Coordinate frame (Sec. 3.1): origin at the ground projection of the radar,
Y along the monitored lanes, Z up, X across the lanes.  The radar sits on a
6 m pole (Table 1).

Every generator is deterministic given its integer seed
(``numpy.random.default_rng(seed)``).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

C0 = 299_792_458.0          # speed of light in vacuum, m/s
F0_DEFAULT = 77.0e9         # chirp start frequency (pinned by Table 2's v_max)
T_IDLE = 10.0e-6            # chirp idle time: Table 2 pulse time - M/fs = 10 us

# Table 1 (Sec. 3.1)
RADAR_HEIGHT = 6.0
LANE_CENTERS_X = (2.0, 5.75, 9.5)
LANE_WIDTH = 3.75
INTERSECTION_WIDTH = 22.5


# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Mesh:
    """Triangle mesh in its local frame.  ``tris`` are counter-clockwise seen
    from outside, so (v1-v0)x(v2-v0) is the outward normal."""
    verts: np.ndarray              # (nv, 3) float64
    tris: np.ndarray               # (nf, 3) int32
    rho: np.ndarray                # (nf,)  float32 reflectivity (1 = PEC)
    name: str = "mesh"
    two_sided: bool = False        # facets scatter from both sides (open surfaces)

    def __post_init__(self):
        self.verts = np.ascontiguousarray(self.verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(self.tris, dtype=np.int32)
        self.rho = np.ascontiguousarray(self.rho, dtype=np.float32)
        assert self.verts.ndim == 2 and self.verts.shape[1] == 3
        assert self.tris.ndim == 2 and self.tris.shape[1] == 3
        assert self.rho.shape == (self.tris.shape[0],)

    @property
    def nf(self) -> int:
        return int(self.tris.shape[0])


@dataclasses.dataclass
class Instance:
    """A rigid placement of a mesh: x_world(t) = rot @ x_local + pos + vel*t."""
    mesh_id: int
    pos: np.ndarray                # (3,) float64
    rot: np.ndarray                # (3,3) float64, row-major
    vel: np.ndarray                # (3,) float64, m/s
    rho_scale: float = 1.0

    def __post_init__(self):
        self.pos = np.asarray(self.pos, dtype=np.float64).reshape(3)
        self.rot = np.asarray(self.rot, dtype=np.float64).reshape(3, 3)
        self.vel = np.asarray(self.vel, dtype=np.float64).reshape(3)


@dataclasses.dataclass
class Radar:
    """FMCW MIMO radar profile (Sec. 2.1, Sec. 3.2, Sec. 3.3).

    ``tx``/``rx`` are absolute antenna phase-centre positions (m).  Channel
    ``o = p*Q + q`` pairs TX ``p`` with RX ``q``; the ADC cube is stored
    [O][N][M] with the fast-time sample index contiguous.
    """
    f0: float                      # chirp start frequency, Hz
    slope: float                   # mu, Hz/s
    fs: float                      # ADC sampling rate, samples/s
    Tc: float                      # chirp repetition period, s
    M: int                         # samples per chirp
    N: int                         # chirps per frame
    tx: np.ndarray                 # (P,3)
    rx: np.ndarray                 # (Q,3)
    intra_chirp_motion: bool = True
    tdm: bool = False              # time-division MIMO: TX p sends chirp n at (n P + p) Tc
    delay_ref: bool = False        # reference-point delay form (one tau(t) per instance)
    far_field: bool = False        # plane waves from each instance origin, at its ranges
    grazing_eps: float = 1e-6      # |cos| below which a facet grazes its antenna
    double_bounce: bool = False    # add the two-facet (double-bounce) paths

    def __post_init__(self):
        self.tx = np.ascontiguousarray(np.asarray(self.tx, np.float64).reshape(-1, 3))
        self.rx = np.ascontiguousarray(np.asarray(self.rx, np.float64).reshape(-1, 3))

    @property
    def P(self) -> int:
        return int(self.tx.shape[0])

    @property
    def Q(self) -> int:
        return int(self.rx.shape[0])

    @property
    def O(self) -> int:
        return self.P * self.Q

    @property
    def antennas(self) -> np.ndarray:
        """TX antennas first (index p), then RX antennas (index P+q)."""
        return np.concatenate([self.tx, self.rx], axis=0)


@dataclasses.dataclass
class Scene:
    meshes: List[Mesh]
    instances: List[Instance]
    radar: Radar
    t0: float = 0.0
    name: str = "scene"

    @property
    def nf(self) -> int:
        return int(sum(self.meshes[i.mesh_id].nf for i in self.instances))


# --------------------------------------------------------------------------
# radar profiles (Table 2 arithmetic: B = mu*M/fs, T_c = M/fs + idle)
# --------------------------------------------------------------------------
def radar_profile(M: int, fs: float = 5.12e6, slope: float = 12.5e12,
                  f0: float = F0_DEFAULT) -> dict:
    """Derived FMCW quantities for an M-sample chirp (Sec. 4.1, Table 2).

    Returns sweep bandwidth B = mu*M/fs, chirp period T_c = M/fs + 10 us,
    range resolution c/(2B), maximum unambiguous speed lambda_c/(4 T_c) with
    lambda_c taken at the band centre, and maximum IF range fs*c/(2 mu).
    """
    B = slope * M / fs
    Tc = M / fs + T_IDLE
    lam_c = C0 / (f0 + 0.5 * B)
    return dict(M=M, B=B, Tc=Tc, range_res=C0 / (2.0 * B),
                v_max=lam_c / (4.0 * Tc), r_max=fs * C0 / (2.0 * slope),
                lam_c=lam_c)


def ula(n: int, spacing: float, centre: Sequence[float]) -> np.ndarray:
    """n elements along X, centred on ``centre``."""
    c = np.asarray(centre, np.float64)
    off = (np.arange(n) - 0.5 * (n - 1)) * spacing
    out = np.tile(c, (n, 1))
    out[:, 0] += off
    return out


def make_radar(M: int, N: int, P: int, Q: int, fs: float, slope: float,
               tx_spacing_wl: float, rx_spacing_wl: float = 0.5,
               centre=(0.0, 0.0, RADAR_HEIGHT), f0: float = F0_DEFAULT,
               intra_chirp_motion: bool = True, tdm: bool = False,
               delay_ref: bool = False) -> Radar:
    lam0 = C0 / f0
    prof = radar_profile(M, fs, slope, f0)
    return Radar(f0=f0, slope=slope, fs=fs, Tc=prof["Tc"], M=M, N=N,
                 tx=ula(P, tx_spacing_wl * lam0, centre),
                 rx=ula(Q, rx_spacing_wl * lam0, centre),
                 intra_chirp_motion=intra_chirp_motion, tdm=tdm, delay_ref=delay_ref)


# --------------------------------------------------------------------------
# primitive meshes
# --------------------------------------------------------------------------
def plate(size_x: float = 1.0, size_z: float = 1.0, n: int = 10,
          rho: float = 1.0) -> Mesh:
    """Flat rectangular plate in the local X-Z plane, outward normal -Y,
    meshed as an n x n grid of squares, 2 triangles each (2 n^2 facets)."""
    xs = (np.arange(n + 1) / n - 0.5) * size_x
    zs = (np.arange(n + 1) / n - 0.5) * size_z
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    verts = np.stack([X.ravel(), np.zeros(X.size), Z.ravel()], axis=1)
    idx = lambda i, j: i * (n + 1) + j
    tris = []
    for i in range(n):
        for j in range(n):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            # CCW seen from -Y: (a, b, c) and (a, c, d) give normal -Y
            tris.append((a, b, c))
            tris.append((a, c, d))
    tris = np.asarray(tris, np.int32)
    return Mesh(verts, tris, np.full(len(tris), rho, np.float32), "plate")


def ground(size: float = 100.0, n: int = 158, centre=(0.0, 50.0),
           rho: float = 1.0) -> Mesh:
    """Flat ground grid at z = 0, outward normal +Z, 2 n^2 facets."""
    xs = centre[0] + (np.arange(n + 1) / n - 0.5) * size
    ys = centre[1] + (np.arange(n + 1) / n - 0.5) * size
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a = (i * (n + 1) + j).ravel()
    b = ((i + 1) * (n + 1) + j).ravel()
    c = ((i + 1) * (n + 1) + j + 1).ravel()
    d = (i * (n + 1) + j + 1).ravel()
    t1 = np.stack([a, b, c], 1)     # CCW seen from +Z
    t2 = np.stack([a, c, d], 1)
    tris = np.stack([t1, t2], 1).reshape(-1, 3).astype(np.int32)
    return Mesh(verts, tris, np.full(len(tris), rho, np.float32), "ground")


def dihedral(size: float = 0.1, n: int = 2, rho: float = 1.0) -> Mesh:
    """Right-angle dihedral corner: two square plates of side ``size`` on the
    local Z axis (the fold), plate A in the X-Z plane (x in [0, size],
    normal +Y) and plate B in the Y-Z plane (y in [0, size], normal +X), z in
    [-size/2, size/2]; each an n x n grid of squares, 2 triangles each.  The
    opening faces the local direction (1, 1, 0)."""
    s = (np.arange(n + 1) / n) * size
    z = (np.arange(n + 1) / n - 0.5) * size
    verts, tris = [], []
    for plate_id in range(2):
        base = len(verts)
        for i in range(n + 1):
            for j in range(n + 1):
                verts.append((s[i], 0.0, z[j]) if plate_id == 0 else (0.0, s[i], z[j]))
        want = np.array([0.0, 1.0, 0.0]) if plate_id == 0 else np.array([1.0, 0.0, 0.0])
        idx = lambda i, j: base + i * (n + 1) + j
        for i in range(n):
            for j in range(n):
                for t in ((idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)),
                          (idx(i, j), idx(i + 1, j + 1), idx(i, j + 1))):
                    v0, v1, v2 = (np.array(verts[k]) for k in t)
                    if np.dot(np.cross(v1 - v0, v2 - v0), want) < 0:
                        t = (t[0], t[2], t[1])
                    tris.append(t)
    tris = np.asarray(tris, np.int32)
    return Mesh(np.asarray(verts), tris, np.full(len(tris), rho, np.float32), "dihedral")


def icosphere(radius: float = 0.1, subdiv: int = 5, rho: float = 1.0) -> Mesh:
    """Geodesic sphere: icosahedron subdivided ``subdiv`` times (20*4^s faces)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.asarray(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdiv):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.asarray(verts) * radius
    F = np.asarray(faces, np.int32)
    return Mesh(V, F, np.full(len(F), rho, np.float32), "icosphere")


def rounded_box(hx: float, hy: float, hz: float, r: float, ntri: int,
                centre=(0.0, 0.0, 0.0)) -> tuple:
    """Closed rounded box: the Minkowski sum of a box with half extents
    (hx-r, hy-r, hz-r) and a sphere of radius r, meshed with ~``ntri``
    near-uniform triangles.  Each face of the outer box gets a regular grid;
    every grid point q is moved to core(q) + r (q - core(q))/|q - core(q)|,
    core(q) = clamp(q, -(h-r), h-r).  Vertices shared along the cube edges
    are merged, and every triangle is wound CCW seen from outside."""
    h = np.array([hx, hy, hz], np.float64)
    area = 8.0 * (hx * hy + hy * hz + hx * hz)
    edge = math.sqrt(2.0 * area / max(ntri, 12))
    ns = [max(2, int(round(2.0 * e / edge))) for e in h]
    verts, tris = [], []
    off = 0
    for ax in range(3):
        u_ax, v_ax = [a for a in range(3) if a != ax]
        nu, nv = ns[u_ax], ns[v_ax]
        uu = np.linspace(-h[u_ax], h[u_ax], nu + 1)
        vv = np.linspace(-h[v_ax], h[v_ax], nv + 1)
        U, V = np.meshgrid(uu, vv, indexing="ij")
        for sgn in (-1.0, 1.0):
            q = np.zeros((U.size, 3))
            q[:, ax] = sgn * h[ax]
            q[:, u_ax] = U.ravel()
            q[:, v_ax] = V.ravel()
            verts.append(q)
            i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
            a = (i * (nv + 1) + j).ravel() + off
            b = ((i + 1) * (nv + 1) + j).ravel() + off
            c = ((i + 1) * (nv + 1) + j + 1).ravel() + off
            d = (i * (nv + 1) + j + 1).ravel() + off
            tris.append(np.stack([a, b, c], 1))
            tris.append(np.stack([a, c, d], 1))
            off += q.shape[0]
    Q = np.concatenate(verts, 0)
    T = np.concatenate(tris, 0)
    key = np.round(Q / (1e-9 * max(h))).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    Q = Q[first]
    T = inv.reshape(-1)[T]
    core = np.clip(Q, -(h - r), h - r)
    d = Q - core
    dn = np.linalg.norm(d, axis=1)
    P = core + r * d / np.where(dn > 0, dn, 1.0)[:, None]
    v = P[T]
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    flip = (n * v.mean(1)).sum(1) < 0.0            # convex: outward = away from centre
    T[flip] = T[flip][:, ::-1]
    return P + np.asarray(centre, np.float64), T.astype(np.int32)


def merge(meshes: Sequence[tuple], rho: float = 1.0, name: str = "mesh") -> Mesh:
    verts, tris, off = [], [], 0
    for v, t in meshes:
        verts.append(v)
        tris.append(t + off)
        off += v.shape[0]
    V = np.concatenate(verts, 0)
    F = np.concatenate(tris, 0).astype(np.int32)
    return Mesh(V, F, np.full(F.shape[0], rho, np.float32), name)


# vehicle classes: (length along local Y, width, height) nominal extents, m,
# and nominal triangle budgets (car 20k, SUV 40k, bus 120k, truck 200k)
VEHICLE_CLASSES = {
    "car":   dict(ext=(4.5, 1.8, 1.5), ntri=20_000),
    "suv":   dict(ext=(4.9, 2.0, 1.8), ntri=40_000),
    "bus":   dict(ext=(12.0, 2.55, 3.2), ntri=120_000),
    "truck": dict(ext=(16.0, 2.5, 4.0), ntri=200_000),
}


def vehicle(cls: str = "car", seed: int = 0, ntri: Optional[int] = None,
            jitter: float = 0.05, rho: float = 1.0) -> Mesh:
    """Procedural rounded-box vehicle: a rounded-box lower body plus a
    rounded-box cabin, extents jittered by +-``jitter`` (seeded); the
    triangle budget is split in proportion to surface area.

    Local frame: length along Y (front at +Y), ground contact plane z = 0,
    ground clearance 0.25 m.  Two closed shells; the part of the cabin
    inside the body is shadowed by the body during visibility.
    """
    spec = VEHICLE_CLASSES[cls]
    rng = np.random.default_rng(seed)
    L, W, H = (e * (1.0 + jitter * rng.uniform(-1.0, 1.0)) for e in spec["ext"])
    ntri = spec["ntri"] if ntri is None else int(ntri)
    clear = 0.25
    body_h = 0.6 * (H - clear)
    cab_h = (H - clear) - body_h + 0.1        # cabin overlaps body by 0.1 m
    cab_l = 0.53 * L if cls in ("car", "suv") else 0.25 * L
    cab_w = 0.9 * W
    cab_y = -0.05 * L if cls in ("car", "suv") else 0.35 * L
    a_body = 2 * (L * W + L * body_h + W * body_h)
    a_cab = 2 * (cab_l * cab_w + cab_l * cab_h + cab_w * cab_h)
    n_body = int(ntri * a_body / (a_body + a_cab))
    n_cab = ntri - n_body
    vb, tb = rounded_box(0.5 * W, 0.5 * L, 0.5 * body_h, 0.2 * body_h, n_body,
                         centre=(0.0, 0.0, clear + 0.5 * body_h))
    vc, tc = rounded_box(0.5 * cab_w, 0.5 * cab_l, 0.5 * cab_h, 0.25 * cab_h, n_cab,
                         centre=(0.0, cab_y, clear + body_h - 0.1 + 0.5 * cab_h))
    return merge([(vb, tb), (vc, tc)], rho, name=f"{cls}{seed}")


def rot_z(angle: float) -> np.ndarray:
    c, s = math.cos(angle), math.sin(angle)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


# --------------------------------------------------------------------------
# workload scenes
# --------------------------------------------------------------------------
def plate_scene(range_m: float = 20.0, n: int = 10, M: int = 128, N: int = 64,
                slope: float = 30e12, fs: float = 5.12e6) -> Scene:
    """Static 1 m x 1 m PEC plate (2 n^2 triangles), broadside at ``range_m``
    on the Y axis; radar at the origin, 1 TX x 4 RX ULA at lambda0/2."""
    radar = make_radar(M, N, 1, 4, fs, slope, tx_spacing_wl=2.0,
                       centre=(0.0, 0.0, 0.0))
    inst = Instance(0, pos=(0.0, range_m, 0.0), rot=np.eye(3), vel=(0.0, 0.0, 0.0))
    return Scene([plate(1.0, 1.0, n)], [inst], radar, name="plate")


def car_scene(seed: int = 2, ntri: int = 20_000, slant: float = 30.0,
              speed: float = 10.0, M: int = 256, N: int = 128,
              P: int = 3, Q: int = 4, lane: int = 0) -> Scene:
    """One procedural sedan in a Table 1 lane at slant range ``slant`` from
    the pole-mounted radar, moving ``speed`` m/s along the line of sight
    toward it.  3 TX at 2 lambda0 x 4 RX at lambda0/2 (12 virtual channels)."""
    radar = make_radar(M, N, P, Q, 5.12e6, 12.5e12, tx_spacing_wl=2.0)
    x = LANE_CENTERS_X[lane]
    y = math.sqrt(slant ** 2 - x ** 2 - RADAR_HEIGHT ** 2)
    pos = np.array([x, y, 0.0])
    los = pos - np.array([0.0, 0.0, RADAR_HEIGHT])
    vel = -speed * los / np.linalg.norm(los)
    mesh = vehicle("car", seed, ntri)
    inst = Instance(0, pos=pos, rot=rot_z(math.pi), vel=vel)   # front faces -Y
    return Scene([mesh], [inst], radar, name="car")


def intersection_scene(seed: int = 3, n_vehicles: int = 12, M: int = 512,
                       N: int = 256, P: int = 12, Q: int = 16,
                       ground_n: int = 158, tri_scale: float = 1.0) -> Scene:
    """Table 1 intersection: ``n_vehicles`` vehicles drawn uniformly from the
    four classes, lanes X in {2, 5.75, 9.5}, Y in [10, 80] m without overlap,
    v_y in [-15, 15] m/s, on a 100 m x 100 m ground grid.  12 TX at 8 lambda0
    x 16 RX at lambda0/2 (192 virtual channels), fs = 10.24 Msps."""
    rng = np.random.default_rng(seed)
    radar = make_radar(M, N, P, Q, 10.24e6, 12.5e12, tx_spacing_wl=8.0)
    meshes = [ground(100.0, ground_n, centre=(0.0, 50.0))]
    insts = [Instance(0, pos=(0.0, 0.0, 0.0), rot=np.eye(3), vel=(0.0, 0.0, 0.0))]
    classes = list(VEHICLE_CLASSES)
    occupied = {0: [], 1: [], 2: []}
    for k in range(n_vehicles):
        placed = False
        for _ in range(200):                 # redraw the class if it won't fit
            cls = classes[int(rng.integers(0, 4))]
            L = VEHICLE_CLASSES[cls]["ext"][0] * 1.06
            for _ in range(200):
                lane = int(rng.integers(0, 3))
                y = float(rng.uniform(10.0 + 0.5 * L, 80.0 - 0.5 * L))
                if all(abs(y - y2) > 0.5 * (L + L2) + 1.0
                       for y2, L2 in occupied[lane]):
                    placed = True
                    break
            if placed:
                break
        if not placed:
            raise RuntimeError("could not place vehicle without overlap")
        occupied[lane].append((y, L))
        vy = float(rng.uniform(-15.0, 15.0))
        ntri = int(VEHICLE_CLASSES[cls]["ntri"] * tri_scale)
        meshes.append(vehicle(cls, seed * 1000 + k, ntri))
        heading = 0.0 if vy > 0 else math.pi
        insts.append(Instance(len(meshes) - 1, pos=(LANE_CENTERS_X[lane], y, 0.0),
                              rot=rot_z(heading), vel=(0.0, vy, 0.0)))
    return Scene(meshes, insts, radar, name="intersection")


def batch_scene(index: int, base_seed: int = 4, M: int = 256, N: int = 128,
                tri_min: int = 5_000, tri_max: int = 200_000) -> Scene:
    """One scene of the batched RDM dataset: 1-8 vehicles from the four
    classes in Table 1 lanes (25-40 m, approaching at 0.5-10 m/s, the sweep
    of Sec. 3.4), with one uniform level-of-detail factor so the scene's
    total triangle count lies in [tri_min, tri_max].  Radar as the car scene."""
    rng = np.random.default_rng(base_seed * 1_000_003 + index)
    radar = make_radar(M, N, 3, 4, 5.12e6, 12.5e12, tx_spacing_wl=2.0)
    nveh = int(rng.integers(1, 9))
    classes = list(VEHICLE_CLASSES)
    picks = [classes[int(rng.integers(0, 4))] for _ in range(nveh)]
    nominal = sum(VEHICLE_CLASSES[c]["ntri"] for c in picks)
    total = float(rng.uniform(tri_min, tri_max))
    lod = total / nominal
    meshes, insts = [], []
    occupied = {0: [], 1: [], 2: []}
    for k, cls in enumerate(picks):
        L = VEHICLE_CLASSES[cls]["ext"][0] * 1.06
        for _ in range(1000):
            lane = int(rng.integers(0, 3))
            y = float(rng.uniform(25.0, 40.0 + 8.0 * L))
            if all(abs(y - y2) > 0.5 * (L + L2) + 1.0 for y2, L2 in occupied[lane]):
                break
        occupied[lane].append((y, L))
        v = float(rng.uniform(0.5, 10.0))
        ntri = max(200, int(VEHICLE_CLASSES[cls]["ntri"] * lod))
        meshes.append(vehicle(cls, base_seed * 7919 + index * 17 + k, ntri))
        insts.append(Instance(len(meshes) - 1, pos=(LANE_CENTERS_X[lane], y, 0.0),
                              rot=rot_z(math.pi), vel=(0.0, -v, 0.0)))
    return Scene(meshes, insts, radar, name=f"batch{index}")


def point_target_scene(range_m: float, speed: float = 0.0, M: int = 128,
                       N: int = 64, slope: float = 30e12, fs: float = 5.12e6,
                       edge: float = 0.4e-3, P: int = 1, Q: int = 1) -> Scene:
    """A tiny square plate (two triangles of edge ``edge`` << lambda) facing
    a radar at the origin from ``range_m`` on the Y axis, moving ``speed``
    m/s away along +Y (negative = approaching)."""
    radar = make_radar(M, N, P, Q, fs, slope, tx_spacing_wl=2.0,
                       centre=(0.0, 0.0, 0.0))
    inst = Instance(0, pos=(0.0, range_m, 0.0), rot=np.eye(3),
                    vel=(0.0, speed, 0.0))
    return Scene([plate(edge, edge, 1)], [inst], radar, name="point")


def small_car_scene(seed: int = 11, ntri: int = 1500, M: int = 128, N: int = 6,
                    P: int = 2, Q: int = 2, slant: float = 18.0,
                    speed: float = 12.0) -> Scene:
    """Reduced car scene sized for full-cube oracle parity: a coarse sedan,
    2 TX x 2 RX, a few chirps.  Same geometry recipe as ``car_scene``."""
    s = car_scene(seed=seed, ntri=ntri, slant=slant, speed=speed, M=M, N=N, P=P, Q=Q)
    s.name = "small_car"
    return s


def dihedral_scene(range_m: float = 6.0, size: float = 0.1, n: int = 2, alpha_deg: float = 45.0,
                   M: int = 128, N: int = 4, P: int = 1, Q: int = 2, speed: float = 0.0,
                   slope: float = 30e12, fs: float = 5.12e6) -> Scene:
    """A dihedral corner (``dihedral``) on the Y axis at ``range_m`` from a
    radar at the origin, its fold vertical, turned so that the radar sees
    plate A at ``alpha_deg`` (45: along the opening's bisector); moving
    ``speed`` m/s along +Y.  Double-bounce paths on."""
    radar = make_radar(M, N, P, Q, fs, slope, tx_spacing_wl=2.0, centre=(0.0, 0.0, 0.0))
    radar.double_bounce = True
    # the local direction (cos a, sin a, 0) toward the radar: world -Y
    a = math.radians(alpha_deg)
    inst = Instance(0, pos=(0.0, range_m, 0.0), rot=rot_z(-math.pi / 2 - a),
                    vel=(0.0, speed, 0.0))
    return Scene([dihedral(size, n)], [inst], radar, name="dihedral")


def car_ground_scene(seed: int = 11, ntri: int = 1500, ground_size: float = 12.0,
                     ground_n: int = 6, M: int = 128, N: int = 4, P: int = 2, Q: int = 2,
                     slant: float = 18.0, speed: float = 12.0) -> Scene:
    """``small_car_scene``'s sedan on a static ground patch (``ground_size``
    square, ``ground_n`` x ``ground_n`` squares) centred under it, double-
    bounce paths on: the car-ground and ground-car multipath of a road."""
    s = small_car_scene(seed=seed, ntri=ntri, M=M, N=N, P=P, Q=Q, slant=slant, speed=speed)
    pos = s.instances[0].pos
    s.meshes.append(ground(ground_size, ground_n, centre=(pos[0], pos[1])))
    s.instances.append(Instance(1, pos=(0.0, 0.0, 0.0), rot=np.eye(3), vel=(0.0, 0.0, 0.0)))
    s.radar.double_bounce = True
    s.name = "car_ground"
    return s


def sedan_ground_scene(ground_size: float = 20.0, ground_n: int = 40, **kw) -> Scene:
    """``car_scene``'s moving sedan (20k triangles, 3 TX x 4 RX, 128 chirps x
    256 samples) on a static ground patch (``ground_size`` square of
    ``ground_n`` x ``ground_n`` squares, 0.5 m cells by default) centred
    under it, double-bounce paths on."""
    s = car_scene(**kw)
    pos = s.instances[0].pos
    s.meshes.append(ground(ground_size, ground_n, centre=(pos[0], pos[1])))
    s.instances.append(Instance(1, pos=(0.0, 0.0, 0.0), rot=np.eye(3), vel=(0.0, 0.0, 0.0)))
    s.radar.double_bounce = True
    s.name = "sedan_ground"
    return s


def flatten(scene: Scene):
    """Concatenate instance meshes: per-facet local vertex triples, instance
    index, reflectivity, and the per-instance pose arrays.  Pure bookkeeping."""
    lv, inst_idx, rho = [], [], []
    for i, ins in enumerate(scene.instances):
        m = scene.meshes[ins.mesh_id]
        lv.append(m.verts[m.tris].reshape(-1, 9))
        inst_idx.append(np.full(m.nf, i, np.int32))
        rho.append(m.rho * np.float32(ins.rho_scale))
    pos = np.stack([i.pos for i in scene.instances])
    rot = np.stack([i.rot.reshape(9) for i in scene.instances])
    vel = np.stack([i.vel for i in scene.instances])
    return (np.ascontiguousarray(np.concatenate(lv, 0)),
            np.concatenate(inst_idx), np.concatenate(rho).astype(np.float32),
            np.ascontiguousarray(pos), np.ascontiguousarray(rot),
            np.ascontiguousarray(vel))


def facet_two_sided(scene: Scene) -> np.ndarray:
    """Per-facet two-sided flags (uint8) in the order of ``flatten``."""
    return np.concatenate([np.full(scene.meshes[i.mesh_id].nf, int(scene.meshes[i.mesh_id].two_sided),
                                   np.uint8) for i in scene.instances])
