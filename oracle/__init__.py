"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` import this package.  The product
path (``paper_2208_10939_gb300``) never imports, links or runs it.

The heavy loops are plain C (``oracle.c``, built with gcc, OpenMP,
``-ffp-contract=off``); the range-Doppler step uses ``numpy.fft`` as a
library primitive.  Every function cites the passage of arXiv 2208.10939 it
follows; readings of silent or garbled passages are stated where used.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute force, invariants, the paper's Table 2).  The absolute
PO amplitude convention for curved, non-spherical bodies is pinned only by
construction (the same definition), see the flat-plate and sphere pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BACK, LIT, GRAZE, OCCL, LIT_REV = 0, 1, 2, 3, 4
EPS_FACE = 1e-6      # |cos| below which a facet is grazing its antenna
EPS_B = 1e-9         # barycentric margin of the segment/triangle test
EPS_T = 1e-9         # segment-parameter margin of the segment/triangle test
C0 = 299_792_458.0


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Radar(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("slope", ctypes.c_double),
                ("fs", ctypes.c_double), ("Tc", ctypes.c_double),
                ("M", ctypes.c_int), ("N", ctypes.c_int), ("P", ctypes.c_int),
                ("Q", ctypes.c_int), ("intra_chirp_motion", ctypes.c_int),
                ("tdm", ctypes.c_int), ("delay_ref", ctypes.c_int), ("far_field", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.orc_world_vertices.argtypes = [P, P, ctypes.c_int64, P, P, P,
                                               ctypes.c_double, P]
            lib.orc_visibility.argtypes = [P, ctypes.c_int64, P, ctypes.c_int, P, P,
                                           ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, P]
            lib.orc_facet_integral.argtypes = [P, P, P, P]
            lib.orc_visibility_bvh.argtypes = [P, ctypes.c_int64, P, ctypes.c_int, P, P,
                                               ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, P]
            lib.orc_visibility_pairs.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int64, P, P,
                                                 ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, P]
            lib.orc_rcs_farfield.argtypes = [P, ctypes.c_int64, P, P, P, P, P,
                                             ctypes.c_int, P]
            lib.orc_adc_full.argtypes = [P, P, P, P, P, P, ctypes.c_int64, P, P,
                                         ctypes.POINTER(_Radar), P]
            lib.orc_adc_entries.argtypes = [P, P, P, P, P, P, ctypes.c_int64, P, P,
                                            ctypes.POINTER(_Radar), P,
                                            ctypes.c_int64, P]
            lib.orc_bounce2_facets.argtypes = [P, P, P, P, ctypes.c_int64, P, ctypes.c_int, P,
                                               ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int64, P, P, P, P, P]
            lib.orc_bounce2_facets.restype = ctypes.c_int64
            lib.orc_rcs_farfield_bounce2.argtypes = [P, ctypes.c_int64, P, P, P, P, P,
                                                     ctypes.c_int, P]
            lib.orc_adc_bounce2_entries.argtypes = [P, P, P, P, P, ctypes.c_int64, P, P, P,
                                                    ctypes.c_int64, P, P,
                                                    ctypes.POINTER(_Radar), P,
                                                    ctypes.c_int64, P]
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
def flatten(scene):
    """Per-facet local vertices, instance index, reflectivity and pose arrays."""
    import scenegen
    return scenegen.flatten(scene)


def world_facets(scene, t: float):
    """World vertex triples (F x 9) of every facet at absolute time ``t``
    (rigid translation, Sec. 3.2 / Eq. 12), and per-facet velocity (F x 3)."""
    lv, inst, rho, pos, rot, vel = flatten(scene)
    out = np.empty_like(lv)
    _load().orc_world_vertices(_p(lv), _p(inst), lv.shape[0], _p(pos), _p(rot),
                               _p(vel), float(t), _p(out))
    fvel = np.ascontiguousarray(vel[inst])
    return out, fvel, rho


def reference_points(scene, t: float) -> np.ndarray:
    """Per-facet reference point of the facet's instance (the instance
    origin, Eq. 12's target position) at absolute time t: pos + vel t."""
    _, inst, _, pos, _, vel = flatten(scene)
    ref = pos + vel * float(t)
    return np.ascontiguousarray(ref[inst])


def _opt(a, dtype, shape):
    return None if a is None else np.ascontiguousarray(a, dtype).reshape(shape)


def _ptr_or_none(a):
    return None if a is None else _p(a)


def visibility(tri: np.ndarray, antennas: np.ndarray, eps_face: float = EPS_FACE,
               eps_b: float = EPS_B, eps_t: float = EPS_T, fref=None,
               two_sided=None) -> np.ndarray:
    """Facet state per antenna, A x F uint8 (BACK, LIT, GRAZE, OCCL,
    LIT_REV), by brute force over all occluders (BART single bounce, Sec.
    2.2).  ``fref`` (F x 3): far-field segments toward p_a + (c_k - fref_k);
    ``two_sided`` (F,): facets lit from either side."""
    tri = np.ascontiguousarray(tri, np.float64)
    ant = np.ascontiguousarray(antennas, np.float64).reshape(-1, 3)
    F, A = tri.shape[0], ant.shape[0]
    fr, ts = _opt(fref, np.float64, (F, 3)), _opt(two_sided, np.uint8, (F,))
    st = np.empty((A, F), np.uint8)
    _load().orc_visibility(_p(tri), F, _p(ant), A, _ptr_or_none(fr), _ptr_or_none(ts),
                           eps_face, eps_b, eps_t, _p(st))
    return st


def visibility_bvh(tri: np.ndarray, antennas: np.ndarray, eps_face: float = EPS_FACE,
                   eps_b: float = EPS_B, eps_t: float = EPS_T, fref=None,
                   two_sided=None) -> np.ndarray:
    """``visibility`` through the oracle's own top-down median-split BVH
    (for scenes too large for all pairs); same definition, same states."""
    tri = np.ascontiguousarray(tri, np.float64)
    ant = np.ascontiguousarray(antennas, np.float64).reshape(-1, 3)
    F, A = tri.shape[0], ant.shape[0]
    fr, ts = _opt(fref, np.float64, (F, 3)), _opt(two_sided, np.uint8, (F,))
    st = np.empty((A, F), np.uint8)
    _load().orc_visibility_bvh(_p(tri), F, _p(ant), A, _ptr_or_none(fr), _ptr_or_none(ts),
                               eps_face, eps_b, eps_t, _p(st))
    return st


def visibility_pairs(tri: np.ndarray, antennas: np.ndarray, pairs: np.ndarray,
                     eps_face: float = EPS_FACE, eps_b: float = EPS_B,
                     eps_t: float = EPS_T, fref=None, two_sided=None) -> np.ndarray:
    """States of selected (antenna, facet) pairs (E x 2), brute force over
    all occluders: the per-pair definition of ``visibility`` (Sec. 2.2)."""
    tri = np.ascontiguousarray(tri, np.float64)
    ant = np.ascontiguousarray(antennas, np.float64).reshape(-1, 3)
    pr = np.ascontiguousarray(pairs, np.int64).reshape(-1, 2)
    F = tri.shape[0]
    fr, ts = _opt(fref, np.float64, (F, 3)), _opt(two_sided, np.uint8, (F,))
    st = np.empty(pr.shape[0], np.uint8)
    _load().orc_visibility_pairs(_p(tri), F, _p(ant), _p(pr), pr.shape[0], _ptr_or_none(fr),
                                 _ptr_or_none(ts), eps_face, eps_b, eps_t, _p(st))
    return st


def facet_integral(tri9: np.ndarray, w: np.ndarray) -> complex:
    """J(w) = integral of exp(j w.(r - c)) over one flat triangle."""
    tri9 = np.ascontiguousarray(tri9, np.float64).reshape(9)
    w = np.ascontiguousarray(w, np.float64).reshape(3)
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_facet_integral(_p(tri9), _p(w), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def rcs_farfield(tri: np.ndarray, rho: np.ndarray, t_hat, r_hat, freqs,
                 two_sided=None) -> np.ndarray:
    """Far-field PO RCS sigma(f) (m^2) of a mesh for plane-wave directions
    (toward TX ``t_hat`` and RX ``r_hat``), Sec. 2.2 / Eq. 7's sigma."""
    tri = np.ascontiguousarray(tri, np.float64)
    rho = np.ascontiguousarray(rho, np.float32)
    t = np.ascontiguousarray(t_hat, np.float64) / np.linalg.norm(t_hat)
    r = np.ascontiguousarray(r_hat, np.float64) / np.linalg.norm(r_hat)
    f = np.ascontiguousarray(np.atleast_1d(freqs), np.float64)
    ts = _opt(two_sided, np.uint8, (tri.shape[0],))
    out = np.empty(f.shape[0], np.float64)
    _load().orc_rcs_farfield(_p(tri), tri.shape[0], _p(rho), _ptr_or_none(ts), _p(t), _p(r),
                             _p(f), f.shape[0], _p(out))
    return out


def bounce2_facets(tri: np.ndarray, fvel: np.ndarray, rho: np.ndarray, antennas: np.ndarray,
                   P: int, state: np.ndarray, two_sided=None, eps_face: float = EPS_FACE,
                   eps_b: float = EPS_B, eps_t: float = EPS_T) -> dict:
    """Virtual facets of the double-bounce paths (Sec. 2.2: forward and
    backward rays connected through two facets; the geometric-optics /
    physical-optics reading stated in ``oracle.c``) of transmitters 0..P-1:
    ``pab`` (V x 4: TX p, first facet a, second facet b, side of b), ``tri``
    (V x 9 frame-start vertices), ``src`` (V x 3 image source), ``usrc``
    (V x 3 its velocity), ``w`` (V: -rho_a rho_b), in (p, a, b, fan) order."""
    tri = np.ascontiguousarray(tri, np.float64)
    F = tri.shape[0]
    fv = np.ascontiguousarray(fvel, np.float64).reshape(F, 3)
    rh = np.ascontiguousarray(rho, np.float32).reshape(F)
    ant = np.ascontiguousarray(antennas, np.float64).reshape(-1, 3)
    st = np.ascontiguousarray(state, np.uint8)
    ts = _opt(two_sided, np.uint8, (F,))
    cap = 1024
    while True:
        out = dict(pab=np.zeros((cap, 4), np.int32), tri=np.zeros((cap, 9)),
                   src=np.zeros((cap, 3)), usrc=np.zeros((cap, 3)), w=np.zeros(cap))
        n = int(_load().orc_bounce2_facets(
            _p(tri), _p(fv), _p(rh), _ptr_or_none(ts), F, _p(ant), int(P), _p(st),
            eps_face, eps_b, eps_t, cap, _p(out["pab"]), _p(out["tri"]), _p(out["src"]),
            _p(out["usrc"]), _p(out["w"])))
        if n <= cap:
            return {k: np.ascontiguousarray(v[:n]) for k, v in out.items()}
        cap = n


def rcs_farfield_bounce2(tri: np.ndarray, rho: np.ndarray, t_hat, r_hat, freqs,
                         two_sided=None) -> np.ndarray:
    """Far-field double-bounce PO cross-section sigma(f) (m^2) of a mesh
    for plane-wave directions (toward TX ``t_hat`` and RX ``r_hat``): the
    double-bounce reading of Sec. 2.2 with the image source at infinity, no
    occlusion test."""
    tri = np.ascontiguousarray(tri, np.float64)
    rho = np.ascontiguousarray(rho, np.float32)
    t = np.ascontiguousarray(t_hat, np.float64) / np.linalg.norm(t_hat)
    r = np.ascontiguousarray(r_hat, np.float64) / np.linalg.norm(r_hat)
    f = np.ascontiguousarray(np.atleast_1d(freqs), np.float64)
    ts = _opt(two_sided, np.uint8, (tri.shape[0],))
    out = np.empty(f.shape[0], np.float64)
    _load().orc_rcs_farfield_bounce2(_p(tri), tri.shape[0], _p(rho), _ptr_or_none(ts), _p(t),
                                     _p(r), _p(f), f.shape[0], _p(out))
    return out


def _radar_struct(radar) -> _Radar:
    ff, dr = bool(getattr(radar, "far_field", False)), bool(getattr(radar, "delay_ref", False))
    if ff and dr:
        raise ValueError("far_field and delay_ref are exclusive delay forms")
    return _Radar(radar.f0, radar.slope, radar.fs, radar.Tc, radar.M, radar.N,
                  radar.P, radar.Q, int(bool(radar.intra_chirp_motion)),
                  int(bool(getattr(radar, "tdm", False))), int(dr), int(ff))


class Frame:
    """Frame-start geometry and visibility of a scene (computed once): brute
    force over all occluders up to 60k facets, the oracle's own BVH above."""

    def __init__(self, scene, state: np.ndarray | None = None, bvh: bool | None = None):
        import scenegen
        self.scene = scene
        self.radar = scene.radar
        self._rs = _radar_struct(self.radar)
        self.tri0, self.fvel, self.rho = world_facets(scene, scene.t0)
        self.fref = reference_points(scene, scene.t0)
        ts = scenegen.facet_two_sided(scene)
        self.two_sided = ts if ts.any() else None
        if state is None:
            use_bvh = self.tri0.shape[0] > 60_000 if bvh is None else bvh
            fn = visibility_bvh if use_bvh else visibility
            state = fn(self.tri0, self.radar.antennas,
                       eps_face=float(getattr(self.radar, "grazing_eps", EPS_FACE)),
                       fref=self.fref if self._rs.far_field else None,
                       two_sided=self.two_sided)
        self.state = state
        self.double_bounce = bool(getattr(self.radar, "double_bounce", False))
        if self.double_bounce and (self._rs.far_field or self._rs.delay_ref):
            raise ValueError("double bounce takes the per-facet delay form")
        self.bounce = None
        if self.double_bounce:
            self.bounce = bounce2_facets(self.tri0, self.fvel, self.rho, self.radar.antennas,
                                         self.radar.P, self.state, two_sided=self.two_sided,
                                         eps_face=float(getattr(self.radar, "grazing_eps",
                                                                EPS_FACE)))

    def bounce_entries(self, entries: np.ndarray) -> np.ndarray:
        """Double-bounce part of selected ADC entries (E x 3: o, n, m)."""
        r = self.radar
        e = np.ascontiguousarray(entries, np.int32).reshape(-1, 3)
        out = np.zeros(e.shape[0], np.complex128)
        b = self.bounce
        if b is None or b["w"].shape[0] == 0:
            return out
        _load().orc_adc_bounce2_entries(
            _p(b["pab"]), _p(b["tri"]), _p(b["src"]), _p(b["usrc"]), _p(b["w"]),
            b["w"].shape[0], _p(self.fvel), _ptr_or_none(self.two_sided), _p(self.state),
            self.tri0.shape[0], _p(r.tx), _p(r.rx), ctypes.byref(self._rs), _p(e), e.shape[0],
            _p(out))
        return out

    def _args(self):
        r = self.radar
        return (_p(self.tri0), _p(self.fvel), _p(self.rho), _p(self.fref),
                _ptr_or_none(self.two_sided), _p(self.state), self.tri0.shape[0], _p(r.tx),
                _p(r.rx), ctypes.byref(self._rs))

    def adc_full(self) -> np.ndarray:
        """ADC cube [O][N][M] complex128 (Eqs. 7, 9-13)."""
        r = self.radar
        out = np.empty((r.O, r.N, r.M), np.complex128)
        _load().orc_adc_full(*self._args(), _p(out))
        if self.double_bounce:
            o, n, m = np.meshgrid(np.arange(r.O), np.arange(r.N), np.arange(r.M), indexing="ij")
            e = np.stack([o.ravel(), n.ravel(), m.ravel()], 1)
            out += self.bounce_entries(e).reshape(out.shape)
        return out

    def adc_entries(self, entries: np.ndarray) -> np.ndarray:
        """Selected ADC entries; ``entries`` is E x 3 (o, n, m)."""
        e = np.ascontiguousarray(entries, np.int32).reshape(-1, 3)
        out = np.empty(e.shape[0], np.complex128)
        _load().orc_adc_entries(*self._args(), _p(e), e.shape[0], _p(out))
        if self.double_bounce:
            out += self.bounce_entries(e)
        return out

    def lit_pairs(self) -> np.ndarray:
        """Boolean [O][F]: facet k seen by channel o (both antennas light the
        same side of it)."""
        r = self.radar
        st = self.state
        t, x = st[:r.P, None, :], st[None, r.P:, :]
        both = ((t == LIT) & (x == LIT)) | ((t == LIT_REV) & (x == LIT_REV))
        return both.reshape(r.O, -1)

    def n_terms(self) -> int:
        """Echo terms per frame: sum over channels of lit facets x N x M."""
        r = self.radar
        return int(self.lit_pairs().sum()) * r.N * r.M


# ---------------------------------------------------------------------------
# range-Doppler map (Sec. 3.3)
# ---------------------------------------------------------------------------
def echo_gradient(scene, W: np.ndarray, h: float = 1e-6, state: np.ndarray | None = None):
    """Reference gradient of the real functional L = Re sum conj(W) adc of
    the ADC cube (every differentiable loss of the cube reduces to one at
    the point of evaluation, with W = dL/dRe(adc) + i dL/dIm(adc)) with
    respect to the mesh-local vertex coordinates and the per-facet
    reflectivities of a scene with one instance, the visibility held at
    ``state`` (default: the scene's own) -- the fixed-mask derivative the
    differentiable echo defines.

    Vertex coordinates: fourth-order central differences
    (8 (L(+h) - L(-h)) - (L(+2h) - L(-2h))) / (12 h) of this module's
    FP64 frame (truncation O(h^4)).  Reflectivities: L is linear in each
    rho_f (Eq. 7's amplitude), so (L(rho_f + 1) - L(rho_f - 1)) / 2 is
    exact.  Returns (dL/dverts (nv, 3), dL/drho (nf,))."""
    import copy
    if len(scene.instances) != 1 or len(scene.meshes) != 1:
        raise ValueError("echo_gradient takes a scene with one mesh and one instance")
    mesh = scene.meshes[0]
    if state is None:
        state = Frame(scene).state

    def loss(verts, rho):
        m = copy.copy(mesh)
        m.verts = verts
        m.rho = rho
        sc = copy.copy(scene)
        sc.meshes = [m]
        return float((np.conj(W) * Frame(sc, state=state).adc_full()).real.sum())

    v0 = np.asarray(mesh.verts, np.float64)
    r0 = np.asarray(mesh.rho)
    gv = np.zeros_like(v0)
    for i in range(v0.shape[0]):
        for c in range(3):
            f = {}
            for k in (-2, -1, 1, 2):
                v = v0.copy()
                v[i, c] += k * h
                f[k] = loss(v, r0)
            gv[i, c] = (8.0 * (f[1] - f[-1]) - (f[2] - f[-2])) / (12.0 * h)
    gr = np.zeros(r0.shape[0])
    for j in range(r0.shape[0]):
        rp, rm = r0.astype(np.float64).copy(), r0.astype(np.float64).copy()
        rp[j] += 1.0
        rm[j] -= 1.0
        gr[j] = 0.5 * (loss(v0, rp) - loss(v0, rm))
    return gv, gr


def hann(L: int) -> np.ndarray:
    """Symmetric Hann window w[i] = 0.5 - 0.5 cos(2 pi i / (L-1))."""
    if L == 1:
        return np.ones(1)
    i = np.arange(L, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * i / (L - 1))


def range_doppler_cube(adc: np.ndarray) -> np.ndarray:
    """Y[o][d][r]: Hann window and forward FFT over fast time (range), then
    Hann window and forward FFT over slow time (Doppler), per channel
    (Sec. 3.3); Doppler index unshifted."""
    O, N, M = adc.shape
    X = np.fft.fft(adc * hann(M)[None, None, :], axis=2)
    return np.fft.fft(X * hann(N)[None, :, None], axis=1)


def range_doppler_map(adc: np.ndarray) -> np.ndarray:
    """RDM[r][d] (FP64) from an ADC cube [O][N][M] (Sec. 3.3): the range and
    Doppler FFTs of ``range_doppler_cube``, |.|^2 summed over the O
    channels, Doppler axis shifted so zero velocity sits at bin N/2."""
    Y = range_doppler_cube(adc)
    P = (np.abs(Y) ** 2).sum(axis=0)                 # [N][M]
    P = np.fft.fftshift(P, axes=0)
    return np.ascontiguousarray(P.T)                 # [M][N]


def rdm_adjoint(adc: np.ndarray, grad_rdm: np.ndarray) -> np.ndarray:
    """Gradient of a real loss L(RDM) with respect to the ADC cube, as
    dL/dRe(x) + i dL/dIm(x), given dL/dRDM = grad_rdm [M][N] (Doppler
    shifted): with Y the windowed range-Doppler cube, Ybar = 2 G Y, then the
    conjugate transposes of the Doppler and range DFT steps (window times the
    unnormalised inverse DFT)."""
    O, N, M = adc.shape
    Y = range_doppler_cube(adc)                                    # [O][N(d)][M(r)]
    G = np.fft.ifftshift(np.asarray(grad_rdm, np.float64).T, axes=0)   # [d][r]
    Ybar = 2.0 * G[None] * Y
    Xbar = hann(N)[None, :, None] * (N * np.fft.ifft(Ybar, axis=1))
    return hann(M)[None, None, :] * (M * np.fft.ifft(Xbar, axis=2))


# ---------------------------------------------------------------------------
# detection, angle and point cloud (Sec. 3.3, Eqs. 4-6)
# ---------------------------------------------------------------------------
def cfar_alpha(n_train: int, pfa: float) -> float:
    """CA-CFAR threshold factor for square-law (exponential) noise:
    Pfa = (1 + alpha/n)^-n  =>  alpha = n (Pfa^(-1/n) - 1)."""
    return n_train * (pfa ** (-1.0 / n_train) - 1.0)


def ca_cfar(rdm: np.ndarray, guard_r: int, guard_d: int, train_r: int, train_d: int,
            pfa: float):
    """Cell-averaging CFAR on RDM[r][d] (Sec. 3.3, CA-CFAR): the noise level
    of a cell is the mean of its training cells -- the cells of the
    rectangle of half-sizes (guard + train) around it that lie outside the
    guard rectangle of half-sizes guard -- and the cell is a detection when
    its power exceeds alpha times that mean.  Doppler wraps cyclically;
    range cells whose rectangle leaves [0, M) are not tested.  Returns
    (detections as a boolean M x N map, threshold map, +inf where untested)."""
    M, N = rdm.shape
    hr, hd = guard_r + train_r, guard_d + train_d
    mask = np.ones((2 * hr + 1, 2 * hd + 1), bool)
    mask[train_r:train_r + 2 * guard_r + 1, train_d:train_d + 2 * guard_d + 1] = False
    n_train = int(mask.sum())
    alpha = cfar_alpha(n_train, pfa)
    det = np.zeros((M, N), bool)
    thr = np.full((M, N), np.inf)
    for r in range(hr, M - hr):
        for d in range(N):
            cols = [(d + k) % N for k in range(-hd, hd + 1)]
            rect = rdm[r - hr:r + hr + 1][:, cols]
            noise = rect[mask].sum() / n_train
            thr[r, d] = alpha * noise
            det[r, d] = rdm[r, d] > thr[r, d]
    return det, thr


def angle_spectrum(values: np.ndarray, xpos: np.ndarray, lam: float, bins: int) -> np.ndarray:
    """|sum_o Y_o exp(+j 2 pi x_o s / lambda)|^2 on the grid s_i = -1 + 2i/bins
    (the angle FFT across the virtual array, Eq. 6, for arbitrary element
    positions x_o along X; s = sin(theta), theta from boresight +Y to +X)."""
    s = -1.0 + 2.0 * np.arange(bins) / bins
    steer = np.exp(2j * np.pi * np.outer(s, xpos) / lam)
    return np.abs(steer @ values) ** 2


def point_cloud(adc: np.ndarray, radar, guard_r=2, guard_d=2, train_r=8, train_d=4,
                pfa=1e-6, angle_bins=512) -> list:
    """Points (range, range rate, azimuth, x, y, power, r_bin, d_bin) of the
    CA-CFAR detections in row-major (range, shifted Doppler) order:
    range R = c fs r / (2 mu M) (Eq. 4), range rate lambda_c (d - N/2) / (2 N T_r)
    (Eq. 5, positive receding; T_r = T_c, or P T_c with time-division MIMO),
    azimuth asin(s*) at the angle-spectrum peak
    (Eq. 6), x = R sin(theta), y = R cos(theta)."""
    O, N, M = adc.shape
    Y = range_doppler_cube(adc)
    rdm = np.fft.fftshift((np.abs(Y) ** 2).sum(axis=0), axes=0).T
    det, _ = ca_cfar(rdm, guard_r, guard_d, train_r, train_d, pfa)
    B = radar.slope * radar.M / radar.fs
    lam_c = C0 / (radar.f0 + 0.5 * B)
    xpos = np.array([radar.tx[p][0] + radar.rx[q][0] for p in range(radar.P)
                     for q in range(radar.Q)])
    pts = []
    for r, ds in zip(*np.nonzero(det)):
        d = (ds + N // 2) % N
        spec = angle_spectrum(Y[:, d, r], xpos, lam_c, angle_bins)
        i = int(np.argmax(spec))
        s = -1.0 + 2.0 * i / angle_bins
        th = float(np.arcsin(np.clip(s, -1.0, 1.0)))
        R = C0 * radar.fs * r / (2.0 * radar.slope * M)
        Tr = radar.Tc * (radar.P if getattr(radar, "tdm", False) else 1)   # chirp repetition
        v = lam_c * (ds - N / 2) / (2.0 * N * Tr)
        pts.append((R, v, th, R * np.sin(th), R * np.cos(th), float(rdm[r, ds]), int(r), int(ds)))
    return pts


# ---------------------------------------------------------------------------
# additive white Gaussian noise (Sec. 3.2: noise "with a certain
# signal-to-noise ratio")
# ---------------------------------------------------------------------------
_PHILOX_M = (np.uint64(0xD2511F53), np.uint64(0xCD9E8D57))
_PHILOX_W = (np.uint64(0x9E3779B9), np.uint64(0xBB67AE85))
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32 with 10 rounds (Salmon et al., SC 2011), vectorised over
    rows of ``ctr`` (E x 4 uint32); ``key`` is two uint32 words."""
    c = [np.asarray(ctr[:, i], np.uint64) for i in range(4)]
    k0, k1 = np.uint64(int(key[0]) & 0xFFFFFFFF), np.uint64(int(key[1]) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = _PHILOX_M[0] * c[0]
        p1 = _PHILOX_M[1] * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + _PHILOX_W[0]) & _MASK32
        k1 = (k1 + _PHILOX_W[1]) & _MASK32
    return np.stack([x.astype(np.uint32) for x in c], axis=1)


def unit_normal_pairs(n: int, seed: int, frame: int) -> np.ndarray:
    """Standard complex normals CN(0, 1) for elements 0..n-1: Philox output
    (counter = element index, frame; key = seed) mapped to (0, 1] uniforms
    u = (w + 1) 2^-32 and through Box-Muller, (g1 + j g2)/sqrt(2)."""
    e = np.arange(n, dtype=np.uint64)
    ctr = np.stack([e & _MASK32, e >> np.uint64(32),
                    np.full(n, frame & 0xFFFFFFFF, np.uint64), np.zeros(n, np.uint64)], 1)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).astype(np.float64)
    u1 = (w[:, 0] + 1.0) * 2.0 ** -32
    u2 = (w[:, 1] + 1.0) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(u1))
    return (r * np.cos(2 * np.pi * u2) + 1j * r * np.sin(2 * np.pi * u2)) / np.sqrt(2.0)


def add_noise(adc: np.ndarray, snr_db: float, seed: int, frame: int = 0) -> np.ndarray:
    """ADC cube plus white complex Gaussian noise of power P / 10^(SNR/10),
    P the cube's mean |x|^2 (a new array)."""
    x = np.asarray(adc, np.complex128)
    p = float(np.mean(np.abs(x) ** 2))
    sigma = np.sqrt(p / 10.0 ** (snr_db / 10.0))
    n = unit_normal_pairs(x.size, seed, frame).reshape(x.shape)
    return x + sigma * n
