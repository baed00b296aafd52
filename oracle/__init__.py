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

BACK, LIT, GRAZE, OCCL = 0, 1, 2, 3
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
                ("pad_", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.orc_world_vertices.argtypes = [P, P, ctypes.c_int64, P, P, P,
                                               ctypes.c_double, P]
            lib.orc_visibility.argtypes = [P, ctypes.c_int64, P, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, P]
            lib.orc_facet_integral.argtypes = [P, P, P, P]
            lib.orc_visibility_bvh.argtypes = [P, ctypes.c_int64, P, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, P]
            lib.orc_visibility_pairs.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int64,
                                                 ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, P]
            lib.orc_rcs_farfield.argtypes = [P, ctypes.c_int64, P, P, P, P,
                                             ctypes.c_int, P]
            lib.orc_adc_full.argtypes = [P, P, P, P, ctypes.c_int64, P, P,
                                         ctypes.POINTER(_Radar), P]
            lib.orc_adc_entries.argtypes = [P, P, P, P, ctypes.c_int64, P, P,
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


def visibility(tri: np.ndarray, antennas: np.ndarray, eps_face: float = EPS_FACE,
               eps_b: float = EPS_B, eps_t: float = EPS_T) -> np.ndarray:
    """Facet state per antenna, A x F uint8 (BACK, LIT, GRAZE, OCCL), by
    brute force over all occluders (BART single bounce, Sec. 2.2)."""
    tri = np.ascontiguousarray(tri, np.float64)
    ant = np.ascontiguousarray(antennas, np.float64).reshape(-1, 3)
    F, A = tri.shape[0], ant.shape[0]
    st = np.empty((A, F), np.uint8)
    _load().orc_visibility(_p(tri), F, _p(ant), A, eps_face, eps_b, eps_t, _p(st))
    return st


def visibility_bvh(tri: np.ndarray, antennas: np.ndarray, eps_face: float = EPS_FACE,
                   eps_b: float = EPS_B, eps_t: float = EPS_T) -> np.ndarray:
    """``visibility`` through the oracle's own top-down median-split BVH
    (for scenes too large for all pairs); same definition, same states."""
    tri = np.ascontiguousarray(tri, np.float64)
    ant = np.ascontiguousarray(antennas, np.float64).reshape(-1, 3)
    F, A = tri.shape[0], ant.shape[0]
    st = np.empty((A, F), np.uint8)
    _load().orc_visibility_bvh(_p(tri), F, _p(ant), A, eps_face, eps_b, eps_t, _p(st))
    return st


def visibility_pairs(tri: np.ndarray, antennas: np.ndarray, pairs: np.ndarray,
                     eps_face: float = EPS_FACE, eps_b: float = EPS_B,
                     eps_t: float = EPS_T) -> np.ndarray:
    """States of selected (antenna, facet) pairs (E x 2), brute force over
    all occluders: the per-pair definition of ``visibility`` (Sec. 2.2)."""
    tri = np.ascontiguousarray(tri, np.float64)
    ant = np.ascontiguousarray(antennas, np.float64).reshape(-1, 3)
    pr = np.ascontiguousarray(pairs, np.int64).reshape(-1, 2)
    st = np.empty(pr.shape[0], np.uint8)
    _load().orc_visibility_pairs(_p(tri), tri.shape[0], _p(ant), _p(pr), pr.shape[0],
                                 eps_face, eps_b, eps_t, _p(st))
    return st


def facet_integral(tri9: np.ndarray, w: np.ndarray) -> complex:
    """J(w) = integral of exp(j w.(r - c)) over one flat triangle."""
    tri9 = np.ascontiguousarray(tri9, np.float64).reshape(9)
    w = np.ascontiguousarray(w, np.float64).reshape(3)
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_facet_integral(_p(tri9), _p(w), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def rcs_farfield(tri: np.ndarray, rho: np.ndarray, t_hat, r_hat, freqs) -> np.ndarray:
    """Far-field PO RCS sigma(f) (m^2) of a mesh for plane-wave directions
    (toward TX ``t_hat`` and RX ``r_hat``), Sec. 2.2 / Eq. 7's sigma."""
    tri = np.ascontiguousarray(tri, np.float64)
    rho = np.ascontiguousarray(rho, np.float32)
    t = np.ascontiguousarray(t_hat, np.float64) / np.linalg.norm(t_hat)
    r = np.ascontiguousarray(r_hat, np.float64) / np.linalg.norm(r_hat)
    f = np.ascontiguousarray(np.atleast_1d(freqs), np.float64)
    out = np.empty(f.shape[0], np.float64)
    _load().orc_rcs_farfield(_p(tri), tri.shape[0], _p(rho), _p(t), _p(r), _p(f),
                             f.shape[0], _p(out))
    return out


def _radar_struct(radar) -> _Radar:
    return _Radar(radar.f0, radar.slope, radar.fs, radar.Tc, radar.M, radar.N,
                  radar.P, radar.Q, int(bool(radar.intra_chirp_motion)), 0)


class Frame:
    """Frame-start geometry and visibility of a scene (computed once): brute
    force over all occluders up to 60k facets, the oracle's own BVH above."""

    def __init__(self, scene, state: np.ndarray | None = None, bvh: bool | None = None):
        self.scene = scene
        self.radar = scene.radar
        self.tri0, self.fvel, self.rho = world_facets(scene, scene.t0)
        if state is None:
            use_bvh = self.tri0.shape[0] > 60_000 if bvh is None else bvh
            fn = visibility_bvh if use_bvh else visibility
            state = fn(self.tri0, self.radar.antennas)
        self.state = state
        self._rs = _radar_struct(self.radar)

    def adc_full(self) -> np.ndarray:
        """ADC cube [O][N][M] complex128 (Eqs. 7, 9-13)."""
        r = self.radar
        out = np.empty((r.O, r.N, r.M), np.complex128)
        _load().orc_adc_full(_p(self.tri0), _p(self.fvel), _p(self.rho),
                             _p(self.state), self.tri0.shape[0], _p(r.tx), _p(r.rx),
                             ctypes.byref(self._rs), _p(out))
        return out

    def adc_entries(self, entries: np.ndarray) -> np.ndarray:
        """Selected ADC entries; ``entries`` is E x 3 (o, n, m)."""
        e = np.ascontiguousarray(entries, np.int32).reshape(-1, 3)
        out = np.empty(e.shape[0], np.complex128)
        r = self.radar
        _load().orc_adc_entries(_p(self.tri0), _p(self.fvel), _p(self.rho),
                                _p(self.state), self.tri0.shape[0], _p(r.tx), _p(r.rx),
                                ctypes.byref(self._rs), _p(e), e.shape[0], _p(out))
        return out

    def n_terms(self) -> int:
        """Echo terms per frame: sum over channels of lit facets x N x M."""
        r = self.radar
        lit = self.state == LIT
        per_ch = (lit[:r.P, None, :] & lit[None, r.P:, :]).sum(axis=2)
        return int(per_ch.sum()) * r.N * r.M


# ---------------------------------------------------------------------------
# range-Doppler map (Sec. 3.3)
# ---------------------------------------------------------------------------
def hann(L: int) -> np.ndarray:
    """Symmetric Hann window w[i] = 0.5 - 0.5 cos(2 pi i / (L-1))."""
    if L == 1:
        return np.ones(1)
    i = np.arange(L, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * i / (L - 1))


def range_doppler_map(adc: np.ndarray) -> np.ndarray:
    """RDM[r][d] (FP64) from an ADC cube [O][N][M] (Sec. 3.3): Hann window
    and forward FFT over fast time (range), Hann window and forward FFT over
    slow time (Doppler), |.|^2 summed over the O channels, Doppler axis
    shifted so zero velocity sits at bin N/2."""
    O, N, M = adc.shape
    X = np.fft.fft(adc * hann(M)[None, None, :], axis=2)
    Y = np.fft.fft(X * hann(N)[None, :, None], axis=1)
    P = (np.abs(Y) ** 2).sum(axis=0)                 # [N][M]
    P = np.fft.fftshift(P, axes=0)
    return np.ascontiguousarray(P.T)                 # [M][N]
