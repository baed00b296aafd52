"""Python binding of ``libbartsim`` (GB300 BART radar echo synthesis).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``libbartsim.so`` (see ``include/bartsim.h``).  Torch supplies
device memory and streams.  There is no CPU fallback: if the library has not
been built, every call raises ``RuntimeError``.

Function names follow the C-ABI (``bart_create``, ``bart_simulate_frame``,
...).  ``Simulator`` bundles them for scene objects that carry ``meshes``,
``instances`` and ``radar`` attributes.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbartsim.so")

BART_OK, BART_EINVAL, BART_ENOMEM, BART_ECUDA = 0, -1, -2, -3
BART_ETIMEOUT, BART_ESTATE, BART_EDEVICE = -4, -5, -6
PATH_FP64, PATH_MIXED, PATH_SPECTRAL = 0, 1, 2
C128, C64 = 0, 1
WINDOW_HANN, WINDOW_RECT = 0, 1
VIS_BACK, VIS_LIT, VIS_GRAZE, VIS_OCCL, VIS_LIT_REV = 0, 1, 2, 3, 4
MESH_TWO_SIDED = 1
MAX_TX = MAX_RX = 16

EXPORTED = ["bart_last_error", "bart_version", "bart_create", "bart_destroy",
            "bart_set_stream", "bart_mesh_upload", "bart_mesh_clear", "bart_scene_set",
            "bart_scene_facets", "bart_radar_set", "bart_simulate_frame", "bart_form_rdm",
            "bart_frame_host", "bart_get_visibility", "bart_set_timing", "bart_get_timing",
            "bart_sync", "bart_form_rdm_static", "bart_add_noise", "bart_detect",
            "bart_scene_partition", "bart_set_graph", "bart_set_synth_layout",
            "bart_autotune", "bart_rdm_adjoint", "bart_simulate_adjoint",
            "bart_simulate_adjoint_mixed",
            "bart_mesh_update", "bart_measure_peaks", "bart_inject_alloc_failure",
            "bart_selftest_wait_timeout", "bart_get_bounce_facets", "bart_get_dims",
            "bart_mesh_dims", "bart_get_bvh"]


class BartError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class bart_instance(ctypes.Structure):
    _fields_ = [("mesh_id", ctypes.c_int32), ("rho_scale", ctypes.c_float),
                ("pos", ctypes.c_double * 3), ("rot", ctypes.c_double * 9),
                ("vel", ctypes.c_double * 3)]


class bart_radar(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("slope", ctypes.c_double),
                ("fs", ctypes.c_double), ("Tc", ctypes.c_double),
                ("M", ctypes.c_int32), ("N", ctypes.c_int32), ("P", ctypes.c_int32),
                ("Q", ctypes.c_int32), ("intra_chirp_motion", ctypes.c_int32),
                ("window", ctypes.c_int32),
                ("tx", (ctypes.c_double * 3) * MAX_TX),
                ("rx", (ctypes.c_double * 3) * MAX_RX),
                ("tdm", ctypes.c_int32), ("delay_ref", ctypes.c_int32),
                ("far_field", ctypes.c_int32), ("double_bounce", ctypes.c_int32),
                ("grazing_eps", ctypes.c_double)]


class bart_stats(ctypes.Structure):
    _fields_ = [("n_facets", ctypes.c_int64), ("n_terms", ctypes.c_int64),
                ("n_lit_pairs", ctypes.c_int64), ("n_grazing", ctypes.c_int64),
                ("n_series", ctypes.c_int64), ("n_edge", ctypes.c_int64),
                ("n_vertex", ctypes.c_int64), ("n_bounce_facets", ctypes.c_int64),
                ("n_bounce_terms", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class bart_dims(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("have_radar", ctypes.c_int32),
                ("n_scenes", ctypes.c_int32), ("O", ctypes.c_int32), ("N", ctypes.c_int32),
                ("M", ctypes.c_int32), ("A", ctypes.c_int32), ("n_meshes", ctypes.c_int32),
                ("n_facets", ctypes.c_int64), ("n_inst_verts", ctypes.c_int64),
                ("vis_antennas", ctypes.c_int64), ("vis_facets", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class bart_timing(ctypes.Structure):
    _fields_ = [("scene_ms", ctypes.c_float), ("bvh_ms", ctypes.c_float),
                ("visibility_ms", ctypes.c_float), ("kinematics_ms", ctypes.c_float),
                ("synthesis_ms", ctypes.c_float), ("rdm_ms", ctypes.c_float),
                ("synthesis_launches", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("detect_ms", ctypes.c_float), ("detect_launches", ctypes.c_int32),
                ("bounce_discovery_ms", ctypes.c_float), ("bounce_synthesis_ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {f: (float(getattr(self, f)) if t is ctypes.c_float else int(getattr(self, f)))
                for f, t in self._fields_}


class bart_detect_cfg(ctypes.Structure):
    _fields_ = [("guard_r", ctypes.c_int32), ("guard_d", ctypes.c_int32),
                ("train_r", ctypes.c_int32), ("train_d", ctypes.c_int32),
                ("pfa", ctypes.c_double), ("angle_bins", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class bart_point(ctypes.Structure):
    _fields_ = [("range", ctypes.c_double), ("rate", ctypes.c_double),
                ("azimuth", ctypes.c_double), ("x", ctypes.c_double), ("y", ctypes.c_double),
                ("power", ctypes.c_double), ("r_bin", ctypes.c_int32), ("d_bin", ctypes.c_int32)]


# numpy view of a bart_point array
POINT_DTYPE = np.dtype([("range", "<f8"), ("rate", "<f8"), ("azimuth", "<f8"), ("x", "<f8"),
                        ("y", "<f8"), ("power", "<f8"), ("r_bin", "<i4"), ("d_bin", "<i4")])
assert POINT_DTYPE.itemsize == ctypes.sizeof(bart_point) == 56

TUNE_MAX = 24


class bart_peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_per_s", ctypes.c_double), ("fp32x2_fma_per_s", ctypes.c_double),
                ("sincos_per_s", ctypes.c_double), ("fp64_fma_per_s", ctypes.c_double),
                ("sms", ctypes.c_int32), ("threads", ctypes.c_int32)]


class bart_tune(ctypes.Structure):
    _fields_ = [("n_trials", ctypes.c_int32), ("best_samples_per_lane", ctypes.c_int32),
                ("best_tiles_per_item", ctypes.c_int32), ("best_ms", ctypes.c_float),
                ("samples_per_lane", ctypes.c_int32 * TUNE_MAX),
                ("tiles_per_item", ctypes.c_int32 * TUNE_MAX),
                ("synthesis_ms", ctypes.c_float * TUNE_MAX)]

    def as_dict(self) -> dict:
        n = int(self.n_trials)
        return {"best": (int(self.best_samples_per_lane), int(self.best_tiles_per_item),
                         float(self.best_ms)),
                "trials": [(int(self.samples_per_lane[i]), int(self.tiles_per_item[i]),
                            float(self.synthesis_ms[i])) for i in range(n)]}


_lib = None
_lock = threading.Lock()


def lib_available() -> bool:
    return os.path.exists(LIB_PATH)


def load_library() -> ctypes.CDLL:
    """Load ``libbartsim.so`` (raises RuntimeError when it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.bart_last_error.restype = ctypes.c_char_p
        L.bart_version.restype = ctypes.c_char_p
        L.bart_create.argtypes = [ctypes.POINTER(P), ctypes.c_int]
        L.bart_destroy.argtypes = [P]
        L.bart_destroy.restype = None
        L.bart_set_stream.argtypes = [P, P]
        L.bart_mesh_upload.argtypes = [P, P, I64, P, I64, P, ctypes.c_uint32, ctypes.POINTER(I32)]
        L.bart_mesh_clear.argtypes = [P]
        L.bart_scene_set.argtypes = [P, P, I32]
        L.bart_scene_facets.argtypes = [P, ctypes.POINTER(I64)]
        L.bart_get_dims.argtypes = [P, ctypes.POINTER(bart_dims)]
        L.bart_mesh_dims.argtypes = [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64)]
        L.bart_radar_set.argtypes = [P, ctypes.POINTER(bart_radar)]
        L.bart_simulate_frame.argtypes = [P, D, I32, P, I32, ctypes.POINTER(bart_stats)]
        L.bart_form_rdm.argtypes = [P, P, I32, P]
        L.bart_frame_host.argtypes = [P, D, I32, P, ctypes.POINTER(bart_stats)]
        L.bart_get_visibility.argtypes = [P, P, ctypes.POINTER(I64)]
        L.bart_get_bvh.argtypes = [P, P, P, P, ctypes.POINTER(I64), ctypes.POINTER(I64),
                                   ctypes.POINTER(I32)]
        L.bart_get_bounce_facets.argtypes = [P, P, P, P, P, P, I64, ctypes.POINTER(I64)]
        L.bart_set_timing.argtypes = [P, I32]
        L.bart_get_timing.argtypes = [P, ctypes.POINTER(bart_timing)]
        L.bart_sync.argtypes = [P]
        L.bart_form_rdm_static.argtypes = [P, I32, I32, I32, I32, I32, P, P]
        L.bart_add_noise.argtypes = [P, P, I32, D, ctypes.c_uint64, ctypes.c_uint32]
        L.bart_scene_partition.argtypes = [P, P, I32]
        L.bart_set_graph.argtypes = [P, I32]
        L.bart_rdm_adjoint.argtypes = [P, P, I32, P, P]
        L.bart_simulate_adjoint.argtypes = [P, D, P, I32, P, P]
        L.bart_simulate_adjoint_mixed.argtypes = [P, D, P, I32, P, P]
        L.bart_mesh_update.argtypes = [P, I32, P, P]
        L.bart_set_synth_layout.argtypes = [P, I32, I32]
        L.bart_autotune.argtypes = [P, D, P, I32, I32, ctypes.POINTER(bart_tune)]
        L.bart_detect.argtypes = [P, P, I32, ctypes.POINTER(bart_detect_cfg), P, P, I32,
                                  ctypes.POINTER(I32)]
        L.bart_measure_peaks.argtypes = [I32, I32, ctypes.POINTER(bart_peaks)]
        L.bart_inject_alloc_failure.argtypes = [I32]
        L.bart_selftest_wait_timeout.argtypes = [P, I32]
        for name in EXPORTED:
            if name not in ("bart_last_error", "bart_version", "bart_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(rc: int) -> None:
    if rc != BART_OK:
        msg = load_library().bart_last_error().decode(errors="replace")
        raise BartError(rc, msg)


def _ptr(t) -> int:
    """Device (or host) address of a torch tensor / numpy array."""
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t.data_ptr())


# ---------------------------------------------------------------------------
# buffer checks: the library receives bare addresses and reads or writes as
# many elements as the context's shapes say, so every buffer is checked here
# against bart_get_dims before the call
# ---------------------------------------------------------------------------
def _dims(ctx: int) -> "bart_dims":
    d = bart_dims()
    _check(load_library().bart_get_dims(ctx, ctypes.byref(d)))
    return d


def _cube(d: "bart_dims", scenes: bool = True) -> Optional[int]:
    """Samples of the ADC buffer (all scenes, or one cube); None before a
    radar is set (the C call then reports BART_ESTATE)."""
    if not d.have_radar:
        return None
    return (d.n_scenes if scenes else 1) * d.O * d.N * d.M


def _rdm_cells(d: "bart_dims", scenes: bool = True) -> Optional[int]:
    if not d.have_radar:
        return None
    return (d.n_scenes if scenes else 1) * d.M * d.N


def _device_buffer(t, name: str, d: "bart_dims", numel: Optional[int], dtype=None) -> None:
    """Raise unless ``t`` is a contiguous CUDA tensor on the context's
    device with ``numel`` elements (when given) of ``dtype`` (when given)."""
    if not getattr(t, "is_cuda", False) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if t.device.index is not None and t.device.index != d.device:
        raise ValueError(f"{name} is on {t.device}, the context on cuda:{d.device}")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements; the context's shapes need {numel}")


def _host_buffer(a, name: str, numel: Optional[int]) -> None:
    """Raise unless ``a`` is a writable C-contiguous float32 host array
    (numpy or a CPU tensor) of ``numel`` elements (when given)."""
    if isinstance(a, np.ndarray):
        ok = a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] and a.flags["WRITEABLE"]
        n = a.size
    else:
        import torch
        ok = (isinstance(a, torch.Tensor) and not a.is_cuda and a.is_contiguous()
              and a.dtype == torch.float32)
        n = a.numel() if isinstance(a, torch.Tensor) else -1
    if not ok:
        raise ValueError(f"{name} must be a writable C-contiguous float32 host array")
    if numel is not None and n != numel:
        raise ValueError(f"{name} has {n} elements; the context's shapes need {numel}")


# ---------------------------------------------------------------------------
# C-ABI mirrors
# ---------------------------------------------------------------------------
def bart_version() -> str:
    return load_library().bart_version().decode()


def bart_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load_library().bart_create(ctypes.byref(h), int(device)))
    return h.value


def bart_destroy(ctx: int) -> None:
    load_library().bart_destroy(ctx)


def bart_set_stream(ctx: int, stream: int) -> None:
    _check(load_library().bart_set_stream(ctx, ctypes.c_void_p(int(stream))))


def bart_mesh_upload(ctx: int, verts: np.ndarray, tris: np.ndarray,
                     rho: Optional[np.ndarray] = None, two_sided: bool = False) -> int:
    v = np.ascontiguousarray(verts, np.float64)
    t = np.ascontiguousarray(tris, np.int32)
    r = None if rho is None else np.ascontiguousarray(rho, np.float32)
    mid = ctypes.c_int32()
    _check(load_library().bart_mesh_upload(
        ctx, v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0],
        None if r is None else r.ctypes.data, MESH_TWO_SIDED if two_sided else 0,
        ctypes.byref(mid)))
    return mid.value


def bart_mesh_update(ctx: int, mesh_id: int, verts, rho=None) -> None:
    """Replace an uploaded mesh's vertices (CUDA float64 nv x 3) and
    optionally reflectivities (CUDA float32 nf) in place, asynchronously."""
    import torch
    d = _dims(ctx)
    nv, nf = bart_mesh_dims(ctx, mesh_id)
    _device_buffer(verts, "verts", d, 3 * nv, torch.float64)
    if rho is not None:
        _device_buffer(rho, "rho", d, nf, torch.float32)
    _check(load_library().bart_mesh_update(ctx, int(mesh_id), ctypes.c_void_p(_ptr(verts)),
                                           None if rho is None else ctypes.c_void_p(_ptr(rho))))


def bart_mesh_clear(ctx: int) -> None:
    _check(load_library().bart_mesh_clear(ctx))


def make_instances(instances) -> ctypes.Array:
    arr = (bart_instance * len(instances))()
    for i, ins in enumerate(instances):
        arr[i].mesh_id = int(ins.mesh_id)
        arr[i].rho_scale = float(getattr(ins, "rho_scale", 1.0))
        for k in range(3):
            arr[i].pos[k] = float(ins.pos[k])
            arr[i].vel[k] = float(ins.vel[k])
        rot = np.asarray(ins.rot, np.float64).reshape(9)
        for k in range(9):
            arr[i].rot[k] = float(rot[k])
    return arr


def bart_scene_set(ctx: int, instances) -> None:
    arr = make_instances(instances)
    _check(load_library().bart_scene_set(ctx, ctypes.cast(arr, ctypes.c_void_p), len(instances)))


def bart_scene_partition(ctx: int, first) -> None:
    """Split the current instances into independent scenes: instances
    [first[b], first[b+1]) form scene b (len(first) = n_scenes + 1)."""
    f = np.ascontiguousarray(first, np.int32)
    _check(load_library().bart_scene_partition(ctx, f.ctypes.data, int(f.size) - 1))


def bart_scene_facets(ctx: int) -> int:
    n = ctypes.c_int64()
    _check(load_library().bart_scene_facets(ctx, ctypes.byref(n)))
    return n.value


def bart_get_dims(ctx: int) -> dict:
    """The context's buffer shapes (bart_dims as a dict)."""
    return _dims(ctx).as_dict()


def bart_mesh_dims(ctx: int, mesh_id: int):
    """(vertex count, facet count) of an uploaded mesh."""
    nv, nf = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().bart_mesh_dims(ctx, int(mesh_id), ctypes.byref(nv), ctypes.byref(nf)))
    return nv.value, nf.value


def make_radar(radar, window: int = WINDOW_HANN) -> bart_radar:
    r = bart_radar()
    r.f0, r.slope, r.fs, r.Tc = float(radar.f0), float(radar.slope), float(radar.fs), float(radar.Tc)
    r.M, r.N = int(radar.M), int(radar.N)
    tx = np.asarray(radar.tx, np.float64).reshape(-1, 3)
    rx = np.asarray(radar.rx, np.float64).reshape(-1, 3)
    r.P, r.Q = tx.shape[0], rx.shape[0]
    r.intra_chirp_motion = int(bool(getattr(radar, "intra_chirp_motion", True)))
    r.window = int(window)
    r.tdm = int(bool(getattr(radar, "tdm", False)))
    r.delay_ref = int(bool(getattr(radar, "delay_ref", False)))
    r.far_field = int(bool(getattr(radar, "far_field", False)))
    r.double_bounce = int(bool(getattr(radar, "double_bounce", False)))
    r.grazing_eps = float(getattr(radar, "grazing_eps", 0.0) or 0.0)
    for p in range(min(r.P, MAX_TX)):
        for k in range(3):
            r.tx[p][k] = float(tx[p, k])
    for q in range(min(r.Q, MAX_RX)):
        for k in range(3):
            r.rx[q][k] = float(rx[q, k])
    return r


def bart_radar_set(ctx: int, radar, window: int = WINDOW_HANN) -> None:
    r = radar if isinstance(radar, bart_radar) else make_radar(radar, window)
    _check(load_library().bart_radar_set(ctx, ctypes.byref(r)))


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise TypeError(f"ADC tensor must be complex64 or complex128, got {t.dtype}")


def bart_simulate_frame(ctx: int, t0: float, path: int, adc, stats: bool = False):
    """Simulate one frame into the contiguous complex CUDA tensor ``adc``
    ([O][N][M]).  Returns the stats dict when ``stats`` (synchronises)."""
    d = _dims(ctx)
    _device_buffer(adc, "adc", d, _cube(d))
    st = bart_stats() if stats else None
    _check(load_library().bart_simulate_frame(
        ctx, float(t0), int(path), ctypes.c_void_p(_ptr(adc)), _dtype_code(adc),
        ctypes.byref(st) if st is not None else None))
    return st.as_dict() if st is not None else None


def bart_form_rdm(ctx: int, adc, rdm) -> None:
    """RDM ([S][M][N] float32) of the ADC cube ([S][O][N][M])."""
    import torch
    d = _dims(ctx)
    _device_buffer(adc, "adc", d, _cube(d))
    _device_buffer(rdm, "rdm", d, _rdm_cells(d), torch.float32)
    _check(load_library().bart_form_rdm(ctx, ctypes.c_void_p(_ptr(adc)), _dtype_code(adc),
                                        ctypes.c_void_p(_ptr(rdm))))


def bart_frame_host(ctx: int, t0: float, path: int, rdm_host, stats: bool = False):
    """Whole frame into a host float32 buffer (numpy array or CPU tensor,
    ideally pinned) of [S][M][N]; synchronises."""
    _host_buffer(rdm_host, "rdm_host", _rdm_cells(_dims(ctx)))
    st = bart_stats() if stats else None
    _check(load_library().bart_frame_host(ctx, float(t0), int(path),
                                          ctypes.c_void_p(_ptr(rdm_host)),
                                          ctypes.byref(st) if st is not None else None))
    return st.as_dict() if st is not None else None


def bart_add_noise(ctx: int, adc, snr_db: float, seed: int, frame: int = 0) -> None:
    """Add white complex Gaussian noise at ``snr_db`` to the CUDA ADC tensor
    in place (Philox4x32-10 counter-based, deterministic per seed/frame).
    ``adc`` is one [O][N][M] cube."""
    d = _dims(ctx)
    _device_buffer(adc, "adc", d, _cube(d, scenes=False))
    _check(load_library().bart_add_noise(ctx, ctypes.c_void_p(_ptr(adc)), _dtype_code(adc),
                                         float(snr_db), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                         int(frame) & 0xFFFFFFFF))


def make_detect_cfg(guard_r: int = 2, guard_d: int = 2, train_r: int = 8, train_d: int = 4,
                    pfa: float = 1e-6, angle_bins: int = 512) -> bart_detect_cfg:
    c = bart_detect_cfg()
    c.guard_r, c.guard_d, c.train_r, c.train_d = int(guard_r), int(guard_d), int(train_r), int(train_d)
    c.pfa, c.angle_bins, c.reserved = float(pfa), int(angle_bins), 0
    return c


def bart_detect(ctx: int, adc, cfg: bart_detect_cfg, points=None, rdm=None,
                sync: bool = True) -> Optional[int]:
    """CA-CFAR detections and their range, rate and azimuth (Sec. 3.3).
    ``points``: CUDA uint8 tensor of max_points * 56 bytes (bart_point
    records) or None; ``rdm``: CUDA float32 M x N tensor or None.  Returns
    the number of detections when ``sync`` (the call then synchronises)."""
    import torch
    d = _dims(ctx)
    _device_buffer(adc, "adc", d, _cube(d, scenes=False))
    max_points = 0
    if points is not None:
        _device_buffer(points, "points", d, None, torch.uint8)
        max_points = points.numel() // POINT_DTYPE.itemsize
    if rdm is not None:
        _device_buffer(rdm, "rdm", d, _rdm_cells(d, scenes=False), torch.float32)
    n = ctypes.c_int32(-1)
    _check(load_library().bart_detect(
        ctx, ctypes.c_void_p(_ptr(adc)), _dtype_code(adc), ctypes.byref(cfg),
        None if rdm is None else ctypes.c_void_p(_ptr(rdm)),
        None if points is None else ctypes.c_void_p(_ptr(points)), int(max_points),
        ctypes.byref(n) if sync else None))
    return n.value if sync else None


def bart_form_rdm_static(adc, rdm, O: int, N: int, M: int, window: int = WINDOW_HANN,
                         stream: Optional[int] = None) -> None:
    """RDM of ``adc`` into ``rdm`` without any device allocation by the
    library (its workspace is a fixed array compiled into it); see
    ``include/bartsim.h`` for the size limit and the sharing rules.

    ``adc`` ([O][N][M] complex64/complex128) and ``rdm`` ([M][N] float32)
    must be contiguous CUDA tensors on one device; the call runs with that
    device current (the C entry point takes the workspace and the launch
    device from the current device)."""
    import torch
    O, N, M = int(O), int(N), int(M)
    if not (isinstance(adc, torch.Tensor) and isinstance(rdm, torch.Tensor)):
        raise TypeError("adc and rdm must be torch tensors")
    if not (adc.is_cuda and rdm.is_cuda and adc.is_contiguous() and rdm.is_contiguous()):
        raise ValueError("adc and rdm must be contiguous CUDA tensors")
    if adc.device != rdm.device:
        raise ValueError(f"adc is on {adc.device}, rdm on {rdm.device}")
    if rdm.dtype != torch.float32:
        raise TypeError(f"rdm must be float32, got {rdm.dtype}")
    code = _dtype_code(adc)
    if min(O, N, M) < 1 or adc.numel() != O * N * M:
        raise ValueError(f"adc has {adc.numel()} samples, O*N*M = {O * N * M}")
    if rdm.numel() != M * N:
        raise ValueError(f"rdm has {rdm.numel()} cells, M*N = {M * N}")
    with torch.cuda.device(adc.device):
        if stream is None:
            stream = torch.cuda.current_stream(adc.device).cuda_stream
        _check(load_library().bart_form_rdm_static(
            ctypes.c_void_p(_ptr(adc)), code, O, N, M, int(window),
            ctypes.c_void_p(_ptr(rdm)), ctypes.c_void_p(int(stream))))


def bart_inject_alloc_failure(nth: int) -> None:
    """Make the library's nth device allocation from now fail with
    BART_ENOMEM (host-side fault injection; 0 disarms)."""
    _check(load_library().bart_inject_alloc_failure(int(nth)))


def bart_selftest_wait_timeout(ctx: int, polls: int = 4096) -> None:
    """Enqueue the bounded-wait self-test: a wait that expires by design;
    the next bart_sync raises BartError(BART_ETIMEOUT)."""
    _check(load_library().bart_selftest_wait_timeout(ctx, int(polls)))


def bart_measure_peaks(device: int = 0, reps: int = 5) -> dict:
    """Measured FP32 FMA (scalar and packed), MUFU sincos and FP64 FMA rates
    of the device (register-only microbenchmarks, CUDA-event timed)."""
    out = bart_peaks()
    _check(load_library().bart_measure_peaks(int(device), int(reps), ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in bart_peaks._fields_}


def bart_get_visibility(ctx: int, state, grazing: bool = False):
    """Copy the frame-start states into ``state`` (A x F uint8 on the
    device); with ``grazing`` also return the number of GRAZE pairs."""
    import torch
    d = _dims(ctx)
    _device_buffer(state, "state", d, d.vis_antennas * d.vis_facets if d.vis_facets else None,
                   torch.uint8)
    n = ctypes.c_int64(-1)
    _check(load_library().bart_get_visibility(ctx, ctypes.c_void_p(_ptr(state)),
                                              ctypes.byref(n) if grazing else None))
    return n.value if grazing else None


def bart_get_bvh(ctx: int) -> dict:
    """Host copy of the last frame's hierarchy: ``nodes`` (F - 1 records of
    ``diagnostics.BVH_NODE_DTYPE``), ``roots`` (int32 per scene) and ``tri``
    (F x 9 frame-start vertices); check it with ``diagnostics.check_bvh``."""
    from .diagnostics import BVH_NODE_DTYPE
    L = load_library()
    nn, nf, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(L.bart_get_bvh(ctx, None, None, None, ctypes.byref(nn), ctypes.byref(nf),
                          ctypes.byref(ns)))
    out = dict(nodes=np.zeros(int(nn.value), BVH_NODE_DTYPE),
               roots=np.zeros(int(ns.value), np.int32), tri=np.zeros((int(nf.value), 9)))
    if out["nodes"].size == 0:               # one facet: no internal node to copy into
        out["nodes"] = np.zeros(1, BVH_NODE_DTYPE)
    _check(L.bart_get_bvh(ctx, *(ctypes.c_void_p(out[k].ctypes.data)
                                 for k in ("nodes", "roots", "tri")),
                          ctypes.byref(nn), ctypes.byref(nf), ctypes.byref(ns)))
    out["nodes"] = out["nodes"][:int(nn.value)]
    return out


def bart_get_bounce_facets(ctx: int) -> dict:
    """The last frame's double-bounce virtual facets (host numpy arrays):
    ``pab`` (V x 4: TX, first facet, second facet, side), ``tri`` (V x 9),
    ``src`` (V x 3 image source), ``usrc`` (V x 3 its velocity), ``w`` (V)."""
    L = load_library()
    n = ctypes.c_int64(0)
    _check(L.bart_get_bounce_facets(ctx, None, None, None, None, None, 0, ctypes.byref(n)))
    V = int(n.value)
    out = dict(pab=np.zeros((V, 4), np.int32), tri=np.zeros((V, 9)), src=np.zeros((V, 3)),
               usrc=np.zeros((V, 3)), w=np.zeros(V))
    if V:
        _check(L.bart_get_bounce_facets(ctx, *(ctypes.c_void_p(out[k].ctypes.data)
                                               for k in ("pab", "tri", "src", "usrc", "w")),
                                        V, ctypes.byref(n)))
    return out


def bart_rdm_adjoint(ctx: int, adc, grad_rdm, grad_adc) -> None:
    """grad_adc = dL/dRe(adc) + i dL/dIm(adc) for dL/dRDM = grad_rdm."""
    import torch
    d = _dims(ctx)
    _device_buffer(adc, "adc", d, _cube(d))
    _device_buffer(grad_rdm, "grad_rdm", d, _rdm_cells(d), torch.float32)
    _device_buffer(grad_adc, "grad_adc", d, _cube(d), adc.dtype)
    _check(load_library().bart_rdm_adjoint(ctx, ctypes.c_void_p(_ptr(adc)), _dtype_code(adc),
                                           ctypes.c_void_p(_ptr(grad_rdm)),
                                           ctypes.c_void_p(_ptr(grad_adc))))


def bart_simulate_adjoint(ctx: int, t0: float, grad_adc, grad_verts, grad_rho=None,
                          mixed: bool = False) -> None:
    """Mesh-vertex (instance-major, mesh-local) and per-facet reflectivity
    gradients of a real loss with dL/dRe(adc) + i dL/dIm(adc) = grad_adc;
    ``mixed`` selects bart_simulate_adjoint_mixed (FP32 per-sample work)."""
    import torch
    d = _dims(ctx)
    _device_buffer(grad_adc, "grad_adc", d, _cube(d))
    _device_buffer(grad_verts, "grad_verts", d, 3 * d.n_inst_verts, torch.float64)
    if grad_rho is not None:
        _device_buffer(grad_rho, "grad_rho", d, d.n_facets, torch.float64)
    lib = load_library()
    fn = lib.bart_simulate_adjoint_mixed if mixed else lib.bart_simulate_adjoint
    _check(fn(ctx, float(t0), ctypes.c_void_p(_ptr(grad_adc)), _dtype_code(grad_adc),
              ctypes.c_void_p(_ptr(grad_verts)),
              None if grad_rho is None else ctypes.c_void_p(_ptr(grad_rho))))


def bart_set_graph(ctx: int, enable: bool) -> None:
    _check(load_library().bart_set_graph(ctx, int(bool(enable))))


def bart_set_synth_layout(ctx: int, samples_per_lane: int = 0, tiles_per_item: int = 0) -> None:
    _check(load_library().bart_set_synth_layout(ctx, int(samples_per_lane), int(tiles_per_item)))


def bart_autotune(ctx: int, t0: float, adc, reps: int = 3) -> dict:
    """Try the mixed-path synthesis layouts on the current scene, keep the
    fastest; returns the trial table (samples/lane, tiles/item, ms)."""
    d = _dims(ctx)
    _device_buffer(adc, "adc", d, _cube(d))
    t = bart_tune()
    _check(load_library().bart_autotune(ctx, float(t0), ctypes.c_void_p(_ptr(adc)),
                                        _dtype_code(adc), int(reps), ctypes.byref(t)))
    return t.as_dict()


def bart_set_timing(ctx: int, enable: bool) -> None:
    _check(load_library().bart_set_timing(ctx, int(bool(enable))))


def bart_get_timing(ctx: int) -> dict:
    t = bart_timing()
    _check(load_library().bart_get_timing(ctx, ctypes.byref(t)))
    return t.as_dict()


def bart_sync(ctx: int) -> None:
    _check(load_library().bart_sync(ctx))


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class _Placed:
    """An instance re-pointed at a mesh id of the batch's mesh pool."""

    def __init__(self, mesh_id: int, ins):
        self.mesh_id = mesh_id
        self.pos, self.rot, self.vel = ins.pos, ins.rot, ins.vel
        self.rho_scale = getattr(ins, "rho_scale", 1.0)

class Simulator:
    """One library context bound to a CUDA device and torch's current stream."""

    def __init__(self, device: int = 0):
        import torch
        self.device = int(device)
        self.ctx = bart_create(self.device)
        with torch.cuda.device(self.device):
            bart_set_stream(self.ctx, torch.cuda.current_stream().cuda_stream)
        self.radar = None
        self.n_facets = 0

    def close(self) -> None:
        if self.ctx:
            bart_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_scene(self, scene, window: int = WINDOW_HANN) -> None:
        """Upload meshes, instances and radar of a scene object."""
        bart_mesh_clear(self.ctx)
        for m in scene.meshes:
            bart_mesh_upload(self.ctx, m.verts, m.tris, m.rho, getattr(m, "two_sided", False))
        bart_scene_set(self.ctx, scene.instances)
        bart_radar_set(self.ctx, scene.radar, window)
        self.n_scenes = 1
        self.scene_foff = [0, sum(int(scene.meshes[i.mesh_id].tris.shape[0])
                                  for i in scene.instances)]
        self.radar = scene.radar
        self.t0 = float(getattr(scene, "t0", 0.0))
        self.n_facets = bart_scene_facets(self.ctx)

    def load_scenes(self, scenes, window: int = WINDOW_HANN) -> None:
        """Upload several scenes sharing one radar profile as one batch
        (bart_scene_partition): outputs gain a leading scene axis."""
        bart_mesh_clear(self.ctx)
        insts, first = [], [0]
        for sc in scenes:
            ids = [bart_mesh_upload(self.ctx, m.verts, m.tris, m.rho, getattr(m, "two_sided", False))
                   for m in sc.meshes]
            for ins in sc.instances:
                insts.append(_Placed(ids[ins.mesh_id], ins))
            first.append(len(insts))
        bart_scene_set(self.ctx, insts)
        bart_scene_partition(self.ctx, first)
        self.scene_foff = [0]
        for sc in scenes:
            self.scene_foff.append(self.scene_foff[-1] + sum(
                int(sc.meshes[i.mesh_id].tris.shape[0]) for i in sc.instances))
        self.radar = scenes[0].radar
        bart_radar_set(self.ctx, self.radar, window)
        self.t0 = float(getattr(scenes[0], "t0", 0.0))
        self.n_facets = bart_scene_facets(self.ctx)
        self.n_scenes = len(scenes)

    def adc_shape(self):
        r = self.radar
        shape = (int(r.tx.shape[0]) * int(r.rx.shape[0]), int(r.N), int(r.M))
        return shape if getattr(self, "n_scenes", 1) == 1 else (self.n_scenes,) + shape

    def simulate(self, path: int = PATH_MIXED, dtype=None, t0: Optional[float] = None,
                 out=None, stats: bool = False):
        import torch
        if dtype is None:
            dtype = torch.complex128 if path == PATH_FP64 else torch.complex64
        if out is None:
            out = torch.empty(self.adc_shape(), dtype=dtype, device=f"cuda:{self.device}")
        st = bart_simulate_frame(self.ctx, self.t0 if t0 is None else t0, path, out, stats)
        return (out, st) if stats else out

    def rdm(self, adc, out=None):
        import torch
        if out is None:
            shape = (int(self.radar.M), int(self.radar.N))
            if getattr(self, "n_scenes", 1) > 1:
                shape = (self.n_scenes,) + shape
            out = torch.empty(shape, dtype=torch.float32, device=adc.device)
        bart_form_rdm(self.ctx, adc, out)
        return out

    def add_noise(self, adc, snr_db: float, seed: int, frame: int = 0):
        bart_add_noise(self.ctx, adc, snr_db, seed, frame)
        return adc

    def detect(self, adc, max_points: int = 4096, rdm=None, **cfg):
        """Point cloud of ``adc``: returns (structured numpy array of the
        detections -- at most ``max_points`` -- and the total count)."""
        import torch
        buf = torch.empty(max(1, max_points) * POINT_DTYPE.itemsize, dtype=torch.uint8,
                          device=adc.device)
        n = bart_detect(self.ctx, adc, make_detect_cfg(**cfg),
                        buf if max_points > 0 else None, rdm)
        k = min(n, max_points)
        host = buf[:k * POINT_DTYPE.itemsize].cpu().numpy()
        return host.view(POINT_DTYPE), n

    def visibility(self, grazing: bool = False):
        """Frame-start states (A x F uint8 tensor); with ``grazing`` the
        tuple (states, number of GRAZE pairs)."""
        import torch
        A = int(self.radar.tx.shape[0]) + int(self.radar.rx.shape[0])
        st = torch.empty((A, self.n_facets), dtype=torch.uint8, device=f"cuda:{self.device}")
        n = bart_get_visibility(self.ctx, st, grazing)
        return (st, n) if grazing else st

    def bvh(self) -> dict:
        """The last frame's hierarchy (bart_get_bvh) with the scenes' facet
        offsets ``foff``, ready for ``diagnostics.check_bvh``."""
        out = bart_get_bvh(self.ctx)
        out["foff"] = list(self.scene_foff)
        return out

    def bounce_facets(self) -> dict:
        """The last frame's double-bounce virtual facets (bart_get_bounce_facets)."""
        return bart_get_bounce_facets(self.ctx)

    def sync(self) -> None:
        bart_sync(self.ctx)
