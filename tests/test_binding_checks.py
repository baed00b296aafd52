"""CPU checks of the Python binding's buffer validation.

The C-ABI receives bare addresses and reads or writes as many elements as
the context's shapes say (bart_get_dims), so the binding must refuse a
buffer of the wrong size, dtype, device or layout before the call.  These
tests replace the library by a stand-in that reports fixed shapes and
records the calls that reach it, and pass stand-in CUDA tensors: no GPU and
no kernel is involved.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2208_10939_gb300 as pkg

S, O, N, M, A, F, V = 3, 12, 8, 64, 7, 500, 260
MESH = {0: (120, 200), 1: (140, 300)}


class FakeTensor:
    """Just enough of a CUDA tensor for the binding's checks."""

    def __init__(self, numel, dtype, device=0, contiguous=True, cuda=True):
        self._n, self.dtype, self._c = int(numel), dtype, contiguous
        self.is_cuda = cuda
        self.device = torch.device("cuda", device) if cuda else torch.device("cpu")

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x10000


class FakeLib:
    def __init__(self, radar=True, scenes=1, frame=True):
        self.radar, self.scenes, self.frame = radar, scenes, frame
        self.calls = []

    def bart_get_dims(self, ctx, ref):
        d = ref._obj
        d.device, d.n_scenes, d.n_meshes = 0, self.scenes, len(MESH)
        d.n_facets, d.n_inst_verts = F, V
        if self.radar:
            d.have_radar, d.O, d.N, d.M, d.A = 1, O, N, M, A
        if self.frame:
            d.vis_antennas, d.vis_facets = A, F
        return pkg.BART_OK

    def bart_mesh_dims(self, ctx, mesh_id, nv, nf):
        if mesh_id not in MESH:
            return pkg.BART_EINVAL
        nv._obj.value, nf._obj.value = MESH[mesh_id]
        return pkg.BART_OK

    def bart_last_error(self):
        return b"stand-in error"

    def __getattr__(self, name):
        if not name.startswith("bart_"):
            raise AttributeError(name)

        def call(*args):
            self.calls.append(name)
            return pkg.BART_OK
        return call


@pytest.fixture
def fake(monkeypatch):
    def install(**kw):
        lib = FakeLib(**kw)
        monkeypatch.setattr(pkg, "load_library", lambda: lib)
        return lib
    return install


C64, C128, F32 = torch.complex64, torch.complex128, torch.float32


def test_simulate_frame_needs_the_whole_cube(fake):
    lib = fake(scenes=S)
    pkg.bart_simulate_frame(1, 0.0, pkg.PATH_MIXED, FakeTensor(S * O * N * M, C64))
    assert lib.calls == ["bart_simulate_frame"]
    for bad in (FakeTensor(O * N * M, C64),                       # one scene of three
                FakeTensor(S * O * N * M + 1, C64),
                FakeTensor(S * O * N * M, C64, contiguous=False),
                FakeTensor(S * O * N * M, C64, device=1),
                FakeTensor(S * O * N * M, C64, cuda=False)):
        with pytest.raises(ValueError):
            pkg.bart_simulate_frame(1, 0.0, pkg.PATH_MIXED, bad)
    assert lib.calls == ["bart_simulate_frame"]


def test_before_a_radar_the_library_reports_the_state(fake):
    lib = fake(radar=False, frame=False)
    pkg.bart_simulate_frame(1, 0.0, pkg.PATH_MIXED, FakeTensor(8, C64))
    assert lib.calls == ["bart_simulate_frame"]


def test_rdm_sizes_follow_the_partition(fake):
    lib = fake(scenes=S)
    pkg.bart_form_rdm(1, FakeTensor(S * O * N * M, C128), FakeTensor(S * M * N, F32))
    with pytest.raises(ValueError):
        pkg.bart_form_rdm(1, FakeTensor(S * O * N * M, C128), FakeTensor(M * N, F32))
    with pytest.raises(TypeError):
        pkg.bart_form_rdm(1, FakeTensor(S * O * N * M, C128),
                          FakeTensor(S * M * N, torch.float64))
    assert lib.calls == ["bart_form_rdm"]


def test_noise_and_detection_take_one_cube(fake):
    lib = fake(scenes=S)
    pkg.bart_add_noise(1, FakeTensor(O * N * M, C64), 20.0, 1)
    pkg.bart_detect(1, FakeTensor(O * N * M, C64), pkg.make_detect_cfg(),
                    FakeTensor(56 * 10, torch.uint8), FakeTensor(M * N, F32), sync=False)
    with pytest.raises(ValueError):
        pkg.bart_add_noise(1, FakeTensor(S * O * N * M, C64), 20.0, 1)
    with pytest.raises(ValueError):
        pkg.bart_detect(1, FakeTensor(O * N * M, C64), pkg.make_detect_cfg(), None,
                        FakeTensor(S * M * N, F32), sync=False)
    with pytest.raises(TypeError):
        pkg.bart_detect(1, FakeTensor(O * N * M, C64), pkg.make_detect_cfg(),
                        FakeTensor(56 * 10, torch.int8), None, sync=False)
    assert lib.calls == ["bart_add_noise", "bart_detect"]


def test_adjoint_buffers(fake):
    lib = fake()
    cube = O * N * M
    pkg.bart_rdm_adjoint(1, FakeTensor(cube, C64), FakeTensor(M * N, F32), FakeTensor(cube, C64))
    with pytest.raises(TypeError):
        pkg.bart_rdm_adjoint(1, FakeTensor(cube, C64), FakeTensor(M * N, F32),
                             FakeTensor(cube, C128))
    pkg.bart_simulate_adjoint(1, 0.0, FakeTensor(cube, C128),
                              FakeTensor(3 * V, torch.float64), FakeTensor(F, torch.float64))
    pkg.bart_simulate_adjoint(1, 0.0, FakeTensor(cube, C64), FakeTensor(3 * V, torch.float64),
                              None, mixed=True)
    with pytest.raises(ValueError):
        pkg.bart_simulate_adjoint(1, 0.0, FakeTensor(cube, C128),
                                  FakeTensor(3 * V - 3, torch.float64), None)
    with pytest.raises(ValueError):
        pkg.bart_simulate_adjoint(1, 0.0, FakeTensor(cube, C128),
                                  FakeTensor(3 * V, torch.float64), FakeTensor(F + 1, torch.float64))
    assert lib.calls == ["bart_rdm_adjoint", "bart_simulate_adjoint",
                         "bart_simulate_adjoint_mixed"]


def test_visibility_states_of_the_last_frame(fake):
    lib = fake()
    pkg.bart_get_visibility(1, FakeTensor(A * F, torch.uint8))
    with pytest.raises(ValueError):
        pkg.bart_get_visibility(1, FakeTensor(A * (F - 1), torch.uint8))
    assert lib.calls == ["bart_get_visibility"]
    lib = fake(frame=False)          # no frame yet: the library reports the state
    pkg.bart_get_visibility(1, FakeTensor(1, torch.uint8))
    assert lib.calls == ["bart_get_visibility"]


def test_mesh_update_sizes_come_from_the_mesh(fake):
    lib = fake()
    nv, nf = MESH[1]
    pkg.bart_mesh_update(1, 1, FakeTensor(3 * nv, torch.float64), FakeTensor(nf, F32))
    with pytest.raises(ValueError):
        pkg.bart_mesh_update(1, 0, FakeTensor(3 * nv, torch.float64))
    with pytest.raises(ValueError):
        pkg.bart_mesh_update(1, 1, FakeTensor(3 * nv, torch.float64), FakeTensor(nf - 1, F32))
    with pytest.raises(pkg.BartError):
        pkg.bart_mesh_update(1, 7, FakeTensor(3 * nv, torch.float64))
    assert lib.calls == ["bart_mesh_update"]


def test_host_rdm_of_a_partitioned_frame(fake):
    lib = fake(scenes=S)
    pkg.bart_frame_host(1, 0.0, pkg.PATH_MIXED, np.empty((S, M, N), np.float32))
    pkg.bart_frame_host(1, 0.0, pkg.PATH_MIXED, torch.empty((S, M, N), dtype=F32))
    frozen = np.empty((S, M, N), np.float32)
    frozen.flags["WRITEABLE"] = False
    for bad in (np.empty((M, N), np.float32), np.empty((S, M, N), np.float64),
                np.empty((S, N, M), np.float32).transpose(0, 2, 1), frozen):
        with pytest.raises(ValueError):
            pkg.bart_frame_host(1, 0.0, pkg.PATH_MIXED, bad)
    assert lib.calls == ["bart_frame_host"] * 2


def test_autotune_takes_the_whole_cube(fake):
    lib = fake(scenes=2)
    with pytest.raises(ValueError):
        pkg.bart_autotune(1, 0.0, FakeTensor(O * N * M, C64))
    assert lib.calls == []


def test_dims_struct_matches_c_layout():
    # 8 int32 then 4 int64: no padding on any ABI the library targets
    assert ctypes.sizeof(pkg.bart_dims) == 64
    assert pkg.bart_dims.n_facets.offset == 32
