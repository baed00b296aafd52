"""GPU parity of the method variants: time-division MIMO timing and the
reference-point delay form (Eqs. 11-13 per target), each alone and
together, on both synthesis paths and through the adjoint, against the
FP64 oracle on the same seeded scenes."""
import numpy as np
import pytest
import torch

import oracle
import paper_2208_10939_gb300 as pkg
import scenegen as sg
from paper_2208_10939_gb300 import autograd as bag

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9
TOL_MIXED = 1e-4
VARIANTS = {"tdm": dict(tdm=True), "ref": dict(delay_ref=True),
            "tdm_ref": dict(tdm=True, delay_ref=True)}


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sim():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    s = pkg.Simulator(0)
    yield s
    s.close()


def variant(scene, flags):
    for k, v in flags.items():
        setattr(scene.radar, k, v)
    return scene


def two_cars(flags):
    """Two coarse sedans (different speeds and lanes) in one scene, 2 TX x 2 RX."""
    a = sg.small_car_scene(seed=11, ntri=900, M=128, N=6, P=2, Q=2)
    b = sg.small_car_scene(seed=12, ntri=700, M=128, N=6, P=2, Q=2, slant=24.0, speed=-6.0)
    inst_b = b.instances[0]
    sc = sg.Scene(a.meshes + b.meshes,
                  a.instances + [sg.Instance(len(a.meshes), inst_b.pos + np.array([3.5, 0, 0]),
                                             inst_b.rot, inst_b.vel)], a.radar)
    return variant(sc, flags)


_cache = {}


def reference(name):
    if name not in _cache:
        sc = two_cars(VARIANTS[name])
        fr = oracle.Frame(sc)
        _cache[name] = (sc, fr, fr.adc_full())
    return _cache[name]


@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("path,tol", [(pkg.PATH_FP64, TOL_FP64), (pkg.PATH_MIXED, TOL_MIXED)])
def test_variant_adc_matches_oracle(sim, name, path, tol):
    sc, fr, ref = reference(name)
    sim.load_scene(sc)
    adc = sim.simulate(path).cpu().numpy().astype(np.complex128)
    err = rel_l2(adc, ref)
    print(f"{name} path {path}: relL2 {err:.3e}")
    assert err <= tol
    # the variant changes the result (it is not silently ignored)
    base = oracle.Frame(two_cars({}), state=fr.state).adc_full()
    assert rel_l2(base, ref) > 1e-3


def test_variant_sedan_full_size_sampled(sim):
    """The 20k-facet sedan, 3 TX x 4 RX, 128 x 256, with both variants:
    512 seeded ADC entries against the oracle, both paths."""
    sc = variant(sg.car_scene(), dict(tdm=True, delay_ref=True))
    fr = oracle.Frame(sc)
    rng = np.random.default_rng(17)
    r = sc.radar
    e = np.stack([rng.integers(0, r.O, 512), rng.integers(0, r.N, 512),
                  rng.integers(0, r.M, 512)], 1)
    ref = fr.adc_entries(e)
    sim.load_scene(sc)
    for path, tol in ((pkg.PATH_FP64, TOL_FP64), (pkg.PATH_MIXED, TOL_MIXED)):
        adc = sim.simulate(path).cpu().numpy()
        got = adc[e[:, 0], e[:, 1], e[:, 2]].astype(np.complex128)
        err = rel_l2(got, ref)
        print(f"sedan tdm+ref path {path}: sampled relL2 {err:.3e}")
        assert err <= tol


@pytest.mark.parametrize("name", ["tdm", "ref"])
def test_variant_adjoint_directional_derivative(sim, name):
    sc = variant(sg.small_car_scene(ntri=600, M=128, N=4, P=2, Q=2), VARIANTS[name])
    es = bag.EchoScene(sim, sc)
    v0 = es.vertex_tensor(sc, "cuda")
    verts = v0.clone().requires_grad_(True)
    adc = bag.echo(verts, None, es)
    W = torch.from_numpy(np.random.default_rng(3).normal(size=tuple(adc.shape))
                         + 1j * np.random.default_rng(4).normal(size=tuple(adc.shape))).cuda()
    (torch.conj(W) * adc).real.sum().backward()
    u = torch.from_numpy(np.random.default_rng(6).normal(size=tuple(v0.shape))).cuda()
    h = 1e-7
    with torch.no_grad():
        lp = (torch.conj(W) * bag.echo(v0 + h * u, None, es)).real.sum().item()
        lm = (torch.conj(W) * bag.echo(v0 - h * u, None, es)).real.sum().item()
    fd = (lp - lm) / (2 * h)
    an = float((verts.grad * u).sum())
    assert abs(fd - an) <= 1e-6 * abs(an), (name, fd, an)


def test_tdm_doppler_period(sim):
    """With P = 2 TX in time division, the Doppler axis spans P times less
    speed: a target at 40 m approaching at 5 m/s shows at
    -2 v (P T_c) N / lambda_c bins, wrapped, and the point cloud reports
    the wrapped rate with the TDM bin width."""
    N = 32
    sc = sg.point_target_scene(40.0, -5.0, M=256, N=N, slope=12.5e12, fs=5.12e6, edge=0.6e-3,
                               P=2, Q=1)
    sc.radar.tx = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    sc.radar.tdm = True
    sim.load_scene(sc)
    adc = sim.simulate(pkg.PATH_FP64)
    rdm = sim.rdm(adc).cpu().numpy()
    rr, dd = np.unravel_index(np.argmax(rdm), rdm.shape)
    prof = sg.radar_profile(256)
    cyc = 2 * (-5.0) * 2 * sc.radar.Tc / prof["lam_c"]
    wrapped = (cyc + 0.5) % 1.0 - 0.5
    assert dd == N // 2 + int(round(wrapped * N))
    pts, n = sim.detect(adc, guard_r=2, guard_d=2, train_r=8, train_d=4, pfa=1e-6, angle_bins=64)
    best = pts[np.argmax(pts["power"])]
    v_bin = prof["lam_c"] / (2 * N * 2 * sc.radar.Tc)
    assert abs(best["rate"] - wrapped * prof["lam_c"] / (2 * 2 * sc.radar.Tc)) <= v_bin
