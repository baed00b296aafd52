"""GPU parity of the differentiable echo: the hand-written adjoints of the
FP64 synthesis and of the RDM (through torch.autograd) against central
differences -- of the FP64 oracle on small scenes, and of the GPU FP64
forward at the sedan size with the perturbed-sedan inverse problem
(vertices jittered by 5 mm, seed 5).  Visibility is held fixed: parameters
whose +-h runs change a visibility state are skipped and counted.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2208_10939_gb300 as pkg
import scenegen as sg
from paper_2208_10939_gb300 import autograd as bag

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    s = pkg.Simulator(0)
    yield s
    s.close()


def oblique_plate():
    s = sg.plate_scene(range_m=12.0, n=6, M=128, N=4)
    s.instances[0].rot = sg.rot_z(0.2)
    s.instances[0].vel = np.array([0.3, -2.0, 0.0])
    return s


def small_car():
    return sg.small_car_scene(ntri=600, M=128, N=4, P=2, Q=2)


def point():
    return sg.point_target_scene(9.0, 3.0, M=128, N=4, edge=0.6e-3)


CASES = {"oblique_plate": oblique_plate, "small_car": small_car, "point": point}


def with_mesh(scene, verts, rho=None):
    m = scene.meshes[0]
    mesh = sg.Mesh(verts, m.tris, m.rho if rho is None else rho)
    return sg.Scene([mesh] + scene.meshes[1:], scene.instances, scene.radar, t0=scene.t0)


def weights(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_matches_oracle_central_differences(sim, name):
    sc = CASES[name]()
    assert len(sc.meshes) == 1 and len(sc.instances) == 1
    es = bag.EchoScene(sim, sc)
    verts = es.vertex_tensor(sc, "cuda").requires_grad_(True)
    rho = torch.from_numpy(sc.meshes[0].rho.copy()).cuda().requires_grad_(True)
    adc = bag.echo(verts, rho, es)
    W = weights(tuple(adc.shape), 7)
    Wt = torch.from_numpy(W).cuda()
    L = (torch.conj(Wt) * adc).real.sum()
    L.backward()
    gv = verts.grad.cpu().numpy()
    gr = rho.grad.cpu().numpy().astype(np.float64)

    def loss(v, r=None):
        fr = oracle.Frame(with_mesh(sc, v, r))
        return float((np.conj(W) * fr.adc_full()).real.sum()), fr.state

    v0 = sc.meshes[0].verts.copy()
    rng = np.random.default_rng(11)
    h = 1e-6
    scale = np.abs(gv).max()
    checked = skipped = 0
    for _ in range(10):
        i, r = int(rng.integers(v0.shape[0])), int(rng.integers(3))
        vp, vm = v0.copy(), v0.copy()
        vp[i, r] += h
        vm[i, r] -= h
        (lp, sp), (lm, sm) = loss(vp), loss(vm)
        if not np.array_equal(sp, sm):
            skipped += 1
            continue
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gv[i, r]) <= 2e-6 * scale + 1e-6 * abs(fd), (name, i, r, fd, gv[i, r])
        checked += 1
    for f in rng.choice(sc.meshes[0].nf, size=min(3, sc.meshes[0].nf), replace=False):
        rp, rm = sc.meshes[0].rho.copy(), sc.meshes[0].rho.copy()
        rp[f] += np.float32(0.25)
        rm[f] -= np.float32(0.25)
        fd = (loss(v0, rp)[0] - loss(v0, rm)[0]) / (float(rp[f]) - float(rm[f]))
        assert abs(fd - gr[f]) <= 1e-7 * np.abs(gr).max() + 1e-6 * abs(fd), (name, f, fd, gr[f])
    print(f"{name}: {checked} vertex coordinates checked, {skipped} skipped (visibility)")
    assert checked >= 6


@pytest.mark.parametrize("name", ["oblique_plate", "point"])
def test_adjoint_matches_oracle_reference_gradient(sim, name):
    """The whole gradient vector (every vertex coordinate and reflectivity)
    of both adjoints against the oracle's reference gradient
    (oracle.echo_gradient: fourth-order central differences of the FP64
    oracle frame, the visibility held at the scene's own)."""
    sc = CASES[name]()
    sim.load_scene(sc)
    shape = sim.adc_shape()
    W = weights(shape, 21)
    gv_ref, gr_ref = oracle.echo_gradient(sc, W)
    Wt = torch.from_numpy(W).cuda()
    nv, nf = sc.meshes[0].verts.shape[0], sc.meshes[0].nf
    for mixed, tol in ((False, 1e-7), (True, 3e-5)):
        gv = torch.empty((nv, 3), dtype=torch.float64, device="cuda")
        gr = torch.empty(nf, dtype=torch.float64, device="cuda")
        pkg.bart_simulate_adjoint(sim.ctx, 0.0, Wt, gv, gr, mixed=mixed)
        ev = np.linalg.norm(gv.cpu().numpy() - gv_ref) / np.linalg.norm(gv_ref)
        er = np.linalg.norm(gr.cpu().numpy() - gr_ref) / np.linalg.norm(gr_ref)
        print(f"{name}: {'mixed' if mixed else 'fp64'} adjoint vs oracle reference gradient: "
              f"vertices {ev:.3e}, reflectivity {er:.3e}")
        assert ev <= tol and er <= tol


def test_directional_derivative_matches_gpu_forward(sim):
    sc = small_car()
    es = bag.EchoScene(sim, sc)
    v0 = es.vertex_tensor(sc, "cuda")
    verts = v0.clone().requires_grad_(True)
    adc = bag.echo(verts, None, es)
    Wt = torch.from_numpy(weights(tuple(adc.shape), 3)).cuda()
    (torch.conj(Wt) * adc).real.sum().backward()
    g = verts.grad
    u = torch.from_numpy(np.random.default_rng(4).normal(size=tuple(v0.shape))).cuda()
    h = 1e-7
    with torch.no_grad():
        lp = (torch.conj(Wt) * bag.echo(v0 + h * u, None, es)).real.sum().item()
        sp = sim.visibility().clone()
        lm = (torch.conj(Wt) * bag.echo(v0 - h * u, None, es)).real.sum().item()
        sm = sim.visibility().clone()
    assert torch.equal(sp, sm)
    fd = (lp - lm) / (2 * h)
    an = float((g * u).sum())
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_rdm_chain_directional_derivative(sim):
    """Loss on the RDM: the chain of both adjoints against central differences."""
    sc = small_car()
    es = bag.EchoScene(sim, sc)
    v0 = es.vertex_tensor(sc, "cuda")
    verts = v0.clone().requires_grad_(True)
    rdm = bag.range_doppler_map(bag.echo(verts, None, es), sim)
    G = torch.from_numpy(np.random.default_rng(5).normal(size=tuple(rdm.shape))).cuda().float()
    (G * rdm).sum().backward()
    g = verts.grad
    u = torch.from_numpy(np.random.default_rng(6).normal(size=tuple(v0.shape))).cuda()
    h = 1e-7

    def L(v):
        with torch.no_grad():
            a = bag.echo(v, None, es)
            # the RDM in FP64 for the difference quotient (the GPU RDM is FP32)
            return float((G.double().cpu().numpy() * oracle.range_doppler_map(a.cpu().numpy())).sum())

    fd = (L(v0 + h * u) - L(v0 - h * u)) / (2 * h)
    an = float((g * u).sum())
    assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)


def test_perturbed_sedan_inverse_problem_gradient():
    """Config-5 workload: the 20k-facet sedan as target, its copy with 5 mm
    vertex noise (seed 5) as the variable; L = ||adc(v) - adc_target||^2.
    The adjoint gradient against GPU FP64 central differences on 8 seeded
    vertex coordinates and one random direction; prints the adjoint time."""
    s = pkg.Simulator(0)
    try:
        sc = sg.car_scene()
        es = bag.EchoScene(s, sc)
        v_true = es.vertex_tensor(sc, "cuda")
        with torch.no_grad():
            target = bag.echo(v_true, None, es).clone()
        rng = np.random.default_rng(5)
        v0 = v_true + torch.from_numpy(0.005 * rng.normal(size=tuple(v_true.shape))).cuda()
        verts = v0.clone().requires_grad_(True)
        adc = bag.echo(verts, None, es)
        L = (adc - target).abs().pow(2).sum()
        torch.cuda.synchronize()
        t = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t.record()
        L.backward()
        t1.record()
        torch.cuda.synchronize()
        g = verts.grad.clone()
        st = pkg.bart_simulate_frame(s.ctx, 0.0, pkg.PATH_FP64, adc.detach().clone(), stats=True)
        print(f"sedan adjoint: {t.elapsed_time(t1):.1f} ms for {st['n_terms']} terms")

        def loss(v):
            with torch.no_grad():
                a = bag.echo(v, None, es)
                return float((a - target).abs().pow(2).sum()), s.visibility().clone()

        h = 1e-6
        scale = float(g.abs().max())
        idx = rng.choice(v0.numel(), size=8, replace=False)
        checked = 0
        for flat in idx:
            e = torch.zeros_like(v0).view(-1)
            e[int(flat)] = h
            e = e.view_as(v0)
            (lp, sp), (lm, sm) = loss(v0 + e), loss(v0 - e)
            if not torch.equal(sp, sm):
                continue
            fd = (lp - lm) / (2 * h)
            an = float(g.view(-1)[int(flat)])
            assert abs(fd - an) <= 1e-5 * scale + 1e-5 * abs(an), (int(flat), fd, an)
            checked += 1
        assert checked >= 6
        u = torch.from_numpy(rng.normal(size=tuple(v0.shape))).cuda()
        (lp, sp), (lm, sm) = loss(v0 + 1e-7 * u), loss(v0 - 1e-7 * u)
        if torch.equal(sp, sm):
            fd = (lp - lm) / 2e-7
            an = float((g * u).sum())
            assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)
    finally:
        s.close()


def test_sedan_rdm_loss_chain_against_central_differences():
    """Config-5 chain at full size: the 20k-facet sedan's RDM as target, its
    copy with 5 mm vertex noise (seed 5) as the variable,
    L = ||RDM(v, rho) - RDM_target||^2 through both adjoints (the RDM's,
    then the FP64 echo's); the vertex and reflectivity gradients against
    central differences of the GPU FP64 forward with an FP64 RDM
    (oracle.range_doppler_map) on seeded coordinates, two facets'
    reflectivities and one random direction."""
    s = pkg.Simulator(0)
    try:
        sc = sg.car_scene()
        es = bag.EchoScene(s, sc)
        v_true = es.vertex_tensor(sc, "cuda")
        rho0 = torch.from_numpy(sc.meshes[0].rho.copy()).cuda()
        with torch.no_grad():
            target = bag.range_doppler_map(bag.echo(v_true, None, es), s).clone()
        rng = np.random.default_rng(5)
        v0 = v_true + torch.from_numpy(0.005 * rng.normal(size=tuple(v_true.shape))).cuda()
        verts = v0.clone().requires_grad_(True)
        rho = rho0.clone().requires_grad_(True)
        rdm = bag.range_doppler_map(bag.echo(verts, rho, es), s)
        (rdm - target).pow(2).sum().backward()
        gv, gr = verts.grad.clone(), rho.grad.clone()
        T = target.double().cpu().numpy()

        def loss(v, r=None):
            with torch.no_grad():
                a = bag.echo(v, r, es)
                vis = s.visibility().clone()
                return float(((oracle.range_doppler_map(a.cpu().numpy()) - T) ** 2).sum()), vis

        h = 1e-6
        scale = float(gv.abs().max())
        checked = 0
        for flat in rng.choice(v0.numel(), size=8, replace=False):
            e = torch.zeros_like(v0).view(-1)
            e[int(flat)] = h
            e = e.view_as(v0)
            (lp, sp), (lm, sm) = loss(v0 + e), loss(v0 - e)
            if not torch.equal(sp, sm):
                continue
            fd = (lp - lm) / (2 * h)
            an = float(gv.view(-1)[int(flat)])
            assert abs(fd - an) <= 1e-4 * scale + 1e-4 * abs(an), (int(flat), fd, an)
            checked += 1
        assert checked >= 6
        directions = 0
        for _ in range(4):              # a direction whose +-h runs keep the visibility
            u = torch.zeros_like(v0)      # (over 100 random vertices: fewer grazing facets)
            pick = torch.from_numpy(rng.choice(v0.shape[0], size=100, replace=False)).cuda()
            u[pick] = torch.from_numpy(rng.normal(size=(100, 3))).cuda()
            (lp, sp), (lm, sm) = loss(v0 + 1e-7 * u), loss(v0 - 1e-7 * u)
            if not torch.equal(sp, sm):
                continue
            fd = (lp - lm) / 2e-7
            an = float((gv * u).sum())
            assert abs(fd - an) <= 1e-4 * abs(an), (fd, an)
            directions += 1
            break
        assert directions == 1
        for f in rng.choice(rho0.numel(), size=2, replace=False):
            dr = torch.zeros_like(rho0)
            dr[int(f)] = 1e-3
            rp, rm = rho0 + dr, rho0 - dr            # float32: divide by the real step
            fd = (loss(v0, rp)[0] - loss(v0, rm)[0]) / (float(rp[int(f)]) - float(rm[int(f)]))
            assert abs(fd - float(gr[int(f)])) <= 1e-4 * float(gr.abs().max()) + 1e-4 * abs(fd)
        print(f"sedan RDM-loss chain: {checked} coordinates, one direction, 2 reflectivities "
              f"match central differences")
    finally:
        s.close()
