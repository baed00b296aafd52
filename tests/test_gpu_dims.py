"""bart_get_dims / bart_mesh_dims on a real context, and the binding's
buffer checks in front of the library: the reported shapes follow the mesh
uploads, the partition, the radar and the last frame, and a buffer of the
wrong size is refused before any work is enqueued."""
import numpy as np
import pytest
import torch

import paper_2208_10939_gb300 as pkg
import scenegen as sg

pytestmark = pytest.mark.gpu


def test_dims_follow_scene_partition_and_frame():
    car = sg.small_car_scene(seed=11, ntri=900, M=64, N=4, P=2, Q=2)
    car2 = sg.small_car_scene(seed=12, ntri=600, M=64, N=4, P=2, Q=2, slant=24.0)
    car2.radar = car.radar
    r = car.radar
    O, A = r.P * r.Q, r.P + r.Q
    nf = [int(sc.meshes[0].tris.shape[0]) for sc in (car, car2)]
    nv = [int(sc.meshes[0].verts.shape[0]) for sc in (car, car2)]
    sim = pkg.Simulator(0)
    try:
        d = pkg.bart_get_dims(sim.ctx)
        assert d["have_radar"] == 0 and d["n_facets"] == 0 and d["vis_facets"] == 0
        assert d["device"] == 0
        sim.load_scene(car)
        d = pkg.bart_get_dims(sim.ctx)
        assert (d["have_radar"], d["n_scenes"], d["O"], d["N"], d["M"], d["A"]) == \
            (1, 1, O, r.N, r.M, A)
        assert (d["n_facets"], d["n_inst_verts"], d["n_meshes"]) == (nf[0], nv[0], 1)
        assert d["vis_facets"] == 0                    # no frame yet
        assert pkg.bart_mesh_dims(sim.ctx, 0) == (nv[0], nf[0])
        with pytest.raises(pkg.BartError):
            pkg.bart_mesh_dims(sim.ctx, 1)

        sim.load_scenes([car, car2])
        adc = sim.simulate(pkg.PATH_MIXED)
        assert tuple(adc.shape) == (2, O, r.N, r.M)
        d = pkg.bart_get_dims(sim.ctx)
        assert d["n_scenes"] == 2 and d["n_facets"] == sum(nf) and d["n_inst_verts"] == sum(nv)
        assert (d["vis_antennas"], d["vis_facets"]) == (A, sum(nf))

        # wrong sizes are refused before the call; the right ones still work
        rdm = torch.empty((2, r.M, r.N), dtype=torch.float32, device="cuda")
        with pytest.raises(ValueError):
            pkg.bart_form_rdm(sim.ctx, adc, rdm[0])
        with pytest.raises(ValueError):
            pkg.bart_simulate_frame(sim.ctx, 0.0, pkg.PATH_MIXED, adc[0])
        with pytest.raises(ValueError):
            pkg.bart_add_noise(sim.ctx, adc, 20.0, 1)
        sim.rdm(adc, rdm)
        host = np.empty((2, r.M, r.N), np.float32)
        pkg.bart_frame_host(sim.ctx, 0.0, pkg.PATH_MIXED, host)
        torch.cuda.synchronize()
        assert np.isfinite(host).all()
        assert np.abs(host - rdm.cpu().numpy()).max() <= 1e-6 * host.max()
        with pytest.raises(ValueError):
            pkg.bart_frame_host(sim.ctx, 0.0, pkg.PATH_MIXED, host[0])
        st = sim.visibility()
        assert tuple(st.shape) == (A, sum(nf))
        sim.sync()
    finally:
        sim.close()
