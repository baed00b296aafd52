"""torch.autograd bindings of the differentiable echo: the plain FP64 echo
synthesis and the range-Doppler map, with their hand-written adjoints
(``bart_simulate_adjoint``, ``bart_rdm_adjoint``).  Argument marshalling
only: forward and backward run in the library's kernels.

Parameters are the mesh-local vertices of the scene's instances,
instance-major (one float64 (nv, 3) block per instance, in instance order)
and the per-facet reflectivities (instance-major facets).  With one
instance per mesh these are exactly the meshes' vertex and reflectivity
arrays, which is the layout ``EchoScene`` sets up.
"""
from __future__ import annotations

from typing import List

import torch

from . import (PATH_FP64, PATH_MIXED, Simulator, bart_form_rdm, bart_mesh_update,
               bart_rdm_adjoint, bart_simulate_adjoint, bart_simulate_frame)


class EchoScene:
    """A scene whose every instance has its own mesh, so that the instance
    vertices are the mesh vertices (the differentiable parameters).

    ``precision="mixed"`` runs the mixed-path forward (complex64 cube) and
    the adjoint with FP32 per-sample work (``bart_simulate_adjoint_mixed``);
    the default ``"fp64"`` runs both in FP64."""

    def __init__(self, sim: Simulator, scene, precision: str = "fp64"):
        if precision not in ("fp64", "mixed"):
            raise ValueError("precision must be 'fp64' or 'mixed'")
        self.precision = precision
        self.sim = sim
        sim.load_scene(scene)
        self.nv = [int(scene.meshes[i.mesh_id].verts.shape[0]) for i in scene.instances]
        self.nf = [int(scene.meshes[i.mesh_id].tris.shape[0]) for i in scene.instances]
        if len({i.mesh_id for i in scene.instances}) != len(scene.instances):
            raise ValueError("EchoScene needs one mesh per instance")
        self.mesh_ids: List[int] = [i.mesh_id for i in scene.instances]
        self.t0 = float(getattr(scene, "t0", 0.0))

    def vertex_tensor(self, scene, device) -> torch.Tensor:
        """Instance-major mesh-local vertices as one (sum nv, 3) float64 tensor."""
        import numpy as np
        return torch.from_numpy(np.concatenate([scene.meshes[m].verts for m in self.mesh_ids])
                                ).to(device)

    def upload(self, verts: torch.Tensor, rho: torch.Tensor | None) -> None:
        v0 = f0 = 0
        for mid, nv, nf in zip(self.mesh_ids, self.nv, self.nf):
            bart_mesh_update(self.sim.ctx, mid, verts[v0:v0 + nv].contiguous(),
                             None if rho is None else rho[f0:f0 + nf].contiguous())
            v0 += nv
            f0 += nf


class _Echo(torch.autograd.Function):
    @staticmethod
    def forward(ctx, verts, rho, scene: EchoScene):
        scene.upload(verts.detach(), None if rho is None else rho.detach().float())
        mixed = scene.precision == "mixed"
        adc = torch.empty(scene.sim.adc_shape(),
                          dtype=torch.complex64 if mixed else torch.complex128,
                          device=verts.device)
        bart_simulate_frame(scene.sim.ctx, scene.t0, PATH_MIXED if mixed else PATH_FP64, adc)
        ctx.scene = scene
        ctx.has_rho = rho is not None
        ctx.shapes = (verts.shape, None if rho is None else rho.shape)
        return adc

    @staticmethod
    def backward(ctx, grad_adc):
        scene = ctx.scene
        gv = torch.empty(ctx.shapes[0], dtype=torch.float64, device=grad_adc.device)
        gr = (torch.empty(sum(scene.nf), dtype=torch.float64, device=grad_adc.device)
              if ctx.has_rho else None)
        bart_simulate_adjoint(scene.sim.ctx, scene.t0, grad_adc.contiguous(), gv, gr,
                              mixed=scene.precision == "mixed")
        return gv, (None if gr is None else gr.to(torch.float32).view(ctx.shapes[1])), None


def echo(verts: torch.Tensor, rho: torch.Tensor | None, scene: EchoScene) -> torch.Tensor:
    """ADC cube (complex128, or complex64 for a mixed-precision EchoScene,
    [O][N][M]) of the scene with the given
    instance-major vertices (float64, (sum nv, 3)) and optional per-facet
    reflectivities (float32); differentiable in both."""
    return _Echo.apply(verts, rho, scene)


class _RDM(torch.autograd.Function):
    @staticmethod
    def forward(ctx, adc, sim: Simulator):
        adc = adc.contiguous()
        out = torch.empty((int(sim.radar.M), int(sim.radar.N)), dtype=torch.float32,
                          device=adc.device)
        bart_form_rdm(sim.ctx, adc, out)
        ctx.save_for_backward(adc)
        ctx.sim = sim
        return out

    @staticmethod
    def backward(ctx, grad_rdm):
        (adc,) = ctx.saved_tensors
        g = torch.empty_like(adc)
        bart_rdm_adjoint(ctx.sim.ctx, adc, grad_rdm.contiguous().float(), g)
        return g, None


def range_doppler_map(adc: torch.Tensor, sim: Simulator) -> torch.Tensor:
    """RDM (float32, [M][N]) of an ADC cube; differentiable in the cube."""
    return _RDM.apply(adc, sim)
