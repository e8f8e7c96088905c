"""The paper's two test problems (Section 3) assembled by libirk's host P1 /
P2 assemblers on the seeded meshes of the synth module."""
from __future__ import annotations

import numpy as np

import synth

from .binding import irk_fem_assemble, irk_fem_assemble_p2, irk_fem_quad_points


def heat(N: int, kappa=None) -> dict:
    """u_t = div(kappa grad u) on the unit square, zero Dirichlet (Eq. testProblemHeat)."""
    mesh = synth.structured_mesh(N, "unit")
    rowptr, col, valM, valF, g = irk_fem_assemble(mesh.xy, mesh.tri, mesh.dof, mesh.n, kappa=kappa)
    return dict(kind="heat", N=N, n=mesh.n, mesh=mesh, rowptr=rowptr, col=col, valM=valM, valF=valF, g=g,
                mesh_arrays=dict(xy=mesh.xy, tri=mesh.tri, dof=mesh.dof))


def heat_p2(N: int) -> dict:
    """The heat problem with quadratic triangles (the paper's heat runs,
    Section 5): (2N-1)^2 unknowns per stage."""
    mesh = synth.structured_mesh_p2(N)
    rowptr, col, valM, valF, g = irk_fem_assemble_p2(mesh.xy, mesh.tri, mesh.dof, mesh.n)
    return dict(kind="heat_p2", N=N, n=mesh.n, mesh=mesh, rowptr=rowptr, col=col, valM=valM, valF=valF, g=g,
                mesh_arrays=None)


def double_glazing(N: int, eps: float = 1.0 / 200.0) -> dict:
    """u_t + w.grad u - eps Lap u = 0 on [-1,1]^2, hot east wall (Eq. testProblemAD)."""
    mesh = synth.structured_mesh(N, "box")
    xq = irk_fem_quad_points(mesh.xy, mesh.tri)
    wind = synth.double_glazing_wind(xq[..., 0], xq[..., 1])
    ub = synth.double_glazing_boundary(mesh)
    kappa = np.full(mesh.n_tri, eps)
    rowptr, col, valM, valF, g = irk_fem_assemble(mesh.xy, mesh.tri, mesh.dof, mesh.n, kappa=kappa, wind=wind, ub=ub)
    return dict(kind="double_glazing", N=N, n=mesh.n, mesh=mesh, rowptr=rowptr, col=col, valM=valM, valF=valF, g=g,
                eps=eps, mesh_arrays=None)
