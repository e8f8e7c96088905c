"""The paper's two test problems (Section 3) assembled by libirk's host P1 /
P2 assemblers on the seeded meshes of the synth module."""
from __future__ import annotations

import numpy as np

import synth

from .binding import (irk_fem_assemble, irk_fem_assemble_p2, irk_fem_assemble_streamline, irk_fem_assemble_supg,
                      irk_fem_quad_points)


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


def double_glazing_supg(N: int, eps: float = 1.0 / 200.0, gamma: float = 10.0) -> dict:
    """Double glazing with SUPG stabilisation and Nitsche boundary conditions
    (the paper's advection-diffusion runs, Section 5): every node an unknown,
    n = (N+1)^2; u0 = the boundary values (1 on the east wall, 0 elsewhere)."""
    mesh = synth.structured_mesh(N, "box")
    xq = irk_fem_quad_points(mesh.xy, mesh.tri)
    wind = synth.double_glazing_wind(xq[..., 0], xq[..., 1])
    cen = mesh.xy[mesh.tri].mean(axis=1)
    wind_c = synth.double_glazing_wind(cen[:, 0], cen[:, 1])
    ub = synth.double_glazing_boundary(mesh)
    rowptr, col, valM, valF, g = irk_fem_assemble_supg(mesh.xy, mesh.tri, eps, wind, wind_c, ub=ub, gamma=gamma)
    valT = irk_fem_assemble_streamline(mesh.xy, mesh.tri, eps, wind_c, rowptr, col)
    return dict(kind="double_glazing_supg", N=N, n=mesh.n_nodes, mesh=mesh, rowptr=rowptr, col=col, valM=valM,
                valF=valF, g=g, eps=eps, u0=ub.copy(), mesh_arrays=None, valT=valT)
