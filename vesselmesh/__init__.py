"""Seeded synthetic vessel meshes: the inputs shared by the solver and by the oracle.

This package holds input generation only (geometry, connectivity, node tags and
inflow-boundary descriptors). It contains none of the solver's arithmetic: no
residual, Jacobian, preconditioner or Krylov code. Both the CUDA solver and the
CPU oracle take the arrays it produces as their inputs.
"""
from .mesh import (FLUID, WALL, INTERFACE, INLET, OUTLET, WALL_END, OUTER,
                   Mesh, count_unknowns, interface_faces, tag_nodes, concat_meshes)
from .tube import tube_mesh, tube_config, batch_tubes
from .tree import tree_mesh, tree_config, box_mesh
from .state import poiseuille_state

__all__ = ["FLUID", "WALL", "INTERFACE", "INLET", "OUTLET", "WALL_END", "OUTER", "Mesh",
           "count_unknowns", "interface_faces", "tag_nodes", "concat_meshes", "tube_mesh",
           "tube_config", "batch_tubes", "tree_mesh", "tree_config", "box_mesh", "poiseuille_state"]
