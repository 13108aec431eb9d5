"""Seeded synthetic inputs for the direct domain-decomposition solver.

Mesh generation, lowest-order Nedelec assembly, domain partition and tearing.
This package only produces inputs (matrices, couplings, loads); it holds none
of the solver's arithmetic, and both the CPU oracle and the GPU library take
their inputs from it.
"""
from .mesh import Mesh, box_mesh, kuhn_edge_count, boundary_edge_mask
from .problems import (Problem, Subdomain, build_problem, plain_c1, batched_c2, medium, big_domains, large_c4,
                       multi_rhs_c5, tiny, linear_field_loads, K0)

__all__ = ["Mesh", "box_mesh", "kuhn_edge_count", "boundary_edge_mask", "Problem", "Subdomain",
           "build_problem", "plain_c1", "batched_c2", "medium", "big_domains", "large_c4", "multi_rhs_c5", "tiny", "linear_field_loads", "K0"]
