"""CPU FP64 oracle for the direct domain-decomposition solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package; only the tests, `__graft_entry__.smoke()` and the CPU
baseline leg of `bench.py` do.  It shares no code with the GPU library: its
only inputs are the seeded problems from `femgen`.

Routes to the same solution x = A^{-1} b of the assembled FEM system:
  * dense.lu_solve          - dense LU with partial pivoting (tiny systems);
  * skyline.BandLDLT        - RCM + band-profile LDL^T of the undecomposed system;
  * skyline.envelope_entries - its skyline (envelope) factor size: O2's factor memory;
  * dd.DDOracle             - the paper's decomposition route (Section II):
                              per-domain LDL^T, F = sum B_i A_i^{-1} B_i^T,
                              F lambda = d, primal recovery;
  * dd.SparseDDOracle       - the same route with sparse (SuperLU) domain
                              factorizations, for domains beyond the dense reach;
  * tree.TreeDDOracle       - the same route with F eliminated block by block
                              over the domain tree (nested dissection): the
                              route that reaches the 512- and 2048-domain
                              workloads, and a subtree of one as a timed sample;
  * dd.arrow_solve          - the arrowhead system solved undecomposed by LU with
                              partial pivoting (inputs whose LDL^T needs pivoting);
  * dense.ldlt_bk_restricted - LDL^T with Bunch-Kaufman pivoting restricted to
                              diagonal blocks (the pivoting rule of Section II);
  * refine.residual_dd      - double-double residuals for iterative refinement;
  * symbolic.fronts_by_elimination / fronts_by_tree - the front tree of the
                              auxiliary matrix's symbolic factorization
                              (Section II), by clique-graph elimination and
                              from the domain tree;
  * shard.plan / ShardedTreeDD - the tree route sharded over ranks along a
                              cut of the front tree (one subtree per rank, the
                              fronts above the cut on rank 0), run on a
                              torch.distributed group (gloo on the CPU);
  * domain_symbolic          - validity of a nested dissection of one domain
                              and its front structure, by row-by-row graph
                              elimination and by reach.

Parity status: pinned by closed forms and library special cases (see the
tests); the paper prints no numerical values, so no value of the paper pins it.
"""
from .dense import lu_solve, ldlt, ldlt_solve, ldlt_bk_restricted, ldlt_bk_solve
from .skyline import BandLDLT, rcm, envelope_entries
from .dd import DDOracle, SparseDDOracle, gather_copies, subdomain_schur, arrow_residual, local_B, arrow_dense, arrow_solve
from .refine import residual_dd, refine, backward_error
from .tree import TreeDDOracle, subtree_nodes
from .symbolic import fronts_by_elimination, fronts_by_tree, lca_fronts, dual_domains
from . import domain_symbolic, shard

__all__ = ["lu_solve", "ldlt", "ldlt_solve", "ldlt_bk_restricted", "ldlt_bk_solve", "BandLDLT", "rcm", "envelope_entries",
           "DDOracle", "SparseDDOracle", "TreeDDOracle", "subtree_nodes", "gather_copies", "subdomain_schur", "arrow_residual", "local_B", "arrow_dense", "arrow_solve",
           "fronts_by_elimination", "fronts_by_tree", "lca_fronts", "dual_domains", "domain_symbolic", "shard",
           "residual_dd", "refine", "backward_error"]
