"""Plain FP64 CPU oracle of the hybridised non-nested multigrid trace solve.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import this package. The product path (the CUDA library and its
Python binding) never calls it, and the two share no code: the only common module is
`paper_2210_11797_gb300.inputs`, which generates seeded meshes, backgrounds and right-hand
sides and contains none of the method's arithmetic.

Every function follows one passage of Betteridge et al., "Hybridised multigrid
preconditioners for a compatible finite element dynamical core" (arXiv 2210.11797):

* `fem`        - local matrices (Sec. 2.2, Eq. bilinear_forms, quadrature rule), the 2x2
                 elimination (Eq. 2x2system), hybridisation, static condensation
                 (Eqs. gh-fem-hybrid, hybrid-S, hybrid-rhs) and recovery (Eq. hybrid-recovery);
                 the unhybridised mixed system used as a pin.
* `smoother`   - the trace line smoother (Algorithm 1) with the Thomas algorithm.
* `pressure_mg`- the pressure operator H (Eq. elliptic_pressure_system), the column
                 block-Jacobi smoother (Eq. pressure_block_jacobi) and the tensor-product
                 multigrid V-cycle (Sec. 2.3).
* `nonnested`  - prolongation/restriction, the coarse scaling Gamma (Eq. scaling_matrix),
                 the non-nested two-level cycle (Algorithm 2) and right-preconditioned
                 BiCGStab (Sec. 3.2).

Where the paper leaves a passage open, the reading taken is stated in the docstring of the
function that uses it. Pins (tests/test_oracle_*.py, marker "not gpu") tie each function to
something other than itself: closed forms on boxes, the divergence theorem, the
hybrid = mixed identity against a dense direct solve, Thomas vs dense LU, and the
convergence behaviour the paper reports.

Parity unpinned: the absolute iteration counts on the synthetic workloads (the paper has
no isothermal random-RHS case), and the coarsest-level sweep count (the paper defers the
pressure multigrid details to Maynard et al. 2020).
"""
