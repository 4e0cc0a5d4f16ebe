"""Named workloads with the solver options they are measured with: synthetic stand-ins, in the
shapes of the paper's runs, for the planar Helmholtz test, the C96 x 30 sphere in FP64, the
C192 x 30 sphere with the FP32 preconditioner, the batch of 64 uneven solves, and the C192
sphere with the learned coarse correction. preset(name) returns (workloads, options): a list
of inputs.Workload and keyword options for hmg.Solver.
"""
from __future__ import annotations

from . import inputs as I

WORKLOADS = {
    # doubly periodic 16 x 16 x 8 box, constant-coefficient Helmholtz, 2-level MG
    "planar16_helmholtz": lambda: [I.planar_helmholtz()],
    # cubed sphere C96 x 30 quadratic levels (1.66M cells), isothermal, Courant 8
    "sphere_c96_fp64": lambda: [I.cubed_sphere(96, 30)],
    # cubed sphere C192 x 30 (6.6M cells)
    "sphere_c192_mixed": lambda: [I.cubed_sphere(192, 30)],
    # 64 independent solves C{12,24,32,48} x L{10,30,50,70} drawn from SplitMix64(3)
    "batch64_mixed": lambda: [I.cubed_sphere(n, L, seed=3 + i, tol=1e-6)
                              for i, (n, L) in enumerate(I.batched_sizes(64, 3))],
    "sphere_c192_learned": lambda: [I.cubed_sphere(192, 30)],
}

OPTIONS = {
    "planar16_helmholtz": dict(tol=1e-10),
    "sphere_c96_fp64": dict(tol=1e-6),
    "sphere_c192_mixed": dict(tol=1e-6, precision="mixed"),
    "batch64_mixed": dict(tol=1e-6, precision="mixed"),
    # the learned coarse correction as the V-cycle's initial guess inside FGMRES(30)
    "sphere_c192_learned": dict(tol=1e-6, krylov="fgmres", coarse="learned_vcycle"),
}


def preset(name: str):
    """(list of Workload, solver options) of a named preset."""
    if name not in WORKLOADS:
        raise KeyError(f"unknown preset {name!r}; one of {sorted(WORKLOADS)}")
    return WORKLOADS[name](), dict(OPTIONS[name])
