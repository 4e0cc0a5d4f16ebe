"""Device-side iteration (CUDA graph with a WHILE node), batched solves in one graph launch,
and launch-shape autotuning: each must give what the host-driven single solve gives."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.nonnested import HybridSolver
from paper_2210_11797_gb300 import inputs as I


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64)).cuda()


def _workloads():
    return [I.planar_helmholtz(), I.cubed_sphere(6, 5, nmg=2, seed=4), I.cubed_sphere(12, 10, seed=5),
            I.cubed_sphere(8, 7, seed=6)]


def test_graph_loop_equals_host_loop():
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(12, 30)
    gpu = Solver(w.hier, w.coeffs, tol=1e-8)
    Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
    gpu.set_options(graph=0)
    lam0, st0 = gpu.solve(Rub, Rpi)
    gpu.set_options(graph=1)
    lam1, st1 = gpu.solve(Rub, Rpi)
    lam2, st2 = gpu.solve(Rub, Rpi)            # cached graph, replayed
    assert st0["status"] == st1["status"] == "ok"
    assert st0["iterations"] == st1["iterations"] == st2["iterations"]
    assert torch.equal(lam0, lam1) and torch.equal(lam1, lam2)
    assert st0["history"] == st1["history"]
    # a changed option rebuilds the graph
    gpu.set_options(max_iter=2, tol=1e-14)
    _l, st3 = gpu.solve(Rub, Rpi, check=False)
    assert st3["status"] == "not_converged" and st3["iterations"] == 2
    gpu.close()


def test_batched_solves_equal_single_solves():
    from paper_2210_11797_gb300.hmg import Solver, solve_batched
    ws = _workloads()
    solvers = [Solver(w.hier, w.coeffs, tol=1e-9, precision="mixed") for w in ws]
    Rubs = [_cuda(w.Rub.ravel()) for w in ws]
    Rpis = [_cuda(w.Rpi) for w in ws]
    lams, stats = solve_batched(solvers, Rubs, Rpis)
    for s, w, r, p, lam, st in zip(solvers, ws, Rubs, Rpis, lams, stats):
        single, st1 = s.solve(r, p)
        assert st["status"] == "ok" and st["iterations"] == st1["iterations"]
        assert torch.equal(lam, single)
        ora = HybridSolver(w.hier, w.coeffs)
        B = ora.rhs(w.Rub, w.Rpi)
        lo = lam.cpu().numpy()
        assert np.linalg.norm(B - ora.S @ lo) / np.linalg.norm(B) <= 1.05e-9
    for s in solvers:
        s.close()


def test_autotuned_shapes_keep_results():
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(12, 30)
    gpu = Solver(w.hier, w.coeffs)
    Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
    lam0, st0 = gpu.solve(Rub, Rpi)
    gpu.autotune()
    lam1, st1 = gpu.solve(Rub, Rpi)
    assert st0["iterations"] == st1["iterations"]
    _sw, mg = gpu.launch_shapes()
    if all(c > 0 for c, _t in mg):
        # the column-block shape changes which block solves which columns, not the arithmetic
        assert torch.equal(lam0, lam1)
    else:   # a warp-per-column level: the column solves' rounding order only
        assert float(torch.linalg.norm(lam1 - lam0) / torch.linalg.norm(lam0)) <= 1e-10
    gpu.close()


def test_batch_of_the_seed3_draw():
    """Members of the batched workload itself (sizes from SplitMix64 seed 3, right-hand sides
    seed 3 + i, FP32 preconditioner, tol 1e-6): 12 columns per panel edge (three multigrid
    levels, the coarsest 3 x 3 per panel), 50 and 70 levels, 10 levels, and the largest panels
    (48 x 48, 70 levels) next to the smallest, all in one graph launch. Each answer equals its
    single solve bit for bit and the oracle's own S certifies its FP64 residual."""
    from paper_2210_11797_gb300.hmg import Solver, solve_batched
    sizes = I.batched_sizes(64, 3)
    pick = [0, 3, 4, 1, 10, 13]                    # C12xL50, C12xL70, C24xL70, C32xL10, C48xL70, C12xL10
    assert [sizes[i] for i in pick] == [(12, 50), (12, 70), (24, 70), (32, 10), (48, 70), (12, 10)]
    ws = [I.cubed_sphere(n, L, seed=3 + i, tol=1e-6) for i, (n, L) in ((i, sizes[i]) for i in pick)]
    assert ws[0].hier.nmg == 3 and ws[4].hier.nmg == 4
    solvers = [Solver(w.hier, w.coeffs, tol=w.tol, precision="mixed") for w in ws]
    for s in solvers:
        s.autotune()
    Rubs = [_cuda(w.Rub.ravel()) for w in ws]
    Rpis = [_cuda(w.Rpi) for w in ws]
    lams, stats = solve_batched(solvers, Rubs, Rpis)
    for s, w, r, p, lam, st in zip(solvers, ws, Rubs, Rpis, lams, stats):
        single, st1 = s.solve(r, p)
        assert st["status"] == "ok" and st["iterations"] == st1["iterations"]
        assert torch.equal(lam, single)
        if w.mesh.ncell <= 300_000:                # the oracle's setup stays within seconds
            ora = HybridSolver(w.hier, w.coeffs)
            B = ora.rhs(w.Rub, w.Rpi)
            lo = lam.cpu().numpy()
            assert np.linalg.norm(B - ora.S @ lo) / np.linalg.norm(B) <= 1.05e-6
    for s in solvers:
        s.close()


def test_batch_graph_is_kept_and_captured_again_when_stale():
    """The instantiated batch graph is reused while the contexts, their vectors and options
    stay the same; new values in the same vectors are read at launch; a changed option, launch
    shape, member order or vector makes it capture again. Every answer equals the member's
    single solve."""
    from paper_2210_11797_gb300.hmg import Solver, solve_batched
    ws = _workloads()[1:]
    solvers = [Solver(w.hier, w.coeffs, tol=1e-9, precision="mixed") for w in ws]
    Rubs = [_cuda(w.Rub.ravel()) for w in ws]
    Rpis = [_cuda(w.Rpi) for w in ws]
    lams = [torch.empty(s.ntrace, dtype=torch.float64, device="cuda") for s in solvers]

    def check_against_single(lams_, stats_):
        for s, r, p, lam, st in zip(solvers, Rubs, Rpis, lams_, stats_):
            single, st1 = s.solve(r, p, check=False)
            assert st["status"] == st1["status"] and st["iterations"] == st1["iterations"]
            assert torch.equal(lam, single)

    _l, st_a = solve_batched(solvers, Rubs, Rpis, lams)
    first = [l.clone() for l in lams]
    _l, st_b = solve_batched(solvers, Rubs, Rpis, lams)          # the kept graph
    assert all(torch.equal(a, b) for a, b in zip(first, lams))
    assert [s["iterations"] for s in st_a] == [s["iterations"] for s in st_b]
    check_against_single(lams, st_b)
    # new values in the same vectors: the kept graph reads them (the answer scales by 2 exactly)
    Rubs[0].mul_(2.0)
    Rpis[0].mul_(2.0)
    _l, st_c = solve_batched(solvers, Rubs, Rpis, lams)
    assert torch.equal(lams[0], 2.0 * first[0]) and st_c[0]["iterations"] == st_a[0]["iterations"]
    check_against_single(lams, st_c)
    # a changed option of one member
    solvers[1].set_options(max_iter=2, tol=1e-14)
    _l, st_d = solve_batched(solvers, Rubs, Rpis, lams, check=False)
    assert st_d[1]["status"] == "not_converged" and st_d[1]["iterations"] == 2
    assert st_d[0]["status"] == st_d[2]["status"] == "ok"
    check_against_single(lams, st_d)
    solvers[1].set_options(max_iter=500, tol=1e-9)
    # a changed launch shape of one member (the block form with 2 columns per block)
    sw, mg = solvers[2].launch_shapes()
    solvers[2].set_launch_shapes((2, 128), [(2, 128) for _ in mg])
    _l, st_e = solve_batched(solvers, Rubs, Rpis, lams)
    check_against_single(lams, st_e)
    # another order of the same members, then a member replaced by a new context
    order = [2, 0, 1]
    lo = [lams[i] for i in order]
    _l, st_f = solve_batched([solvers[i] for i in order], [Rubs[i] for i in order],
                             [Rpis[i] for i in order], lo)
    assert [s["iterations"] for s in st_f] == [st_e[i]["iterations"] for i in order]
    solvers[0].close()
    solvers[0] = Solver(ws[0].hier, ws[0].coeffs, tol=1e-9, precision="mixed")
    _l, st_g = solve_batched(solvers, Rubs, Rpis, lams)
    check_against_single(lams, st_g)
    for s in solvers:
        s.close()
