"""Pins of the degree-p oracle (oracle/higher_order.py) against what the mathematics and the
paper fix: the one-dimensional rules, the RT_p basis (divergence theorem, facet fluxes), the
dof counts of the paper's table of unknowns per cell, the reduction to the lowest-order oracle
at p = 0, hybridise-then-recover against a direct solve of the unhybridised mixed system at
p = 1, 2 and 3 (plane and sphere), symmetry and definiteness of S with its row lengths, the
convergence order of a smooth solution (p = 0, 1, 2), and the two-level preconditioner at
p = 1 and 3."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import higher_order as HO
from oracle.nonnested import HybridSolver
from paper_2210_11797_gb300 import inputs as I


def test_one_dimensional_rules():
    for n in (1, 2, 3, 4):
        x, w = HO.gauss_legendre(n)
        for d in range(2 * n):                     # exact up to degree 2n - 1
            assert np.dot(w, x ** d) == pytest.approx(1.0 / (d + 1), rel=1e-13)
    np.testing.assert_allclose(HO.gauss_lobatto(2), [0.0, 1.0])
    np.testing.assert_allclose(HO.gauss_lobatto(3), [0.0, 0.5, 1.0], atol=1e-15)
    np.testing.assert_allclose(HO.gauss_lobatto(4), [0.0, 0.5 - np.sqrt(5) / 10, 0.5 + np.sqrt(5) / 10, 1.0],
                               atol=1e-14)
    nodes = HO.gauss_lobatto(4)
    for i, xi in enumerate(nodes):                 # cardinal property and derivative
        v, _d = HO.lagrange(nodes, xi)
        np.testing.assert_allclose(v, np.eye(4)[i], atol=1e-13)
    h = 1e-6
    v1, d0 = HO.lagrange(nodes, 0.3)
    vp, _ = HO.lagrange(nodes, 0.3 + h)
    vm, _ = HO.lagrange(nodes, 0.3 - h)
    np.testing.assert_allclose(d0, (vp - vm) / (2 * h), rtol=1e-7, atol=1e-8)
    assert v1.sum() == pytest.approx(1.0)


@pytest.mark.parametrize("p,nu_avg,npr,nlam_avg,mixed,hybrid", [
    (0, 3, 1, 3, 7, 6), (1, 24, 8, 12, 44, 24), (2, 81, 27, 27, 135, 54), (3, 192, 64, 48, 304, 96)])
def test_dof_counts_match_the_table_of_unknowns(p, nu_avg, npr, nlam_avg, mixed, hybrid):
    """Unknowns per cell and cell-matrix sizes (the paper's table of unknowns per cell; shared
    facet unknowns weighted 1/2)."""
    el = HO.Element(p)
    assert el.nfacet // 2 + (el.nu - el.nfacet) == nu_avg
    assert el.npr == npr and el.nlam // 2 == nlam_avg
    assert el.nu + el.npr == mixed and el.nlam == hybrid


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_rt_basis_fluxes_and_divergence_theorem(p):
    """Facet dof (f, s, t) has outward flux equal to the Lagrange function of node (s, t) on
    face f and zero flux through every other face; interior dofs have no flux; and the volume
    integral of each divergence equals its total outward flux."""
    el = HO.Element(p)
    qx, qw = HO.gauss_legendre(p + 3)
    # faces: (fixed coordinate, value, outward normal sign)
    faces = [(1, 0.0, -1), (0, 1.0, 1), (1, 1.0, 1), (0, 0.0, -1), (2, 0.0, -1), (2, 1.0, 1)]
    flux_total = np.zeros(el.nu)
    for f, (d, val, sgn) in enumerate(faces):
        others = [q for q in range(3) if q != d]
        for a, xa in enumerate(qx):
            for b, xb in enumerate(qx):
                pt = [0.0, 0.0, 0.0]
                pt[d], pt[others[0]], pt[others[1]] = val, xa, xb
                V, _div = el.velocity(*pt)
                flux_total += qw[a] * qw[b] * sgn * V[:, d]
        # nodal property at the facet's own Gauss-Legendre nodes
        for s in range(el.nt):
            for t in range(el.nt):
                pt = [0.0, 0.0, 0.0]
                pt[d] = val
                # the tangential coordinates of node (s, t) in this face's numbering
                if f in (0, 1):
                    u1, u2 = el.gl_x[s], el.gl_x[t]
                elif f in (2, 3):
                    u1, u2 = el.gl_x[el.p - s], el.gl_x[t]
                else:
                    u1, u2 = el.gl_x[s], el.gl_x[t]
                pt[others[0]], pt[others[1]] = u1, u2
                V, _div = el.velocity(*pt)
                flux = sgn * V[:, d]
                want = np.zeros(el.nu)
                want[(f * el.nt + s) * el.nt + t] = 1.0
                # dofs of the other faces of the same direction vanish here, interior ones too
                same_dir = [g for g, fc in enumerate(faces) if fc[0] == d]
                mask = np.zeros(el.nu, bool)
                for g in same_dir:
                    mask[g * el.nt * el.nt:(g + 1) * el.nt * el.nt] = True
                mask[el.nfacet:] = np.array([dd == d for (dd, _a, _t, _s) in el.vdofs[el.nfacet:]])
                np.testing.assert_allclose(flux[mask], want[mask], atol=1e-13)
    # divergence theorem
    vol_div = np.zeros(el.nu)
    for a, xa in enumerate(qx):
        for b, xb in enumerate(qx):
            for c, xc in enumerate(qx):
                _V, div = el.velocity(xa, xb, xc)
                vol_div += qw[a] * qw[b] * qw[c] * div
    np.testing.assert_allclose(vol_div, flux_total, atol=1e-13)
    np.testing.assert_allclose(flux_total[el.nfacet:], 0.0, atol=1e-13)


def _planar(n=4, nlev=3, nmg=2):
    return I.planar_helmholtz(n=n, nlev=nlev, nmg=nmg)


def _sphere_helmholtz(n=2, nlev=2):
    """The Helmholtz preset on cubed-sphere cells (curved, non-affine trilinear hexahedra) of a
    unit sphere with a shell of depth 0.3, so that the direct solves stay well conditioned."""
    hier = I.sphere_hierarchy(n, nlev, I.quadratic_levels(nlev, 0.3), 1, radius=1.0)
    co = I.Coefficients([I.unit_background(m) for m in hier.meshes], dt=1.0, preset=1, sigma=10.0)
    return hier, co


def test_degree_zero_reduces_to_the_lowest_order_oracle():
    """At p = 0 the degree-p code builds the same S, B_lambda, Gamma and two-level cycle as the
    lowest-order oracle (on affine cells, where the Gauss and one-point volumes agree)."""
    w = _planar()
    ho = HO.HigherOrderHybrid(w.hier, w.coeffs, 0)
    lo = HybridSolver(w.hier, w.coeffs)
    scale = abs(lo.S).max()
    assert abs(ho.S - lo.S).max() <= 1e-13 * scale
    Rpi = w.Rpi[:, None]
    B = ho.rhs(w.Rub, Rpi)
    B0 = lo.rhs(w.Rub, w.Rpi)
    assert np.abs(B - B0).max() <= 1e-13 * np.abs(B0).max()
    np.testing.assert_allclose(ho.gamma, lo.gamma, rtol=1e-12)
    r = lo.S @ np.random.default_rng(1).standard_normal(lo.S.shape[0])
    np.testing.assert_allclose(ho.two_level(r), lo.two_level(r), rtol=1e-10, atol=1e-12 * np.abs(r).max())


def _hybrid_equals_mixed(hier, co, p, seed):
    ho = HO.HigherOrderHybrid(hier, co, p)
    rng = np.random.default_rng(seed)
    C = ho.mesh.ncell
    Ru, Rpi = rng.standard_normal((C, ho.el.nu)), rng.standard_normal((C, ho.el.npr))
    B = ho.rhs(Ru, Rpi)
    lam = spla.spsolve(ho.S.tocsc(), B)
    u, pi = ho.reconstruct(lam, Ru, Rpi)
    uf, uint, pim = HO.mixed_solve(ho, Ru, Rpi)
    nf = ho.el.nfacet
    sg = HO.facet_orientation(ho.mesh, ho.el)
    # continuity: both cells of a facet see the same global flux; it is the mixed solution's
    assert np.abs(u[:, :nf] * sg - uf[ho.gid]).max() <= 1e-12 * np.abs(uf).max()
    assert np.abs(u[:, nf:] - uint).max() <= 1e-12 * np.abs(uint).max()
    assert np.abs(pi - pim).max() <= 1e-12 * np.abs(pim).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_hybridised_solution_equals_the_mixed_solution_on_the_plane(p):
    w = _planar(n=3, nlev=2, nmg=1)
    _hybrid_equals_mixed(w.hier, w.coeffs, p, 3 + p)


@pytest.mark.parametrize("p", [1, 2])
def test_hybridised_solution_equals_the_mixed_solution_on_the_sphere(p):
    """Curved cells and the reversed traversal of every vertical facet by its second column
    (the s <-> p - s map; at p = 2 the middle node maps to itself)."""
    hier, co = _sphere_helmholtz()
    _hybrid_equals_mixed(hier, co, p, 11 + p)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_trace_operator_is_symmetric_positive_definite(p):
    w = _planar(n=3, nlev=2, nmg=1)
    ho = HO.HigherOrderHybrid(w.hier, w.coeffs, p)
    S = ho.S.toarray()
    assert np.abs(S - S.T).max() <= 1e-13 * np.abs(S).max()
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0
    # an interior row couples two cells x 6 (p+1)^2 facet nodes with the shared facet's
    # (p+1)^2 once: 11 (p+1)^2 (44, 99, 176); ground and lid rows 6 (p+1)^2
    nb = (p + 1) ** 2
    nnz = np.diff(ho.S.indptr)
    assert nnz.max() == 11 * nb and nnz.min() == 6 * nb


def test_smooth_solution_converges_at_order_p_plus_one():
    """sigma Pi - lap Pi = f on the periodic box with Pi = sin(2 pi x) cos(2 pi y) cos(pi z / H):
    the L2 error of the DG_p pressure falls by 2^(p+1) per halving of the mesh (p = 0: 2,
    p = 1: 4, p = 2: 8)."""
    H = 0.1

    def pi_exact(x):
        return np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]) * np.cos(np.pi * x[:, 2] / H)

    rates = {}
    for p in (0, 1, 2):
        errs = []
        for n in (4, 8):
            w = I.planar_helmholtz(n=n, nlev=n, nmg=1, top=H)
            sigma = w.coeffs.sigma

            def f_exact(x, sigma=sigma):
                return (sigma + 8 * np.pi ** 2 + (np.pi / H) ** 2) * pi_exact(x)
            ho = HO.HigherOrderHybrid(w.hier, w.coeffs, p)
            Ru, Rpi, l2 = HO.manufactured_rhs(ho, pi_exact, f_exact)
            lam = spla.spsolve(ho.S.tocsc(), ho.rhs(Ru, Rpi))
            _u, pi = ho.reconstruct(lam, Ru, Rpi)
            errs.append(l2(pi))
        rates[p] = np.log2(errs[0] / errs[1])
    assert 0.8 < rates[0] < 1.3, rates
    assert 1.8 < rates[1] < 2.4, rates
    assert 2.7 < rates[2] < 3.5, rates


@pytest.mark.parametrize("p,n", [(1, 8), (3, 4)])
def test_two_level_preconditioner_at_degree_p(p, n):
    """Algorithm 2 with the piecewise-constant coarse space at p = 1 and 3: BiCGStab reaches
    1e-10, well before the iteration count of the unpreconditioned method, and the converged
    lambda is the direct solution."""
    w = _planar(n=n, nlev=4, nmg=2 if n >= 8 else 1)
    ho = HO.HigherOrderHybrid(w.hier, w.coeffs, p)
    rng = np.random.default_rng(7)
    Ru, Rpi = rng.standard_normal((ho.mesh.ncell, ho.el.nu)), rng.standard_normal((ho.mesh.ncell, ho.el.npr))
    lam, hist, st = ho.solve(Ru, Rpi, 1e-10)
    assert st == "ok" and len(hist) - 1 <= 20, len(hist)
    ref = spla.spsolve(ho.S.tocsc(), ho.rhs(Ru, Rpi))
    assert np.linalg.norm(lam - ref) / np.linalg.norm(ref) < 1e-8
    from oracle.nonnested import bicgstab
    _x, hist0, _st = bicgstab(lambda x: ho.S @ x, ho.rhs(Ru, Rpi), lambda v: v, 1e-10, 400)
    assert len(hist0) > 2 * len(hist)


def test_smoother_blocks_are_the_facet_and_column_blocks():
    """D of Algorithm 1 at p = 1: (p+1)^2 = 4 rows per vertical-facet block, and each column's
    horizontal facets couple only to their neighbours above and below (block tridiagonal)."""
    w = _planar(n=3, nlev=3, nmg=1)
    ho = HO.HigherOrderHybrid(w.hier, w.coeffs, 1)
    D = ho.D.tocoo()
    h = D.row < ho.NH
    assert np.all(D.row[h] // 4 == D.col[h] // 4)
    z = ~h
    zr, zc = (D.row[z] - ho.NH) // 4, (D.col[z] - ho.NH) // 4      # horizontal facet of each entry
    assert np.all(zr // 4 == zc // 4)                              # same column (L + 1 = 4 facets)
    assert np.abs(zr - zc).max() == 1
