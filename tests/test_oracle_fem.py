"""Pins of the oracle's cell matrices, condensation and recovery (CPU only).

Each test checks the oracle against something other than itself: the defining flux
property of RT0, exact volumes, closed forms on boxes, Sherman-Morrison, and a dense
direct solve of the unhybridised mixed system (Sec. 2.4: hybridisation reproduces the
mixed solution).
"""
import numpy as np
import pytest

from oracle import fem
from oracle.nonnested import HybridSolver
from paper_2210_11797_gb300 import inputs as I

# 4-point Gauss rule per direction for face integrals (exact for the degrees involved)
_GX, _GW = np.polynomial.legendre.leggauss(4)
GX4, GW4 = 0.5 * (_GX + 1.0), 0.5 * _GW

# reference faces: (fixed axis, fixed value) per local face
FACES = [(1, 0.0), (0, 1.0), (1, 1.0), (0, 0.0), (2, 0.0), (2, 1.0)]


def _face_points(face):
    axis, val = FACES[face]
    free = [a for a in range(3) if a != axis]
    for s, ws in zip(GX4, GW4):
        for t, wt in zip(GX4, GW4):
            p = np.zeros(3)
            p[axis], p[free[0]], p[free[1]] = val, s, t
            yield p, ws * wt, free


def test_rt0_reference_flux_and_divergence():
    """Each reference basis function has unit outward flux through its own face, none
    through the others, and divergence 1 (checked by central differences)."""
    for g, (axis, val) in enumerate(FACES):
        for f in range(6):
            flux = 0.0
            for p, w, _free in _face_points(g):
                n = np.zeros(3)
                n[axis] = 1.0 if val == 1.0 else -1.0
                flux += w * fem.rt0_reference_basis(*p)[f] @ n
            assert flux == pytest.approx(1.0 if f == g else 0.0, abs=1e-14)
    h = 1e-6
    p = np.array([0.3, 0.6, 0.2])
    for f in range(6):
        div = sum((fem.rt0_reference_basis(*(p + h * e))[f][a] - fem.rt0_reference_basis(*(p - h * e))[f][a]) / (2 * h)
                  for a, e in enumerate(np.eye(3)))
        assert div == pytest.approx(1.0, abs=1e-8)


def _physical_flux(verts, f, g):
    """Flux of the Piola-mapped basis v_f through physical face g, with the surface
    normal taken from the cross product of the face's tangent vectors."""
    axis, val = FACES[g]
    flux = 0.0
    for p, w, free in _face_points(g):
        N, dN = fem.trilinear_shape(*p)
        J = verts.T @ dN
        v = J @ fem.rt0_reference_basis(*p)[f] / np.linalg.det(J)
        t1, t2 = J[:, free[0]], J[:, free[1]]
        nda = np.cross(t1, t2)                         # area-weighted normal
        # orient outward: along +axis if val == 1
        sign = 1.0 if np.dot(nda, J[:, axis]) > 0 else -1.0
        if val == 0.0:
            sign = -sign
        flux += w * v @ (sign * nda)
    return flux


def test_piola_fluxes_on_curved_sphere_cell():
    mesh = I.cubed_sphere_mesh(3, 2, I.quadratic_levels(2, 30000.0))
    for cell in (0, 5, mesh.ncell - 1):
        verts = fem.cell_vertices(mesh, [cell])[0]
        for f in range(6):
            for g in range(6):
                want = 1.0 if f == g else 0.0
                assert _physical_flux(verts, f, g) == pytest.approx(want, abs=1e-12)


def test_box_mass_matrix_closed_form():
    """On a box hx x hy x hz, RT0 gives per direction (h_d / (A_d)) [[1/3, -1/6], [-1/6, 1/3]]
    in the outward convention, the vertical block scaled by (1 + c22)."""
    hx, hy, hz, c22 = 0.7, 0.3, 0.05, 4.0
    verts = np.zeros((1, 8, 3))
    for v in range(8):
        verts[0, v] = ((v & 1) * hx, ((v >> 1) & 1) * hy, ((v >> 2) & 1) * hz)
    M, vol, vol1, zv = fem.local_mass(verts, np.array([c22]), 0)
    blk = np.array([[1 / 3, -1 / 6], [-1 / 6, 1 / 3]])
    want = np.zeros((6, 6))
    want[np.ix_([1, 3], [1, 3])] = hx / (hy * hz) * blk
    want[np.ix_([0, 2], [0, 2])] = hy / (hx * hz) * blk
    want[np.ix_([4, 5], [4, 5])] = (1 + c22) * hz / (hx * hy) * blk
    np.testing.assert_allclose(M[0], want, rtol=1e-14, atol=1e-14 * np.abs(want).max())
    assert vol[0] == pytest.approx(hx * hy * hz, rel=1e-15)
    assert vol1[0] == pytest.approx(hx * hy * hz, rel=1e-15)
    # zhat . v at the centre: +-1/(2 hx hy) for top/bottom, 0 for the vertical faces
    np.testing.assert_allclose(zv[0], [0, 0, 0, 0, -0.5 / (hx * hy), 0.5 / (hx * hy)], atol=1e-12)


def _polyhedron_volume(verts):
    """|K| = (1/3) sum over faces of the surface integral of x.n (divergence theorem)."""
    vol = 0.0
    for g, (axis, val) in enumerate(FACES):
        for p, w, free in _face_points(g):
            N, dN = fem.trilinear_shape(*p)
            x = N @ verts
            J = verts.T @ dN
            nda = np.cross(J[:, free[0]], J[:, free[1]])
            sign = 1.0 if np.dot(nda, J[:, axis]) > 0 else -1.0
            if val == 0.0:
                sign = -sign
            vol += w * x @ (sign * nda) / 3.0
    return vol


def test_gauss_volume_matches_divergence_theorem_on_sphere():
    mesh = I.cubed_sphere_mesh(4, 3, I.quadratic_levels(3, 30000.0))
    cells = [0, 7, 40, mesh.ncell - 1]
    verts = fem.cell_vertices(mesh, cells)
    _M, vol, _v1, _zv = fem.local_mass(verts, np.zeros(len(cells)), 1)
    for i in range(len(cells)):
        assert vol[i] == pytest.approx(_polyhedron_volume(verts[i]), rel=1e-12)
    assert (vol > 0).all()


def test_helmholtz_condensation_matches_sherman_morrison():
    """Config-1 cells: A_K = [[M, -1], [1^T, sigma |K|]], so by Sherman-Morrison
    S_K = M^-1 - M^-1 1 1^T M^-1 / (m + 1^T M^-1 1), with the block inverse of each
    direction (A_d / h_d) [[4, 2], [2, 4]]."""
    w = I.planar_helmholtz()
    mesh = w.mesh
    A, Kd, _cc = fem.cell_system(mesh, w.coeffs.levels[0], w.coeffs, cells=[0, 9])
    S_K = fem.condense(A, Kd)
    hx = hy = 1.0 / 16
    hz = 0.1 / 8
    Minv = np.zeros((6, 6))
    blk = np.array([[4.0, 2.0], [2.0, 4.0]])
    Minv[np.ix_([1, 3], [1, 3])] = hy * hz / hx * blk
    Minv[np.ix_([0, 2], [0, 2])] = hx * hz / hy * blk
    Minv[np.ix_([4, 5], [4, 5])] = hx * hy / hz * blk
    m = w.coeffs.sigma * hx * hy * hz
    one = np.ones(6)
    want = Minv - np.outer(Minv @ one, Minv @ one) / (m + one @ Minv @ one)
    for i in range(2):
        np.testing.assert_allclose(S_K[i], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_config1_trace_operator_spd_and_row_structure():
    w = I.planar_helmholtz(n=4, nlev=3, nmg=1)
    s = HybridSolver(w.hier, w.coeffs)
    S = s.S.toarray()
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S).max()
    np.linalg.cholesky(S)                        # positive definite
    mesh = w.mesh
    nnz = (np.abs(S) > 0).sum(axis=1)
    NH, L = mesh.n_trace_h, mesh.nlev
    assert (nnz[:NH] == 11).all()
    zrow = nnz[NH:].reshape(mesh.ncol, L + 1)
    assert (zrow[:, 1:L] == 11).all() and (zrow[:, 0] == 6).all() and (zrow[:, L] == 6).all()
    assert S.shape[0] == 3 * mesh.ncell + mesh.ncol   # 3 trace unknowns per cell + lids


def _physical_box(n, nlev, length=3.0e5, top=3000.0, dt=600.0):
    hier = I.planar_hierarchy(n, nlev, length, I.quadratic_levels(nlev, top), 1)
    bg = I.isothermal_background(hier.meshes[0], 250.0)
    # perturb the background horizontally so theta* is not column-uniform
    rng = np.random.default_rng(5)
    bg.theta_lev = bg.theta_lev * (1.0 + 0.01 * rng.standard_normal(bg.theta_lev.shape))
    co = I.Coefficients([bg], dt=dt, preset=0)
    return hier, co


@pytest.mark.parametrize("case", ["box2", "box3", "sphere2"])
def test_hybridised_solution_equals_mixed_solution(case):
    """Sec. 2.4: solving S lambda = B_lambda directly and recovering (u^b, Pi) reproduces the
    direct solution of the unhybridised 2x2 mixed system (continuous RT0)."""
    if case == "sphere2":
        hier = I.sphere_hierarchy(2, 3, I.quadratic_levels(3, 30000.0), 1)
        co = I.Coefficients([I.isothermal_background(hier.meshes[0])], dt=1200.0, preset=0)
    else:
        n = 2 if case == "box2" else 3
        hier, co = _physical_box(n, n)
    mesh = hier.meshes[0]
    rub, rpi = I.draw_rhs(mesh.ncell, 11, "normal")
    A, Kd, _cc = fem.cell_system(mesh, co.levels[0], co)
    S = fem.assemble_trace_operator(mesh, fem.condense(A, Kd)).toarray()
    B = fem.trace_rhs(mesh, A, rub, rpi)
    lam = np.linalg.solve(S, B)
    ub, pi = fem.reconstruct(mesh, A, Kd, lam, rub, rpi)
    Mx, rhs, interior = fem.mixed_system(mesh, co.levels[0], co, rub, rpi)
    sol = np.linalg.solve(Mx, rhs)
    u_mixed, pi_mixed = sol[: len(interior)], sol[len(interior):]
    np.testing.assert_allclose(pi, pi_mixed, rtol=0, atol=1e-12 * np.abs(pi_mixed).max())
    # broken fluxes = orientation sign x continuous flux; zero on ground and lid
    g = fem.trace_dof_ids(mesh)
    s = fem.face_orientation(mesh)
    pos = -np.ones(mesh.n_trace, np.int64)
    pos[interior] = np.arange(len(interior))
    want = np.where(pos[g] >= 0, s * u_mixed[np.maximum(pos[g], 0)], 0.0)
    np.testing.assert_allclose(ub, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_continuity_jump_equals_trace_residual():
    """C^T u^b(lambda) = B_lambda - S lambda for ANY lambda (Eqs. hybrid-S, hybrid-rhs,
    hybrid-recovery), and u^b is continuous once lambda solves the trace system."""
    hier, co = _physical_box(3, 4)
    mesh = hier.meshes[0]
    rub, rpi = I.draw_rhs(mesh.ncell, 2, "normal")
    A, Kd, _cc = fem.cell_system(mesh, co.levels[0], co)
    S = fem.assemble_trace_operator(mesh, fem.condense(A, Kd))
    B = fem.trace_rhs(mesh, A, rub, rpi)
    lam = np.random.default_rng(0).standard_normal(mesh.n_trace)
    ub, _pi = fem.reconstruct(mesh, A, Kd, lam, rub, rpi)
    jump = fem.continuity_jump(mesh, ub)
    resid = B - S @ lam
    np.testing.assert_allclose(jump, resid, rtol=0, atol=1e-10 * np.abs(resid).max())
    lam = np.linalg.solve(S.toarray(), B)
    ub, _pi = fem.reconstruct(mesh, A, Kd, lam, rub, rpi)
    assert np.abs(fem.continuity_jump(mesh, ub)).max() <= 1e-10 * np.abs(ub).max()


def test_pressure_row_and_gradient_structure():
    """G_K = -K_K 1 (Sec. 2.4: the volume term of g and the facet term k share theta on
    each face), and the q32 term vanishes for a horizontally uniform box background on
    the vertical faces."""
    hier, co = _physical_box(2, 3)
    A, Kd, cc = fem.cell_system(hier.meshes[0], co.levels[0], co)
    np.testing.assert_array_equal(A[:, :6, 6], -Kd)
    np.testing.assert_allclose(cc["b"][:, :4], co.tau_rho * co.dt, rtol=1e-14)


def test_box_pressure_row_closed_form():
    """One-point rules on a box hx x hy x hz (Sec. 2.2): q32 gives +-tau_theta dt dtheta/(2 theta_c)
    on top/bottom (theta linear in the layer), M3^rho M3^-1 D gives tau_rho dt on every face,
    and M3^Pi = (1-kappa)/kappa |K| / Pi*."""
    hier, co = _physical_box(2, 3)
    mesh = hier.meshes[0]
    bg = co.levels[0]
    _A, _Kd, cc = fem.cell_system(mesh, bg, co)
    hx = 3.0e5 / 2
    for cell in range(mesh.ncell):
        c, k = divmod(cell, mesh.nlev)
        th0, th1 = bg.theta_lev[c, k], bg.theta_lev[c, k + 1]
        hz = mesh.z_levels[k + 1] - mesh.z_levels[k]
        dq = co.tau_theta * co.dt * (th1 - th0) / (th0 + th1)
        assert cc["b"][cell, 5] == pytest.approx(co.tau_rho * co.dt + dq, rel=1e-12)
        assert cc["b"][cell, 4] == pytest.approx(co.tau_rho * co.dt - dq, rel=1e-12)
        vol = hx * hx * hz
        assert cc["m"][cell] == pytest.approx((1 - co.kappa) / co.kappa * vol / bg.exner[c, k], rel=1e-12)


def test_buoyancy_weight_is_tau_squared_dt_squared_n_squared():
    """In a hydrostatic isothermal atmosphere -c_p d_z Pi* d_z theta* = N^2 = g^2/(c_p T), so
    the vertical mass weight from -Q22 is tau_u tau_theta dt^2 N^2 (up to O(dz^2))."""
    T = 250.0
    hier = I.planar_hierarchy(2, 40, 1.0e5, I.uniform_levels(40, 2000.0), 1)
    co = I.Coefficients([I.isothermal_background(hier.meshes[0], T)], dt=900.0)
    cc = fem.cell_coefficients(hier.meshes[0], co.levels[0], co)
    n2 = I.GRAVITY ** 2 / (I.CP * T)
    want = co.tau_u * co.tau_theta * co.dt ** 2 * n2
    np.testing.assert_allclose(cc["c22"], want, rtol=1e-4)
    assert (cc["c22"] > 0).all()


def test_buoyancy_weight_of_a_constant_n_background_varies_only_with_n():
    """Over a horizontally varying surface temperature, a constant-N hydrostatic background
    still gives -c_p d_z Pi* d_z theta* = N^2 in every cell (theta_s cancels), so the vertical
    weight is tau_u tau_theta dt^2 N^2 everywhere, up to O(dz^2)."""
    N = 0.012
    hier = I.planar_hierarchy(3, 40, 1.0, I.uniform_levels(40, 2000.0), 1)
    mesh = hier.meshes[0]
    bg = I.stratified_background(mesh, brunt=N)
    assert np.ptp(bg.theta_lev[:, 0]) > 5.0                 # the surface really varies
    co = I.Coefficients([bg], dt=900.0)
    cc = fem.cell_coefficients(mesh, bg, co)
    np.testing.assert_allclose(cc["c22"], co.tau_u * co.tau_theta * co.dt ** 2 * N ** 2, rtol=1e-4)
    # and the background is hydrostatic: c_p d_z Pi* = -g / theta* at the level midpoints
    z = mesh.z_levels
    dpi = np.diff(bg.exner_lev, axis=1) / np.diff(z)[None, :]
    theta_mid = np.sqrt(bg.theta_lev[:, 1:] * bg.theta_lev[:, :-1])
    np.testing.assert_allclose(I.CP * dpi, -I.GRAVITY / theta_mid, rtol=1e-4)


def test_local_inverse_matches_extended_precision():
    """A_K^-1 (hence S_K) of physical cubed-sphere cells agrees with a 60-digit inverse to a
    few ulps of each row's scale, although A_K's entries span ~20 orders of magnitude."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    w = I.cubed_sphere(12, 30)
    cells = [0, 29, 31, 500, w.mesh.ncell - 1]
    A, Kd, _cc = fem.cell_system(w.mesh, w.coeffs.levels[0], w.coeffs, cells=cells)
    Ainv = fem.local_inverse(A)
    SK = fem.condense(A, Kd)
    for i in range(len(cells)):
        ex = mp.matrix(A[i].tolist()) ** -1
        exn = np.array([[float(ex[r, c]) for c in range(7)] for r in range(7)])
        scale = np.abs(exn).max(axis=1, keepdims=True)
        assert (np.abs(Ainv[i] - exn) / scale).max() < 1e-14
        exs = exn[:6, :6] * Kd[i][None, :]
        assert (np.abs(SK[i] - exs) / np.abs(exs).max(axis=1, keepdims=True)).max() < 1e-14


def test_trace_row_sums_identity():
    """S 1 = sum_K m_K (A_K^-1)_{u,p} equals the plain row sums of S up to their cancellation
    error, and equals the 60-digit row sums of S_K on sample cells."""
    w = I.cubed_sphere(6, 8, nmg=1)
    A, Kd, _cc = fem.cell_system(w.mesh, w.coeffs.levels[0], w.coeffs)
    SK = fem.condense(A, Kd)
    S = fem.assemble_trace_operator(w.mesh, SK)
    rs = fem.trace_row_sums(w.mesh, A)
    plain = S @ np.ones(w.mesh.n_trace)
    cond = abs(S) @ np.ones(w.mesh.n_trace)
    assert np.all(np.abs(rs - plain) <= 1e-13 * cond)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    for cell in (0, 17, w.mesh.ncell - 1):
        ex = mp.matrix(A[cell].tolist()) ** -1
        exact = [float(sum(ex[i, j] * mp.mpf(Kd[cell, j]) for j in range(6))) for i in range(6)]
        got = A[cell, 6, 6] * fem.local_inverse(A[cell:cell + 1])[0, :6, 6]
        np.testing.assert_allclose(got, exact, rtol=1e-12)


def test_coriolis_block_on_a_box_closed_form():
    """f-plane box, c = tau_u dt 2 Omega zhat: v_f.(c x v_g) couples only the x faces with the
    y faces, C(f,g) = -c/hz * A_f * B_g with A, B = +1/2 on the faces at 1 and -1/2 at 0,
    antisymmetric; rows and columns of the vertical faces stay untouched."""
    hx, hy, hz, c = 0.7, 0.3, 0.05, 2.5
    verts = np.zeros((1, 8, 3))
    for v in range(8):
        verts[0, v] = ((v & 1) * hx, ((v >> 1) & 1) * hy, ((v >> 2) & 1) * hz)
    M0 = fem.local_mass(verts, np.zeros(1), 0)[0][0]
    M1 = fem.local_mass(verts, np.zeros(1), 0, (0.0, 0.0, c))[0][0]
    C = M1 - M0
    half = {0: -0.5, 1: 0.5, 2: 0.5, 3: -0.5}      # local faces: 0 y=0, 1 x=1, 2 y=1, 3 x=0
    want = np.zeros((6, 6))
    for f in (1, 3):
        for g in (0, 2):
            want[f, g] = -c / hz * half[f] * half[g]
            want[g, f] = -want[f, g]
    np.testing.assert_allclose(C, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


def test_rotation_adds_an_antisymmetric_block_and_keeps_the_pressure_operator():
    """On curved sphere cells the Coriolis part of M_K is antisymmetric and the symmetric part
    is the non-rotating M_K; the lumped mass (diagonal and opposite-face entries) and so H
    do not see the rotation."""
    from oracle.pressure_mg import pressure_operator
    w0 = I.cubed_sphere(4, 3, seed=1)
    w1 = I.cubed_sphere(4, 3, seed=1, omega=10 * I.EARTH_OMEGA)
    cells = [0, 5, 40, w0.mesh.ncell - 1]
    M0 = fem.cell_coefficients(w0.mesh, w0.coeffs.levels[0], w0.coeffs, cells)["M"]
    M1 = fem.cell_coefficients(w1.mesh, w1.coeffs.levels[0], w1.coeffs, cells)["M"]
    C = M1 - M0
    assert np.abs(C).max() > 1e-6 * np.abs(M0).max()
    np.testing.assert_allclose(C + C.transpose(0, 2, 1), 0.0, atol=1e-13 * np.abs(M0).max())
    H0 = pressure_operator(w0.mesh, w0.coeffs.levels[0], w0.coeffs)
    H1 = pressure_operator(w1.mesh, w1.coeffs.levels[0], w1.coeffs)
    assert abs(H1 - H0).max() <= 1e-12 * abs(H0).max()


def test_rotating_hybridised_solution_equals_mixed_solution():
    """With Coriolis the cell matrices are not symmetric; hybridise-then-recover still equals
    the dense direct solve of the unhybridised 2x2 system."""
    w = I.cubed_sphere(2, 3, seed=3, omega=20 * I.EARTH_OMEGA)
    Mx, rhs, interior = fem.mixed_system(w.mesh, w.coeffs.levels[0], w.coeffs, w.Rub, w.Rpi)
    x = np.linalg.solve(Mx, rhs)
    nf = len(interior)
    hs = HybridSolver(w.hier, w.coeffs)
    S = hs.S.toarray()
    assert np.abs(S - S.T).max() > 1e-8 * np.abs(S).max()          # really non-symmetric
    lam = np.linalg.solve(S, hs.rhs(w.Rub, w.Rpi))
    ub, pi = hs.reconstruct(lam, w.Rub, w.Rpi)
    np.testing.assert_allclose(pi, x[nf:], rtol=1e-9, atol=1e-10 * np.abs(x[nf:]).max())
    s = fem.face_orientation(w.mesh)
    g = fem.trace_dof_ids(w.mesh)
    u = np.zeros(w.mesh.n_trace)
    u[interior] = x[:nf]
    np.testing.assert_allclose(ub, s * u[g], rtol=1e-9, atol=1e-10 * np.abs(ub).max())
