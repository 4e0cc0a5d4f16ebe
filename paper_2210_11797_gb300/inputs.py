"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds NO arithmetic of the solver method. It only produces the inputs a
caller would hand to the library:

* extruded meshes (column corners, level heights, edge/column incidence tables and the
  horizontal coarsening maps of the pressure multigrid hierarchy);
* background reference profiles (theta*, Exner*) sampled at level heights / cell centres;
* the scalar coefficients (dt, tau_u, tau_rho, tau_theta, c_p, kappa);
* right-hand sides drawn from a counter-based SplitMix64 stream.

Workloads stand in for the paper's LFRic baroclinic-wave runs (Sec. 3.2: C96 cubed
sphere, 30 quadratically stretched layers, 30 km lid), which are not available.

Conventions (fixed, relied on by every consumer):

* columns: planar N x N -> c = j*N + i; cubed sphere C_N -> c = p*N*N + j*N + i;
* cell (c, k) has index c*nlev + k, k = 0 at the ground;
* local faces of a cell: e0..e3 = vertical faces along the column's corners taken
  counter-clockwise seen from above (e0 = corner0->corner1, e1 = corner1->corner2,
  e2 = corner2->corner3, e3 = corner3->corner0), then bottom (4) and top (5);
* reference coordinates: xi along corner0->corner1, eta along corner0->corner3,
  zeta upwards, so e0 <-> eta=0, e1 <-> xi=1, e2 <-> eta=1, e3 <-> xi=0;
* trace dofs: lambda = [lambda^h as [edge][level] | lambda^z as [column][interface 0..L]];
* edge e joins columns edge_cols[e,0] (its owner; the global normal points out of it)
  and edge_cols[e,1], through their local faces edge_face[e,0] and edge_face[e,1].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Physical constants of the synthetic atmosphere (the paper uses a perfect gas, Sec. 2.1).
GRAVITY = 9.80616
CP = 1004.5
R_DRY = 287.05
KAPPA = R_DRY / CP
EARTH_OMEGA = 7.292e-5   # rad/s
EARTH_RADIUS = 6.371e6


# --------------------------------------------------------------------------------------
# Counter-based random numbers: SplitMix64 (Steele, Lea & Flood 2014), one stream per seed.
# --------------------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the SplitMix64 stream started at state=seed."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """U[0,1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """U[-1,1)."""
    return 2.0 * uniform01(seed, n) - 1.0


def normal(seed: int, n: int) -> np.ndarray:
    """N(0,1) by the Box-Muller transform on consecutive pairs of U[0,1) draws."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = 1.0 - u[0::2], u[1::2]  # u1 in (0,1]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:n]


# --------------------------------------------------------------------------------------
# Meshes
# --------------------------------------------------------------------------------------
@dataclass
class ExtrudedMesh:
    geometry: int            # 0 planar (doubly periodic), 1 cubed sphere
    ncol: int
    nlev: int
    nedge: int
    radius: float            # sphere only (0 for planar)
    corners: np.ndarray      # [ncol,4,3] planar (x,y,0) unwrapped per column, or unit vectors
    z_levels: np.ndarray     # [nlev+1], z_0 = 0
    col_edges: np.ndarray    # [ncol,4] int32 edge id of local faces e0..e3
    edge_cols: np.ndarray    # [nedge,2] int32
    edge_face: np.ndarray    # [nedge,2] int8
    n_per_side: int = 0      # N of the N x N panel(s)

    @property
    def ncell(self) -> int:
        return self.ncol * self.nlev

    @property
    def n_trace_h(self) -> int:
        return self.nedge * self.nlev

    @property
    def n_trace_z(self) -> int:
        return self.ncol * (self.nlev + 1)

    @property
    def n_trace(self) -> int:
        return self.n_trace_h + self.n_trace_z


@dataclass
class MeshHierarchy:
    meshes: list                    # finest first
    parents: list = field(default_factory=list)  # parents[l]: [ncol_l] column of level l+1

    @property
    def nmg(self) -> int:
        return len(self.meshes)


def uniform_levels(nlev: int, top: float) -> np.ndarray:
    return top * np.arange(nlev + 1, dtype=np.float64) / nlev


def quadratic_levels(nlev: int, top: float) -> np.ndarray:
    """z_k = top * (k/L)^2: spacing growing quadratically with height (Sec. 3.2)."""
    s = np.arange(nlev + 1, dtype=np.float64) / nlev
    return top * s * s


def planar_periodic_mesh(n: int, nlev: int, length: float, z_levels: np.ndarray) -> ExtrudedMesh:
    """Doubly periodic n x n columns on [0,length]^2. Column (i,j) owns its south (e0) and
    west (e3) edges: edge 2c is the south edge of c, edge 2c+1 its west edge."""
    if n < 2:
        raise ValueError("a periodic mesh needs at least 2 columns per direction")
    h = length / n
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    ii, jj = ii.ravel(), jj.ravel()            # c = j*n + i
    ncol = n * n
    corners = np.zeros((ncol, 4, 3))
    corners[:, 0, 0], corners[:, 0, 1] = ii * h, jj * h
    corners[:, 1, 0], corners[:, 1, 1] = (ii + 1) * h, jj * h
    corners[:, 2, 0], corners[:, 2, 1] = (ii + 1) * h, (jj + 1) * h
    corners[:, 3, 0], corners[:, 3, 1] = ii * h, (jj + 1) * h
    col = lambda i, j: (j % n) * n + (i % n)
    c = np.arange(ncol)
    south = col(ii, jj - 1)
    west = col(ii - 1, jj)
    east = col(ii + 1, jj)
    north = col(ii, jj + 1)
    nedge = 2 * ncol
    edge_cols = np.zeros((nedge, 2), np.int32)
    edge_face = np.zeros((nedge, 2), np.int8)
    edge_cols[0::2, 0], edge_cols[0::2, 1] = c, south
    edge_face[0::2, 0], edge_face[0::2, 1] = 0, 2
    edge_cols[1::2, 0], edge_cols[1::2, 1] = c, west
    edge_face[1::2, 0], edge_face[1::2, 1] = 3, 1
    col_edges = np.stack([2 * c, 2 * east + 1, 2 * north, 2 * c + 1], axis=1).astype(np.int32)
    return ExtrudedMesh(0, ncol, nlev, nedge, 0.0, corners, np.asarray(z_levels, np.float64),
                        col_edges, edge_cols, edge_face, n)


_PANELS = [  # (centre, e1, e2) with e1 x e2 = centre: counter-clockwise seen from outside
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((0, 1, 0), (-1, 0, 0), (0, 0, 1)),
    ((-1, 0, 0), (0, -1, 0), (0, 0, 1)),
    ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
    ((0, 0, 1), (0, 1, 0), (-1, 0, 0)),
    ((0, 0, -1), (0, 1, 0), (1, 0, 0)),
]


def _balanced_owner(ncol: int, col_nbr_edges: list) -> np.ndarray:
    """Orient the 4-regular column graph along an Euler circuit (Hierholzer), so that
    every column owns exactly two of its four edges. col_nbr_edges[c] = [(edge, nbr)]."""
    nedge = sum(len(x) for x in col_nbr_edges) // 2
    owner = -np.ones(nedge, np.int64)
    ptr = [0] * ncol
    stack = [0]
    while stack:
        u = stack[-1]
        adj = col_nbr_edges[u]
        while ptr[u] < len(adj) and owner[adj[ptr[u]][0]] >= 0:
            ptr[u] += 1
        if ptr[u] == len(adj):
            stack.pop()
            continue
        e, v = adj[ptr[u]]
        owner[e] = u
        stack.append(v)
    return owner


def cubed_sphere_mesh(n: int, nlev: int, z_levels: np.ndarray,
                      radius: float = EARTH_RADIUS) -> ExtrudedMesh:
    """Equiangular gnomonic cubed sphere C_n (6 n^2 columns); corners are unit vectors.
    Edges are numbered by owning column (two per column, Euler-circuit orientation)."""
    t = np.tan(-math.pi / 4 + np.arange(n + 1) * (math.pi / (2 * n)))
    t[0] = -1.0
    for i in range((n + 1) // 2):       # exact antisymmetry t[n-i] = -t[i], so points on
        t[n - i] = -t[i]                # panel boundaries come out bit-identical from
    if n % 2 == 0:                      # both panels that share them
        t[n // 2] = 0.0
    keys = {}
    vid = np.zeros((6, n + 1, n + 1), np.int64)
    for p, (cen, e1, e2) in enumerate(_PANELS):
        cen, e1, e2 = (np.array(v, np.float64) for v in (cen, e1, e2))
        for j in range(n + 1):
            for i in range(n + 1):
                v = cen + t[i] * e1 + t[j] * e2
                v = v / np.sqrt(v @ v)
                key = tuple(np.round(v * 1e12).astype(np.int64))
                if key not in keys:
                    keys[key] = (len(keys), v)
                vid[p, i, j] = keys[key][0]
    verts = np.zeros((len(keys), 3))
    for k_, (idx, v) in keys.items():
        verts[idx] = v
    ncol = 6 * n * n
    corner_vid = np.zeros((ncol, 4), np.int64)
    for p in range(6):
        for j in range(n):
            for i in range(n):
                c = p * n * n + j * n + i
                corner_vid[c] = (vid[p, i, j], vid[p, i + 1, j], vid[p, i + 1, j + 1], vid[p, i, j + 1])
    corners = verts[corner_vid]
    # edges: dedup by vertex pair
    ekey = {}
    col_face_edge = np.zeros((ncol, 4), np.int64)
    edge_inc = []
    for c in range(ncol):
        for f in range(4):
            a, b = corner_vid[c, f], corner_vid[c, (f + 1) % 4]
            key = (min(a, b), max(a, b))
            if key not in ekey:
                ekey[key] = len(edge_inc)
                edge_inc.append([])
            e = ekey[key]
            edge_inc[e].append((c, f))
            col_face_edge[c, f] = e
    nedge = len(edge_inc)
    assert nedge == 2 * ncol and all(len(x) == 2 for x in edge_inc)
    nbrs = [[] for _ in range(ncol)]
    for e, ((c0, _f0), (c1, _f1)) in enumerate(edge_inc):
        nbrs[c0].append((e, c1))
        nbrs[c1].append((e, c0))
    owner = _balanced_owner(ncol, nbrs)
    # renumber edges by (owner, owner's local face)
    own_face = np.array([f if c == owner[e] else g for e, ((c, f), (_d, g)) in enumerate(edge_inc)])
    order = np.lexsort((own_face, owner))
    new_id = np.empty(nedge, np.int64)
    new_id[order] = np.arange(nedge)
    edge_cols = np.zeros((nedge, 2), np.int32)
    edge_face = np.zeros((nedge, 2), np.int8)
    for e_old, ((c0, f0), (c1, f1)) in enumerate(edge_inc):
        e = new_id[e_old]
        if c0 == owner[e_old]:
            edge_cols[e], edge_face[e] = (c0, c1), (f0, f1)
        else:
            edge_cols[e], edge_face[e] = (c1, c0), (f1, f0)
    col_edges = new_id[col_face_edge].astype(np.int32)
    return ExtrudedMesh(1, ncol, nlev, nedge, float(radius), corners,
                        np.asarray(z_levels, np.float64), col_edges, edge_cols, edge_face, n)


def planar_hierarchy(n: int, nlev: int, length: float, z_levels, nmg: int) -> MeshHierarchy:
    meshes, parents = [], []
    for l in range(nmg):
        m = n >> l
        meshes.append(planar_periodic_mesh(m, nlev, length, z_levels))
        if l + 1 < nmg:
            ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
            parents.append(((jj.ravel() // 2) * (m // 2) + ii.ravel() // 2).astype(np.int32))
    return MeshHierarchy(meshes, parents)


def sphere_hierarchy(n: int, nlev: int, z_levels, nmg: int, radius=EARTH_RADIUS) -> MeshHierarchy:
    meshes, parents = [], []
    for l in range(nmg):
        m = n >> l
        meshes.append(cubed_sphere_mesh(m, nlev, z_levels, radius))
        if l + 1 < nmg:
            p, rem = np.divmod(np.arange(6 * m * m), m * m)
            j, i = np.divmod(rem, m)
            mc = m // 2
            parents.append((p * mc * mc + (j // 2) * mc + i // 2).astype(np.int32))
    return MeshHierarchy(meshes, parents)


def mg_levels_for(n: int, want: int = 4) -> int:
    """Pressure-multigrid levels: at most `want`, while the panel side stays even."""
    levels = 1
    while levels < want and n % 2 == 0 and n >= 4:
        n //= 2
        levels += 1
    return levels


# --------------------------------------------------------------------------------------
# Background state and coefficients
# --------------------------------------------------------------------------------------
@dataclass
class LevelBackground:
    theta_lev: np.ndarray    # [ncol, nlev+1]  theta* at level heights (W_theta dofs)
    exner_lev: np.ndarray    # [ncol, nlev+1]  Exner* projected to W_theta (hat Pi*)
    exner: np.ndarray        # [ncol, nlev]    Exner* at cell centres (W3 dofs)


@dataclass
class Coefficients:
    levels: list             # LevelBackground per multigrid level (finest first)
    dt: float = 1.0
    tau_u: float = 0.5
    tau_rho: float = 0.5
    tau_theta: float = 0.5
    cp: float = CP
    kappa: float = KAPPA
    preset: int = 0          # 0 physical, 1 constant-coefficient Helmholtz
    sigma: float = 0.0       # preset 1 shift: m_K = sigma |K|
    omega: float = 0.0       # rotation rate (rad/s) about the polar axis / the vertical


def isothermal_background(mesh: ExtrudedMesh, temperature: float = 250.0) -> LevelBackground:
    """Hydrostatic isothermal atmosphere: Pi*(z) = exp(-g z / (c_p T)), theta* = T / Pi*."""
    z = mesh.z_levels
    zc = 0.5 * (z[1:] + z[:-1])
    pi_lev = np.exp(-GRAVITY * z / (CP * temperature))
    pi_c = np.exp(-GRAVITY * zc / (CP * temperature))
    ones = np.ones((mesh.ncol, 1))
    return LevelBackground(ones * (temperature / pi_lev), ones * pi_lev, ones * pi_c)


def stratified_background(mesh: ExtrudedMesh, brunt: float = 0.012, theta_surface: float = 290.0,
                          theta_amp: float = 20.0) -> LevelBackground:
    """Hydrostatic atmosphere of constant Brunt-Vaisala frequency N over a horizontally varying
    surface: theta*(z) = theta_s exp(N^2 z / g), Pi*(z) = 1 - g^2 / (c_p theta_s N^2)
    (1 - exp(-N^2 z / g)), with theta_s = theta_surface - theta_amp sin^2(latitude) on the
    sphere (latitude of the column centre) and theta_surface - theta_amp (1 + cos 2 pi x
    cos 2 pi y) / 2 on the unit plane."""
    z = mesh.z_levels
    zc = 0.5 * (z[1:] + z[:-1])
    centre = mesh.corners.mean(axis=1)
    if mesh.geometry == 1:
        s = centre[:, 2] / np.linalg.norm(centre, axis=1)
        ts = theta_surface - theta_amp * s * s
    else:
        ts = theta_surface - theta_amp * 0.5 * (1.0 + np.cos(2 * math.pi * centre[:, 0]) *
                                                 np.cos(2 * math.pi * centre[:, 1]))
    n2g = brunt * brunt / GRAVITY
    ts = ts[:, None]

    def exner(height):
        return 1.0 - GRAVITY * GRAVITY / (CP * ts * brunt * brunt) * (1.0 - np.exp(-n2g * height[None, :]))

    return LevelBackground(ts * np.exp(n2g * z[None, :]), exner(z), exner(zc))


def unit_background(mesh: ExtrudedMesh) -> LevelBackground:
    ones_l = np.ones((mesh.ncol, mesh.nlev + 1))
    return LevelBackground(ones_l.copy(), ones_l.copy(), np.ones((mesh.ncol, mesh.nlev)))


def acoustic_dt(n: int, courant: float, temperature: float = 250.0,
                radius: float = EARTH_RADIUS) -> float:
    """dt = Courant * mean spacing / sound speed, mean spacing = sqrt(4 pi R^2 / (6 N^2))."""
    dx = math.sqrt(4.0 * math.pi * radius * radius / (6.0 * n * n))
    cs = math.sqrt(CP / (CP - R_DRY) * R_DRY * temperature)
    return courant * dx / cs


# --------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    hier: MeshHierarchy
    coeffs: Coefficients
    Rub: np.ndarray          # [C,6] broken-velocity residual, order [column][level][face]
    Rpi: np.ndarray          # [C]   pressure residual
    tol: float

    @property
    def mesh(self) -> ExtrudedMesh:
        return self.hier.meshes[0]


def draw_rhs(ncell: int, seed: int, dist: str):
    """R_u^b (6 per cell, [column][level][face]) then R_Pi (1 per cell) from one stream."""
    vals = uniform_pm1(seed, 7 * ncell) if dist == "uniform" else normal(seed, 7 * ncell)
    return vals[: 6 * ncell].reshape(ncell, 6).copy(), vals[6 * ncell:].copy()


def planar_helmholtz(n: int = 16, nlev: int = 8, length: float = 1.0, top: float = 0.1,
                     c_dt: float = 0.05, nmg: int = 2, seed: int = 0, tol: float = 1e-10) -> Workload:
    """Constant-coefficient Helmholtz on a doubly periodic box (shift 1/(c dt)^2)."""
    hier = planar_hierarchy(n, nlev, length, uniform_levels(nlev, top), nmg)
    co = Coefficients([unit_background(m) for m in hier.meshes], dt=1.0, preset=1,
                      sigma=1.0 / (c_dt * c_dt))
    rub, rpi = draw_rhs(hier.meshes[0].ncell, seed, "uniform")
    return Workload(f"planar_helmholtz_{n}x{n}x{nlev}", hier, co, rub, rpi, tol)


def cubed_sphere(n: int, nlev: int = 30, top: float = 30000.0, courant: float = 8.0,
                 temperature: float = 250.0, nmg: int | None = None, seed: int = 0,
                 tol: float = 1e-6, radius: float = EARTH_RADIUS,
                 background: str = "isothermal", omega: float = 0.0) -> Workload:
    """Isothermal (or, with background="stratified", constant-N over a latitude-dependent
    surface temperature) atmosphere on C_n x nlev quadratically stretched levels, N(0,1) RHS."""
    if nmg is None:
        nmg = mg_levels_for(n)
    hier = sphere_hierarchy(n, nlev, quadratic_levels(nlev, top), nmg, radius)
    if background == "stratified":
        bgs = [stratified_background(m) for m in hier.meshes]
    else:
        bgs = [isothermal_background(m, temperature) for m in hier.meshes]
    co = Coefficients(bgs, dt=acoustic_dt(n, courant, temperature, radius), preset=0, omega=omega)
    rub, rpi = draw_rhs(hier.meshes[0].ncell, seed, "normal")
    suffix = ("" if background == "isothermal" else f"_{background}") + ("" if omega == 0.0 else "_rotating")
    return Workload(f"cubed_sphere_C{n}_L{nlev}{suffix}", hier, co, rub, rpi, tol)


def batched_sizes(count: int = 64, seed: int = 3):
    """(N, L) per solve: N then L drawn per solve from one SplitMix64(seed) stream."""
    u = uniform01(seed, 2 * count)
    ns, ls = (12, 24, 32, 48), (10, 30, 50, 70)
    return [(ns[int(u[2 * i] * 4)], ls[int(u[2 * i + 1] * 4)]) for i in range(count)]


# --------------------------------------------------------------------------------------
# Initial weights of the learned coarse model
# --------------------------------------------------------------------------------------
COARSE_MODEL_CHANNELS = 32
COARSE_MODEL_SHAPES = (("W1", (32, 1, 3)), ("W2", (32, 32, 3)), ("M", (32, 3)), ("W3", (1, 32, 3)))


def coarse_model_init(seed: int = 0) -> dict:
    """He-scaled SplitMix64 normals for the convolutions; the horizontal mix starts as the
    identity plus a small positive share of the neighbours (w_c, w_e, w_d) = (1, 0.1, 0.05)."""
    ch = COARSE_MODEL_CHANNELS
    z = normal(seed, ch * 3 + ch * ch * 3 + ch * 3)
    n1, n2 = ch * 3, ch * ch * 3
    return {
        "W1": z[:n1].reshape(ch, 1, 3) * math.sqrt(2.0 / 3.0),
        "W2": z[n1:n1 + n2].reshape(ch, ch, 3) * math.sqrt(2.0 / (3.0 * ch)),
        "M": np.tile(np.array([1.0, 0.1, 0.05]), (ch, 1)),
        "W3": z[n1 + n2:].reshape(1, ch, 3) * math.sqrt(1.0 / (3.0 * ch)),
    }


def flatten_coarse_model(params: dict) -> np.ndarray:
    """The flat FP32 parameter vector of the C ABI: W1, W2, M, W3 in that order."""
    return np.concatenate([np.asarray(params[k], np.float64).reshape(-1) for k, _ in COARSE_MODEL_SHAPES]
                          ).astype(np.float32)


def unflatten_coarse_model(v) -> dict:
    out, o = {}, 0
    for k, shp in COARSE_MODEL_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def panel_patch_columns(n: int, npanel: int, nx: int, ny: int, stride: int | None = None) -> np.ndarray:
    """Column ids of nx x ny patches cut from the regular n x n grid of each panel (column
    p n^2 + j n + i; the planar mesh is one panel): [npatch][nx ny], patch column q = jj nx + ii,
    patch origins every `stride` columns (default: non-overlapping)."""
    sx, sy = (stride or nx), (stride or ny)
    out = []
    for p in range(npanel):
        for j0 in range(0, n - ny + 1, sy):
            for i0 in range(0, n - nx + 1, sx):
                jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
                out.append((p * n * n + (j0 + jj) * n + (i0 + ii)).reshape(-1))
    return np.asarray(out, np.int32)


def random_panel_patches(n: int, npanel: int, nx: int, ny: int, count: int, npairs: int, seed: int):
    """`count` random nx x ny patches inside a panel of the regular n x n grid (as in
    panel_patch_columns): per patch a pair index in [0, npairs), a panel, and an origin
    (i0, j0) with the whole patch inside the panel, drawn in that order from one
    SplitMix64(seed) stream. Returns (pair [count] int32, cols [count][nx ny] int32)."""
    u = uniform01(seed, 4 * count)
    pair = np.minimum((u[0::4] * npairs).astype(np.int64), npairs - 1)
    panel = np.minimum((u[1::4] * npanel).astype(np.int64), npanel - 1)
    i0 = np.minimum((u[2::4] * (n - nx + 1)).astype(np.int64), n - nx)
    j0 = np.minimum((u[3::4] * (n - ny + 1)).astype(np.int64), n - ny)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    cols = (panel[:, None] * n * n + (j0[:, None] + jj.reshape(1, -1)) * n + (i0[:, None] + ii.reshape(1, -1)))
    return pair.astype(np.int32), cols.astype(np.int32)
