"""Seeded synthetic inputs: linear-tet casting/mold meshes and their problem data.

This module only *builds inputs* (coordinates, connectivity, material ids,
boundary faces, initial temperatures, permutations).  It holds none of the
method's arithmetic: no element matrices, no capacities, no enthalpy relation.
Both the CUDA path and the FP64 oracle consume what it produces.

The paper's own meshes (six casting+mold cases, Section 5, Table 2) are not
available, so every workload is a jittered structured hex grid, each hex split
into the 6 Kuhn (Freudenthal) tetrahedra along its main diagonal, with
materials tagged by tet centroid.  All randomness comes from
``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

# Material table rows: (rho, c, k, latent, T_solidus, T_liquidus).
# The alloy is the Al-like casting alloy of the unit-cube and casting
# workloads; steel is the mold / core material (no phase change).
ALLOY = (2700.0, 900.0, 150.0, 3.9e5, 821.0, 913.0)
STEEL = (7800.0, 460.0, 30.0, 0.0, 0.0, 0.0)

T_POUR = 973.0     # alloy pouring temperature, Eq. 2
T_MOLD = 300.0     # mold initial temperature
T_AMB = 300.0      # ambient of the Robin faces, Eq. 4
H_AMB = 1000.0     # heat-transfer coefficient of the Robin faces, Eq. 4


@dataclasses.dataclass
class Problem:
    """A complete heat-conduction problem on a linear-tet mesh (Section 3)."""
    xyz: np.ndarray          # [N,3] float64, metres
    tets: np.ndarray         # [E,4] int32, 0-based node ids (either orientation)
    mat: np.ndarray          # [E] int32 material id
    materials: np.ndarray    # [M,6] float64 rows (rho, c, k, latent, Ts, Tl)
    faces: np.ndarray        # [F,3] int32 Robin faces (node ids)
    h: np.ndarray            # [F] float64 W/m^2K
    t_inf: np.ndarray        # [F] float64 K
    q: np.ndarray            # [F] float64 W/m^2 (prescribed outward flux)
    T0: np.ndarray           # [N] float64 initial temperature, Eq. 2
    dir_nodes: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros(0, np.int32))   # Dirichlet nodes, Eq. 3
    dir_T: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros(0, np.float64))
    # cast-mold interface (Eq. 8): two face lists lying on each other without
    # matching nodes, with their interface coefficients
    iface_a: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros((0, 3), np.int32))
    iface_b: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros((0, 3), np.int32))
    h_ia: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.float64))
    h_ib: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.float64))
    # temperature-dependent conductivity: (material, T points, k points)
    # tables, piecewise linear, evaluated at an element's mean temperature
    k_tables: tuple = ()
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.faces.shape[0])


def rng_of(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# Structured grid -> Kuhn tetrahedra
# --------------------------------------------------------------------------

# The six Kuhn tets of the unit cube along the diagonal (0,0,0)-(1,1,1): one
# per ordering of the three axes; each walks 000 -> +e_p0 -> +e_p1 -> 111.
def _kuhn_corner_offsets() -> np.ndarray:
    out = []
    for perm in itertools.permutations(range(3)):
        p = [0, 0, 0]
        path = [tuple(p)]
        for ax in perm:
            p[ax] = 1
            path.append(tuple(p))
        out.append(path)
    return np.asarray(out, dtype=np.int64)  # [6,4,3]


_KUHN = _kuhn_corner_offsets()


def box_grid(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0,
             lz: float = 1.0, jitter: float = 0.0, seed: int | None = None):
    """Nodes and Kuhn tets of an nx x ny x nz hex grid on [0,lx]x[0,ly]x[0,lz].

    Node (i, j, k) has id i + (nx+1) (j + (ny+1) k); hex (i, j, k) has id
    i + nx (j + ny k) and owns tets 6 id .. 6 id + 5.  ``jitter`` moves every
    interior node by an independent uniform offset in [-jitter, +jitter] x
    spacing along each axis (boundary nodes stay on the box so the Robin faces
    stay planar).  Returns (xyz, tets, hex_index, node_flags) where node_flags
    has bit 2*a (low) / 2*a+1 (high) set for a node on the low / high
    boundary plane of axis a.
    """
    sx, sy = nx + 1, (nx + 1) * (ny + 1)
    n_nodes = sy * (nz + 1)
    node = np.arange(n_nodes, dtype=np.int64)
    ii = node % sx
    jj = (node // sx) % (ny + 1)
    kk = node // sy
    h = np.array([lx / nx, ly / ny, lz / nz])
    xyz = np.empty((n_nodes, 3), dtype=np.float64)
    xyz[:, 0] = ii * h[0]
    xyz[:, 1] = jj * h[1]
    xyz[:, 2] = kk * h[2]
    flags = ((ii == 0) * 1 | (ii == nx) * 2 | (jj == 0) * 4 | (jj == ny) * 8
             | (kk == 0) * 16 | (kk == nz) * 32).astype(np.int32)
    del ii, jj, kk, node
    if jitter > 0.0:
        rng = rng_of(0 if seed is None else seed)
        interior = np.nonzero(flags == 0)[0]
        d = rng.uniform(-jitter, jitter, size=(interior.size, 3)) * h
        xyz[interior] += d
    nh = nx * ny * nz
    hx = np.arange(nh, dtype=np.int64)
    base = (hx % nx) + sx * ((hx // nx) % ny) + sy * (hx // (nx * ny))
    base = base.astype(np.int32)
    del hx
    tets = np.empty((nh, 6, 4), dtype=np.int32)
    for t in range(6):
        for c in range(4):
            o = _KUHN[t, c]
            tets[:, t, c] = base + int(o[0] + sx * o[1] + sy * o[2])
    hex_index = np.repeat(np.arange(nh, dtype=np.int32), 6)
    return xyz, tets.reshape(-1, 4), hex_index, flags


_FACE_OMIT = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])


def box_boundary_faces(tets: np.ndarray, node_flags: np.ndarray,
                       plane_mask: int = 63) -> np.ndarray:
    """Tet faces lying on the box boundary planes selected by ``plane_mask``.

    A face is on the boundary exactly when its three nodes share one boundary
    plane (no interior face of a box grid lies in a boundary plane).  Faces
    are listed by omitted corner (0..3), then by tet.
    """
    # only tets with a boundary node can own a boundary face
    cand = np.nonzero((node_flags[tets] & plane_mask).any(axis=1))[0]
    sub = tets[cand]
    out = []
    for omit in _FACE_OMIT:
        f = sub[:, omit]
        common = (node_flags[f[:, 0]] & node_flags[f[:, 1]]
                  & node_flags[f[:, 2]] & plane_mask)
        out.append(f[common != 0])
    return np.concatenate(out, axis=0).astype(np.int32)


def centroids(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    c = np.zeros((tets.shape[0], 3))
    for k in range(4):
        c += xyz[tets[:, k]]
    return c * 0.25


def _node_touches(n_nodes: int, tets: np.ndarray, elem_mask: np.ndarray) -> np.ndarray:
    touch = np.zeros(n_nodes, dtype=bool)
    touch[tets[elem_mask].ravel()] = True
    return touch


def _robin(faces: np.ndarray, h: float = H_AMB, t_inf: float = T_AMB):
    nf = faces.shape[0]
    return (np.full(nf, h), np.full(nf, t_inf), np.zeros(nf))


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def unit_cube(n: int = 20, h: float = H_AMB, jitter: float = 0.0,
              seed: int = 1000) -> Problem:
    """Unit cube, n^3 hexes x 6 Kuhn tets, one alloy, T0 = 973 K, Robin h to
    300 K on every boundary triangle.  n = 20 gives 9,261 nodes, 48,000 tets
    and 4,800 boundary triangles."""
    xyz, tets, _, flags = box_grid(n, n, n, jitter=jitter, seed=seed)
    faces = box_boundary_faces(tets, flags)
    hh, ti, q = _robin(faces, h=h)
    return Problem(xyz=xyz, tets=tets, mat=np.zeros(tets.shape[0], np.int32),
                   materials=np.array([ALLOY]), faces=faces, h=hh, t_inf=ti,
                   q=q, T0=np.full(xyz.shape[0], T_POUR), name=f"unit_cube_{n}")


def flanged_casting(nx: int = 70, ny: int = 70, nz: int = 68,
                    seed: int = 1005, flange_r: float = 0.15,
                    flange_t: float = 0.03, body_r: float = 0.10,
                    body_h: float = 0.30, dims=(0.40, 0.40, 0.50)) -> Problem:
    """Flanged-cylinder alloy casting inside a steel box mold.

    Box mold dims[0] x dims[1] x dims[2] m; the cavity is a cylinder of radius
    body_r and height body_h, axis along z through the box centre, centred in
    z, with a flange disc (radius flange_r, thickness flange_t) at its bottom.
    Tets whose centroid lies in the cavity are alloy (material 0), the rest
    steel (material 1).  Interior nodes are jittered by +-5% of the spacing.
    Alloy-touching nodes start at 973 K, the others at 300 K.  The outer mold
    faces are Robin faces (h = 1000 W/m^2K to 300 K).  The default grid
    70 x 70 x 68 gives 1,999,200 tets.
    """
    lx, ly, lz = dims
    xyz, tets, _, flags = box_grid(nx, ny, nz, lx, ly, lz, jitter=0.05, seed=seed)
    c = centroids(xyz, tets)
    r = np.hypot(c[:, 0] - lx / 2, c[:, 1] - ly / 2)
    z0 = (lz - body_h) / 2
    body = (r <= body_r) & (c[:, 2] >= z0) & (c[:, 2] <= z0 + body_h)
    flange = (r <= flange_r) & (c[:, 2] >= z0) & (c[:, 2] <= z0 + flange_t)
    alloy = body | flange
    mat = np.where(alloy, 0, 1).astype(np.int32)
    faces = box_boundary_faces(tets, flags)
    hh, ti, q = _robin(faces)
    T0 = np.where(_node_touches(xyz.shape[0], tets, alloy), T_POUR, T_MOLD)
    return Problem(xyz=xyz, tets=tets, mat=mat, materials=np.array([ALLOY, STEEL]),
                   faces=faces, h=hh, t_inf=ti, q=q, T0=T0.astype(np.float64),
                   name=f"flanged_casting_{nx}x{ny}x{nz}")


def casting_instance(target_tets: float, seed: int) -> Problem:
    """One procedural casting + mold of about target_tets tets.

    Seeded parameters: 1-3 flanged-cylinder cavities side by side along x
    (body radius 4-8 cm, height 10-25 cm, flange radius 1.3-1.8 x the body
    radius, flange thickness 1-3 cm, 2-5 cm apart), mold wall thickness
    3-8 cm around them.  The hex spacing is chosen so that 6 nx ny nz is
    close to target_tets; interior nodes jittered by 5 %.  Materials,
    initial temperatures and Robin faces as in flanged_casting.
    """
    rng = rng_of(seed)
    k = int(rng.integers(1, 4))
    body_r = rng.uniform(0.04, 0.08)
    body_h = rng.uniform(0.10, 0.25)
    flange_r = body_r * rng.uniform(1.3, 1.8)
    flange_t = rng.uniform(0.01, 0.03)
    gap = rng.uniform(0.02, 0.05)
    wall = rng.uniform(0.03, 0.08)
    lx = 2 * wall + k * 2 * flange_r + (k - 1) * gap
    ly = 2 * wall + 2 * flange_r
    lz = 2 * wall + body_h
    hsz = (lx * ly * lz * 6.0 / float(target_tets)) ** (1.0 / 3.0)
    nx, ny, nz = (max(2, int(round(v / hsz))) for v in (lx, ly, lz))
    xyz, tets, _, flags = box_grid(nx, ny, nz, lx, ly, lz, jitter=0.05, seed=seed + 7)
    c = centroids(xyz, tets)
    z0 = wall
    alloy = np.zeros(tets.shape[0], dtype=bool)
    for j in range(k):
        xc = wall + flange_r + j * (2 * flange_r + gap)
        r = np.hypot(c[:, 0] - xc, c[:, 1] - ly / 2)
        zin = (c[:, 2] >= z0) & (c[:, 2] <= z0 + body_h)
        alloy |= (r <= body_r) & zin
        alloy |= (r <= flange_r) & (c[:, 2] >= z0) & (c[:, 2] <= z0 + flange_t)
    mat = np.where(alloy, 0, 1).astype(np.int32)
    faces = box_boundary_faces(tets, flags)
    hh, ti, q = _robin(faces)
    T0 = np.where(_node_touches(xyz.shape[0], tets, alloy), T_POUR, T_MOLD)
    return Problem(xyz=xyz, tets=tets, mat=mat, materials=np.array([ALLOY, STEEL]),
                   faces=faces, h=hh, t_inf=ti, q=q, T0=T0.astype(np.float64),
                   name=f"casting_instance_{seed}_{nx}x{ny}x{nz}")


def batched_castings(n_inst: int = 256, seed: int = 1009, lo: float = 2.0e4,
                     hi: float = 5.0e5) -> list:
    """n_inst casting instances with sizes log-uniform in [lo, hi] tets
    (about 38M tets in all for the defaults); instance i uses seed + 1 + i."""
    rng = rng_of(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_inst))
    return [casting_instance(float(sz), seed + 1 + i) for i, sz in enumerate(sizes)]


def concat_problems(probs) -> Problem:
    """The disjoint union of several problems (part k's node i becomes node
    offset_k + i; material ids offset by the parts' material counts)."""
    xyz, tets, mat, mats, faces, hh, ti, q, T0, dn, dT = ([] for _ in range(11))
    ia, ib, ha, hb, kts = [], [], [], [], []
    no = mo = 0
    for p in probs:
        kts.extend((mt + mo, Tk, kk) for mt, Tk, kk in p.k_tables)
        ia.append(p.iface_a + no)
        ib.append(p.iface_b + no)
        ha.append(p.h_ia)
        hb.append(p.h_ib)
        xyz.append(p.xyz)
        tets.append(p.tets + no)
        mat.append(p.mat + mo)
        mats.append(p.materials)
        faces.append(p.faces + no)
        hh.append(p.h)
        ti.append(p.t_inf)
        q.append(p.q)
        T0.append(p.T0)
        dn.append(p.dir_nodes + no)
        dT.append(p.dir_T)
        no += p.n_nodes
        mo += p.materials.shape[0]
    return Problem(xyz=np.concatenate(xyz), tets=np.concatenate(tets).astype(np.int32),
                   mat=np.concatenate(mat).astype(np.int32), materials=np.concatenate(mats),
                   faces=np.concatenate(faces).astype(np.int32), h=np.concatenate(hh),
                   t_inf=np.concatenate(ti), q=np.concatenate(q), T0=np.concatenate(T0),
                   dir_nodes=np.concatenate(dn).astype(np.int32), dir_T=np.concatenate(dT),
                   iface_a=np.concatenate(ia).astype(np.int32),
                   iface_b=np.concatenate(ib).astype(np.int32),
                   h_ia=np.concatenate(ha), h_ib=np.concatenate(hb),
                   k_tables=tuple(kt for kt in kts),
                   name="+".join(p.name for p in probs))


def cast_in_mold(n_cast: int = 9, n_mold: int = 8, h_i: float = 2000.0,
                 side: float = 0.4) -> Problem:
    """Cube casting meshed on its own inside a box mold with a cubic hole:
    the two meshes meet at the hole's surface without matching nodes.

    Mold: [0, side]^3 with n_mold hexes per axis (a multiple of 4), steel,
    300 K, the hexes of the middle half [side/4, 3 side/4]^3 removed; Robin h =
    1000 W/m^2K to 300 K on its outer faces.  Casting: that middle cube with
    n_cast hexes per axis, alloy, 973 K.  Interface (Eq. 8): the casting's
    boundary faces (side A) and the hole's faces (side B), both with h_i.
    No jitter, so both face sets lie exactly on the hole's surface.
    """
    if n_mold % 4:
        raise ValueError("n_mold must be a multiple of 4")
    xm, tm, hexm, flm = box_grid(n_mold, n_mold, n_mold, side, side, side)
    q = n_mold // 4
    hi, hj, hk = hexm % n_mold, (hexm // n_mold) % n_mold, hexm // (n_mold * n_mold)
    hole = ((hi >= q) & (hi < 3 * q) & (hj >= q) & (hj < 3 * q) & (hk >= q) & (hk < 3 * q))
    tm = tm[~hole]   # hex_index is per tet
    used = np.unique(tm)
    remap = np.full(xm.shape[0], -1, np.int64)
    remap[used] = np.arange(used.shape[0])
    xm, flm, tm = xm[used], flm[used], remap[tm].astype(np.int32)
    # boundary faces of the mold: faces of exactly one tet; outer ones lie in
    # a box plane, the rest on the hole
    allf = np.concatenate([np.delete(tm, k, axis=1) for k in range(4)])
    key = np.sort(allf, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    bnd = allf[cnt[inv.ravel()] == 1]
    outer = (flm[bnd[:, 0]] & flm[bnd[:, 1]] & flm[bnd[:, 2]]) != 0
    robin, hole_faces = bnd[outer], bnd[~outer]
    lc = side / 2
    xc, tc, _, flc = box_grid(n_cast, n_cast, n_cast, lc, lc, lc)
    xc = xc + side / 4
    cast_faces = box_boundary_faces(tc, flc)
    no = xm.shape[0]
    xyz = np.concatenate([xm, xc])
    tets = np.concatenate([tm, tc + no]).astype(np.int32)
    mat = np.concatenate([np.ones(tm.shape[0], np.int32), np.zeros(tc.shape[0], np.int32)])
    T0 = np.concatenate([np.full(xm.shape[0], T_MOLD), np.full(xc.shape[0], T_POUR)])
    hh, ti, qq = _robin(robin)
    return Problem(xyz=xyz, tets=tets, mat=mat, materials=np.array([ALLOY, STEEL]),
                   faces=robin.astype(np.int32), h=hh, t_inf=ti, q=qq, T0=T0,
                   iface_a=(cast_faces + no).astype(np.int32),
                   iface_b=hole_faces.astype(np.int32),
                   h_ia=np.full(cast_faces.shape[0], h_i), h_ib=np.full(hole_faces.shape[0], h_i),
                   name=f"cast_in_mold_{n_cast}_{n_mold}")


def block_with_cores(n: int = 220, n_cores: int = 32, seed: int = 1007,
                     side: float = 1.0) -> Problem:
    """Alloy block (side^3 m, n^3 hexes, 5% jitter) with seeded spherical
    steel cores.

    Core centres are uniform in the box shrunk by the largest radius, radii
    uniform in [3%, 8%] of the side.  A tet whose centroid falls in any sphere
    is steel (material 1), otherwise alloy (material 0).  Alloy-touching nodes
    start at 973 K, core-only nodes at 300 K.  Robin h = 1000 W/m^2K to 300 K
    on all outer faces.  n = 220 gives 63,888,000 tets and 10,793,861 nodes.
    """
    xyz, tets, _, flags = box_grid(n, n, n, side, side, side, jitter=0.05, seed=seed)
    rng = rng_of(seed + 1)
    radii = rng.uniform(0.03, 0.08, size=n_cores) * side
    centres = rng.uniform(0.08 * side, 0.92 * side, size=(n_cores, 3))
    steel = np.zeros(tets.shape[0], dtype=bool)
    hsz = side / n
    for cc, rr in zip(centres, radii):
        # only the hexes of the sphere's bounding box (one hex of margin for
        # the jitter) can hold a tet whose centroid is inside the sphere
        lo = np.maximum(np.floor((cc - rr) / hsz).astype(int) - 1, 0)
        hi = np.minimum(np.ceil((cc + rr) / hsz).astype(int) + 1, n - 1)
        gi, gj, gk = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                                 np.arange(lo[2], hi[2] + 1), indexing="ij")
        hexes = (gi + n * (gj + n * gk)).ravel()
        cand = (6 * hexes[:, None] + np.arange(6)[None, :]).ravel()
        c = centroids(xyz, tets[cand])
        steel[cand[((c - cc) ** 2).sum(axis=1) <= rr * rr]] = True
    mat = steel.astype(np.int32)
    faces = box_boundary_faces(tets, flags)
    hh, ti, q = _robin(faces)
    T0 = np.where(_node_touches(xyz.shape[0], tets, ~steel), T_POUR, T_MOLD)
    return Problem(xyz=xyz, tets=tets, mat=mat, materials=np.array([ALLOY, STEEL]),
                   faces=faces, h=hh, t_inf=ti, q=q, T0=T0.astype(np.float64),
                   name=f"block_with_cores_{n}")


def random_small(seed: int, nx: int = 5, ny: int = 4, nz: int = 3,
                 n_mat: int = 2, permute: bool = True,
                 robin_fraction: float = 0.7) -> Problem:
    """A small randomised problem for parity tests.

    Jittered box (interior jitter 15% of spacing), random material per hex
    (alloy-like phase-change materials with random ranges, plus steel-like
    materials), random T0 in [300, 1000] K, a random subset of the boundary
    triangles as Robin faces with random h, T_inf and q, and (optionally)
    random node and element permutations.  Nodes shared by phase-change
    materials with different ranges cannot occur: all phase-change materials
    share one (Ts, Tl).
    """
    rng = rng_of(seed)
    lx, ly, lz = rng.uniform(0.05, 0.2, size=3)
    xyz, tets, hexi, flags = box_grid(nx, ny, nz, lx, ly, lz, jitter=0.15, seed=seed)
    ts = rng.uniform(700.0, 850.0)
    tl = ts + rng.uniform(5.0, 120.0)
    mats = []
    for m in range(n_mat):
        if m % 2 == 0:
            mats.append((rng.uniform(2000, 3000), rng.uniform(700, 1000),
                         rng.uniform(50, 200), rng.uniform(1e5, 4e5), ts, tl))
        else:
            mats.append((rng.uniform(7000, 8000), rng.uniform(400, 600),
                         rng.uniform(10, 50), 0.0, 0.0, 0.0))
    hex_mat = rng.integers(0, n_mat, size=nx * ny * nz)
    mat = hex_mat[hexi].astype(np.int32)
    faces = box_boundary_faces(tets, flags)
    keep = rng.random(faces.shape[0]) < robin_fraction
    faces = faces[keep]
    nf = faces.shape[0]
    h = rng.uniform(100.0, 3000.0, size=nf)
    t_inf = rng.uniform(280.0, 400.0, size=nf)
    q = rng.uniform(-2e4, 2e4, size=nf)
    T0 = rng.uniform(300.0, 1000.0, size=xyz.shape[0])
    p = Problem(xyz=xyz, tets=tets, mat=mat, materials=np.array(mats), faces=faces,
                h=h, t_inf=t_inf, q=q, T0=T0, name=f"random_small_{seed}")
    if permute:
        p = permute_nodes(p, rng_of(seed + 17))
        p = permute_elements(p, rng_of(seed + 23))
    return p


# --------------------------------------------------------------------------
# Orderings (inputs to the reordering experiments, Section 5.2)
# --------------------------------------------------------------------------

def permute_nodes(p: Problem, rng: np.random.Generator) -> Problem:
    """Renumber nodes by a random permutation: old node i becomes new[i]."""
    n = p.n_nodes
    new = rng.permutation(n).astype(np.int64)
    inv = np.empty(n, np.int64)
    inv[new] = np.arange(n)
    q = dataclasses.replace(p)
    q.xyz = p.xyz[inv]
    q.tets = new[p.tets].astype(np.int32)
    q.faces = new[p.faces].astype(np.int32)
    q.T0 = p.T0[inv]
    q.dir_nodes = new[p.dir_nodes].astype(np.int32)
    return q


def permute_elements(p: Problem, rng: np.random.Generator) -> Problem:
    perm = rng.permutation(p.n_tets)
    q = dataclasses.replace(p)
    q.tets = p.tets[perm]
    q.mat = p.mat[perm]
    # rotate each tet's corner list so corner order is not always the grid's
    rot = rng.integers(0, 4, size=p.n_tets)
    idx = (np.arange(4)[None, :] + rot[:, None]) % 4
    q.tets = np.take_along_axis(q.tets, idx, axis=1).astype(np.int32)
    return q


def bar(n: int, length: float = 0.5, material=ALLOY, latent: float | None = None):
    """A 1-hex-thick bar of n cubic hexes along x (cross-section
    length/n x length/n); boundary flags returned for choosing BC faces."""
    hsz = length / n
    xyz, tets, _, flags = box_grid(n, 1, 1, length, hsz, hsz)
    mats = np.array([material], dtype=np.float64)
    if latent is not None:
        mats[0, 3] = latent
    return xyz, tets, flags, mats


# --------------------------------------------------------------------------
# Learned surrogate: seeded initial parameters and training geometries
# --------------------------------------------------------------------------

def surrogate_init(shapes, seed: int = 2024) -> np.ndarray:
    """Seeded initial parameters of a network whose flat parameter vector is
    the concatenation of ``shapes`` ((name, shape) pairs; a 2-D shape is a
    weight matrix (out, in), a 1-D shape a bias or a vector).  Weight
    matrices are drawn from N(0, 2 / in) (He initialisation), the last
    layer's vector (name "d2") from N(0, 0.01 / in); biases are 0.  FP32."""
    rng = rng_of(seed)
    out = []
    for name, shape in shapes:
        n = int(np.prod(shape))
        if len(shape) == 2:
            out.append(rng.normal(0.0, np.sqrt(2.0 / shape[1]), size=n))
        elif name == "d2":
            out.append(rng.normal(0.0, np.sqrt(0.01 / shape[0]), size=n))
        else:
            out.append(np.zeros(n))
    return np.concatenate(out).astype(np.float32)


def flanged_variant(seed: int, scale: float = 1.0, nx: int = 70, ny: int = 70,
                    nz: int = 68) -> Problem:
    """A seeded member of the flanged-casting family of ``flanged_casting``:
    body radius 0.07-0.12 m, height 0.22-0.34 m, flange radius 1.2-1.6 x the
    body radius (at most 0.17 m), flange thickness 0.02-0.05 m, axis moved
    by up to 0.02 m in x and y, inside the 0.40 x 0.40 x 0.50 m steel box.
    ``scale`` shrinks the box and every length of the cavity by the same
    factor and the grid to round(scale * (nx, ny, nz)) hexes, so that the
    hex spacing (5.7 x 5.7 x 7.4 mm at the default grid) stays the same;
    scale = 1 gives the 1,999,200-tet meshes of the casting workload."""
    rng = rng_of(seed)
    body_r = rng.uniform(0.07, 0.12)
    body_h = rng.uniform(0.22, 0.34)
    flange_r = min(0.17, body_r * rng.uniform(1.2, 1.6))
    flange_t = rng.uniform(0.02, 0.05)
    off = rng.uniform(-0.02, 0.02, size=2)
    lx, ly, lz = 0.40 * scale, 0.40 * scale, 0.50 * scale
    gx, gy, gz = (max(4, int(round(scale * v))) for v in (nx, ny, nz))
    xyz, tets, _, flags = box_grid(gx, gy, gz, lx, ly, lz, jitter=0.05, seed=seed + 3)
    c = centroids(xyz, tets)
    r = np.hypot(c[:, 0] - lx / 2 - off[0] * scale, c[:, 1] - ly / 2 - off[1] * scale)
    z0 = (lz - body_h * scale) / 2
    body = (r <= body_r * scale) & (c[:, 2] >= z0) & (c[:, 2] <= z0 + body_h * scale)
    flange = (r <= flange_r * scale) & (c[:, 2] >= z0) & (c[:, 2] <= z0 + flange_t * scale)
    alloy = body | flange
    mat = np.where(alloy, 0, 1).astype(np.int32)
    faces = box_boundary_faces(tets, flags)
    hh, ti, q = _robin(faces)
    T0 = np.where(_node_touches(xyz.shape[0], tets, alloy), T_POUR, T_MOLD)
    return Problem(xyz=xyz, tets=tets, mat=mat, materials=np.array([ALLOY, STEEL]),
                   faces=faces, h=hh, t_inf=ti, q=q, T0=T0.astype(np.float64),
                   name=f"flanged_variant_{seed}_{gx}x{gy}x{gz}")


def surrogate_training_set(n: int = 200, seed: int = 3000, lo: float = 0.40,
                           hi: float = 0.60) -> list:
    """n training castings of the flanged family at the casting workload's
    hex spacing, scale uniform in [lo, hi] (about 130k-430k tets each);
    casting i uses seed + i.  The evaluation geometries (seeds from 4000)
    are not among them."""
    rng = rng_of(seed)
    scales = rng.uniform(lo, hi, size=n)
    return [flanged_variant(seed + 1 + i, float(sc)) for i, sc in enumerate(scales)]


def surrogate_eval_set(n: int = 10, seed: int = 4000) -> list:
    """n unseen full-size (1,999,200-tet) castings of the flanged family."""
    return [flanged_variant(seed + i) for i in range(n)]
