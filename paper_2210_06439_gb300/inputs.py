"""Seeded synthetic inputs for the hydro RHS (shared by the tests, the oracle
checks and the benchmark).

This module holds no step of the method (no reconstruction, flux, divergence,
time integration, ghost exchange or reduction).  It only builds initial
states: a counter-based random stream, the field laws of the workloads and
the subgrid layout (offsets, neighbour tables).  Converting primitive initial
data (rho, v, p) to the conserved fields uses the ideal-gas law
E = p/(gamma-1) + rho |v|^2 / 2 and the entropy tracer tau = e_int^(1/gamma).

Random numbers: splitmix64 (Steele, Lea & Flood 2014) of a per-(seed, stream)
key plus the cell counter, mapped to a uniform double in (0, 1] with 53 bits,
and to N(0, 1) by the Box-Muller transform.

Workloads (the paper's runs use 512 leaf subgrids of 8^3 cells in double
precision, Sec. II "Data-Structure" and Sec. V):
  sod_jump       one 8^3 subgrid, noisy x-plane shock tube, 1 species
  periodic_box   512 subgrids of 8^3 tiling a periodic 64^3 box, 5 species
  mixed_levels   4096 subgrids of edge 8/12/16 on three levels, ghosts given
  binary_star    8^3 subgrids tiling an outflow box holding two n=1.5
                 polytropes in a 1e-10 atmosphere, 5 species
Plus the test problems: sod_tube (noise-free, quasi 1-D) and smooth_wave.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import numpy as np

NG = 3
GAMMA = 5.0 / 3.0
ALIGN = 4  # subgrid offsets are multiples of 4 doubles (32 bytes)

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to uint64 counters."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    k = splitmix64(np.array([(seed & 0xFFFFFFFF) << 20 | (stream & 0xFFFFF)], dtype=np.uint64))
    return k[0]


def uniform(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Uniform doubles in (0, 1] for the given cell counters."""
    with np.errstate(over="ignore"):
        h = splitmix64(np.asarray(counter, dtype=np.uint64) + _key(seed, stream))
    return ((h >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """N(0,1) by Box-Muller from streams (2*stream, 2*stream+1)."""
    u1 = uniform(seed, 2 * stream, counter)
    u2 = uniform(seed, 2 * stream + 1, counter)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class Problem:
    """A batch of ghosted subgrids in the library's state layout.

    U      flat float64 array; subgrid s occupies U[off[s] : off[s] + nf*B^3]
           as [field][z][y][x] with B = edge[s] + 6.
    nbr    26 int32 neighbour indices per subgrid (direction (dx,dy,dz) at
           (dz+1)*9 + (dy+1)*3 + (dx+1), minus one above the centre), -1 at
           a domain edge; None when the ghosts are given.
    bc     0 = ghosts given, 1 = periodic, 2 = outflow.
    """

    name: str
    edge: np.ndarray
    off: np.ndarray
    dx: np.ndarray
    level: np.ndarray
    nf: int
    U: np.ndarray
    bc: int = 0
    nbr: np.ndarray | None = None
    grid: tuple = ()
    gamma: float = GAMMA
    meta: dict = field(default_factory=dict)

    @property
    def n_sub(self) -> int:
        return int(self.edge.shape[0])

    @property
    def n_species(self) -> int:
        return self.nf - 6

    @property
    def n_cells(self) -> int:
        return int(np.sum(self.edge.astype(np.int64) ** 3))

    @property
    def rhs_len(self) -> int:
        return int(self.nf * self.n_cells)

    def block(self, s: int) -> np.ndarray:
        """View of subgrid s as [nf, B, B, B] (z, y, x)."""
        B = int(self.edge[s]) + 2 * NG
        return self.U[self.off[s]: self.off[s] + self.nf * B ** 3].reshape(self.nf, B, B, B)

    def interior(self, s: int) -> np.ndarray:
        E = int(self.edge[s])
        return self.block(s)[:, NG:NG + E, NG:NG + E, NG:NG + E]

    def copy(self) -> "Problem":
        p = Problem(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        p.U = self.U.copy()
        return p


def layout_offsets(edge: np.ndarray, nf: int) -> tuple[np.ndarray, int]:
    """Packed subgrid offsets (in doubles), each a multiple of ALIGN."""
    off = np.zeros(edge.shape[0], np.int64)
    o = 0
    for s, E in enumerate(edge):
        off[s] = o
        n = nf * (int(E) + 2 * NG) ** 3
        o += (n + ALIGN - 1) // ALIGN * ALIGN
    return off, o


def nb_slot(dx: int, dy: int, dz: int) -> int:
    n = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
    return n - 1 if n > 13 else n


def tiling_neighbours(nx: int, ny: int, nz: int, periodic) -> np.ndarray:
    """26-entry neighbour table of an nx*ny*nz lexicographic tiling
    (s = (sz*ny + sy)*nx + sx).  periodic: bool or a per-axis triple."""
    if isinstance(periodic, (bool, np.bool_)):
        periodic = (bool(periodic),) * 3
    n = nx * ny * nz
    nbr = np.full((n, 26), -1, np.int32)
    sz, sy, sx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sx, sy, sz = sx.ravel(), sy.ravel(), sz.ravel()
    dims = (nx, ny, nz)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                c = [sx + dx, sy + dy, sz + dz]
                ok = np.ones(n, bool)
                for a in range(3):
                    if periodic[a]:
                        c[a] = c[a] % dims[a]
                    else:
                        ok &= (c[a] >= 0) & (c[a] < dims[a])
                idx = (c[2] * ny + c[1]) * nx + c[0]
                nbr[:, nb_slot(dx, dy, dz)] = np.where(ok, idx, -1)
    return nbr.ravel()


def conserved(rho, vx, vy, vz, p, species, gamma=GAMMA):
    """Conserved fields [6 + ns, ...] from primitive initial data."""
    ei = p / (gamma - 1.0)
    out = [rho, rho * vx, rho * vy, rho * vz, ei + 0.5 * rho * (vx * vx + vy * vy + vz * vz),
           ei ** (1.0 / gamma)]
    out += list(species)
    return np.stack([np.asarray(a, dtype=np.float64) for a in out])


def _tile_global(name, fields, nsub, E, dxv, bc, periodic, gamma=GAMMA, meta=None):
    """Cut global interior fields [nf, Z, Y, X] into ghosted subgrid blocks of
    edge E (ghosts left at zero, to be filled by the ghost exchange)."""
    nf = fields.shape[0]
    nx, ny, nz = nsub
    n = nx * ny * nz
    edge = np.full(n, E, np.int32)
    off, total = layout_offsets(edge, nf)
    U = np.zeros(total)
    B = E + 2 * NG
    # one edge: block s at s * stride (layout_offsets), subgrids in x-fastest
    # order; the interiors are copied in one strided assignment
    stride = total // n
    blocks = U.reshape(n, stride)[:, : nf * B ** 3].reshape(nz, ny, nx, nf, B, B, B)
    blocks[:, :, :, :, NG:NG + E, NG:NG + E, NG:NG + E] = fields.reshape(nf, nz, E, ny, E, nx, E).transpose(
        1, 3, 5, 0, 2, 4, 6)
    nbr = tiling_neighbours(nx, ny, nz, periodic)
    return Problem(name=name, edge=edge, off=off, dx=np.full(n, dxv), level=np.zeros(n, np.int32), nf=nf, U=U,
                   bc=bc, nbr=nbr, grid=(nx, ny, nz), gamma=gamma, meta=meta or {})


# --------------------------------------------------------------------------
# Workload laws
# --------------------------------------------------------------------------

def _noisy_gas_law(seed, counter, gamma=GAMMA, n_species=5):
    """Log-normal density, noisy adiabat, random velocities, random species
    fractions, keyed on integer cell counters."""
    rho = np.exp(0.5 * normal(seed, 1, counter))
    p0 = rho ** gamma
    p = np.maximum(p0 * (1.0 + 0.1 * normal(seed, 2, counter)), 1e-3 * p0)
    cs = np.sqrt(gamma * p / rho)
    v = [0.3 * cs * normal(seed, 3 + i, counter) for i in range(3)]
    if n_species == 0:
        return conserved(rho, v[0], v[1], v[2], p, [], gamma)
    w = np.stack([uniform(seed, 20 + i, counter) for i in range(n_species)])
    w = w / np.sum(w, axis=0)
    return conserved(rho, v[0], v[1], v[2], p, [w[i] * rho for i in range(n_species)], gamma)


def sod_jump(seed: int = 1001) -> Problem:
    """One 8^3 subgrid (dx = 1/8) with given ghosts: rho = p = 1 for x < 1/2,
    rho = 0.125, p = 0.1 beyond, each times (1 + 0.01 N(0,1)); v = 0;
    one species equal to rho."""
    E, B = 8, 8 + 2 * NG
    dxv = 1.0 / E
    g = np.arange(B ** 3, dtype=np.uint64)
    iz, iy, ix = np.unravel_index(np.arange(B ** 3), (B, B, B))
    xc = (ix - NG + 0.5) * dxv
    left = xc < 0.5
    rho = np.where(left, 1.0, 0.125) * (1.0 + 0.01 * normal(seed, 1, g))
    p = np.where(left, 1.0, 0.1) * (1.0 + 0.01 * normal(seed, 2, g))
    z = np.zeros_like(rho)
    U = conserved(rho, z, z, z, p, [rho], GAMMA).reshape(-1)
    edge = np.array([E], np.int32)
    off, total = layout_offsets(edge, 7)
    assert total == U.size
    return Problem("sod_jump_8", edge, off, np.array([dxv]), np.zeros(1, np.int32), 7, U, bc=0)


def periodic_box(seed: int = 1002, nsub: int = 8, E: int = 8, n_species: int = 5) -> Problem:
    """nsub^3 subgrids of E^3 tiling a periodic box of (nsub*E)^3 cells;
    log-normal rho (sigma 0.5), p = rho^gamma (1 + 0.1 N), |v_i| ~ 0.3 c_s N."""
    N = nsub * E
    g = np.arange(N ** 3, dtype=np.uint64)
    fields = _noisy_gas_law(seed, g, GAMMA, n_species).reshape(6 + n_species, N, N, N)
    return _tile_global(f"periodic_box_{N}", fields, (nsub,) * 3, E, 1.0 / N, 1, True)


def mixed_levels(seed: int = 1003, n: int = 4096, n_species: int = 5) -> Problem:
    """n independent subgrids: edge (8, 12, 16)[i mod 3], level (i // 3) mod 3,
    dx = 1/(64 * 2^level); the noisy gas law is evaluated in every ghosted
    cell (ghosts given)."""
    edges = np.array([(8, 12, 16)[i % 3] for i in range(n)], np.int32)
    levels = np.array([(i // 3) % 3 for i in range(n)], np.int32)
    nf = 6 + n_species
    off, total = layout_offsets(edges, nf)
    U = np.zeros(total)
    for E in (8, 12, 16):
        sel = np.nonzero(edges == E)[0]
        B = E + 2 * NG
        cnt = (sel.astype(np.uint64)[:, None] << np.uint64(20)) + np.arange(B ** 3, dtype=np.uint64)[None, :]
        f = _noisy_gas_law(seed, cnt.ravel(), GAMMA, n_species).reshape(nf, sel.size, B ** 3)
        for j, s in enumerate(sel):
            U[off[s]: off[s] + nf * B ** 3] = f[:, j, :].ravel()
    dx = 1.0 / (64.0 * 2.0 ** levels)
    return Problem("mixed_levels", edges, off, dx, levels, nf, U, bc=0)


# --------------------------------------------------------------------------
# Binary star (two n = 1.5 polytropes)
# --------------------------------------------------------------------------

def lane_emden(n: float = 1.5, h: float = 1e-4):
    """Integrates theta'' + 2 theta'/xi + theta^n = 0, theta(0)=1,
    theta'(0)=0 by classical RK4 up to the first zero.  Returns
    (xi grid, theta grid, xi_1, -xi_1^2 theta'(xi_1))."""
    def rhs(x, y):
        th, dth = y
        thn = max(th, 0.0) ** n
        return np.array([dth, -thn - 2.0 * dth / x])
    x0 = 1e-6
    y = np.array([1.0 - x0 * x0 / 6.0, -x0 / 3.0])
    xs, ths = [0.0, x0], [1.0, y[0]]
    x = x0
    while True:
        k1 = rhs(x, y)
        k2 = rhs(x + h / 2, y + h / 2 * k1)
        k3 = rhs(x + h / 2, y + h / 2 * k2)
        k4 = rhs(x + h, y + h * k3)
        yn = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if yn[0] <= 0.0:
            # linear interpolation of the zero crossing
            t = y[0] / (y[0] - yn[0])
            xi1 = x + t * h
            dth1 = y[1] + t * (yn[1] - y[1])
            xs.append(xi1)
            ths.append(0.0)
            return np.array(xs), np.array(ths), xi1, -xi1 * xi1 * dth1
        x += h
        y = yn
        xs.append(x)
        ths.append(y[0])


def binary_star_law(x, y, z, rho_atm=1e-10, R1=0.12, q=0.7, a=0.45, n_species=5):
    """Conserved fields at points (x, y, z) of the unit box: two n=1.5
    polytropes (mass ratio q, radius ~ M^(-1/3)), centres a apart on the x
    axis about the box centre, rotating rigidly about their centre of mass
    with the Kepler rate; still atmosphere rho_atm at the pressure of star 1's
    adiabat.  Species: core (r < R/2) and envelope of each star, atmosphere."""
    n = 1.5
    gamma = 1.0 + 1.0 / n
    xs, ths, xi1, mu1 = lane_emden(n)
    G = 1.0
    rc1 = 1.0
    al1 = R1 / xi1
    M1 = 4.0 * math.pi * rc1 * al1 ** 3 * mu1
    K1 = 4.0 * math.pi * G * al1 ** 2 * rc1 ** (1.0 - 1.0 / n) / (n + 1.0)
    M2 = q * M1
    R2 = R1 * q ** (-1.0 / 3.0)
    al2 = R2 / xi1
    rc2 = M2 / (4.0 * math.pi * al2 ** 3 * mu1)
    K2 = 4.0 * math.pi * G * al2 ** 2 * rc2 ** (1.0 - 1.0 / n) / (n + 1.0)
    x1 = 0.5 - a * M2 / (M1 + M2)
    x2 = 0.5 + a * M1 / (M1 + M2)
    omega = math.sqrt(G * (M1 + M2) / a ** 3)
    rho = np.full(np.shape(x), rho_atm)
    p = np.full(np.shape(x), K1 * rho_atm ** gamma)
    vx = np.zeros(np.shape(x))
    vy = np.zeros(np.shape(x))
    spc = np.zeros((n_species,) + np.shape(x))
    owner = np.full(np.shape(x), 4)
    for (xc, R, al, rc, K, base) in ((x1, R1, al1, rc1, K1, 0), (x2, R2, al2, rc2, K2, 2)):
        r = np.sqrt((x - xc) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        inside = r < R
        th = np.interp(r / al, xs, ths)
        rs = np.maximum(rc * np.maximum(th, 0.0) ** n, rho_atm)
        rho = np.where(inside, rs, rho)
        p = np.where(inside, K * rs ** gamma, p)
        vx = np.where(inside, -omega * (y - 0.5), vx)
        vy = np.where(inside, omega * (x - 0.5), vy)
        owner = np.where(inside, np.where(r < 0.5 * R, base, base + 1), owner)
    for i in range(n_species):
        spc[i] = np.where(owner == i, rho, 0.0)
    return conserved(rho, vx, vy, np.zeros(np.shape(x)), p, list(spc), gamma), dict(
        M1=M1, M2=M2, R1=R1, R2=R2, K1=K1, K2=K2, omega=omega, xi1=xi1, mu1=mu1)


def binary_star(nsub: int = 16, E: int = 8, n_species: int = 5) -> Problem:
    """nsub^3 subgrids of E^3 tiling the unit box (outflow edges)."""
    N = nsub * E
    c = (np.arange(N) + 0.5) / N
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    fields, meta = binary_star_law(xx, yy, zz, n_species=n_species)
    return _tile_global(f"binary_star_{N}", fields, (nsub,) * 3, E, 1.0 / N, 2, False, meta=meta)


# --------------------------------------------------------------------------
# Test problems
# --------------------------------------------------------------------------

def sod_tube(ncells: int, E: int = 8, gamma: float = GAMMA) -> Problem:
    """Noise-free Sod tube along x over [0, 1): ncells x E x E cells, outflow
    in x, periodic in y and z, diaphragm at x = 1/2, no species."""
    c = (np.arange(ncells) + 0.5) / ncells
    left = c < 0.5
    rho1 = np.where(left, 1.0, 0.125)
    p1 = np.where(left, 1.0, 0.1)
    shape = (E, E, ncells)
    rho = np.broadcast_to(rho1, shape)
    p = np.broadcast_to(p1, shape)
    z = np.zeros(shape)
    fields = conserved(rho, z, z, z, p, [], gamma)
    return _tile_global(f"sod_tube_{ncells}", fields, (ncells // E, 1, 1), E, 1.0 / ncells, 2,
                        (False, True, True), gamma)


def smooth_wave(ncells: int, kvec=(1, 0, 0), E: int = 8, amp: float = 0.2, v=None, p0: float = 1.0) -> Problem:
    """Periodic density wave rho = 1 + amp sin 2 pi (k . x) advected at
    constant velocity v (default v = k) and pressure p0.  The box has ncells
    cells along every axis with k != 0 and E cells along the others."""
    kvec = tuple(int(k) for k in kvec)
    v = tuple(float(k) for k in kvec) if v is None else tuple(v)
    dims = [ncells if kvec[a] != 0 else E for a in range(3)]
    h = 1.0 / ncells
    cs = [(np.arange(dims[a]) + 0.5) * h for a in range(3)]
    zz, yy, xx = np.meshgrid(cs[2], cs[1], cs[0], indexing="ij")
    rho = 1.0 + amp * np.sin(2.0 * math.pi * (kvec[0] * xx + kvec[1] * yy + kvec[2] * zz))
    one = np.ones_like(rho)
    fields = conserved(rho, v[0] * one, v[1] * one, v[2] * one, p0 * one, [rho.copy()])
    nsub = (dims[0] // E, dims[1] // E, dims[2] // E)
    return _tile_global(f"smooth_wave_{ncells}", fields, nsub, E, h, 1, True,
                        meta=dict(kvec=kvec, v=v, amp=amp))


def smooth_wave_exact(prob: Problem, t: float) -> np.ndarray:
    """Exact density of smooth_wave at time t on prob's interior cells,
    returned per subgrid in the RHS layout order of field 0."""
    kvec, v, amp = prob.meta["kvec"], prob.meta["v"], prob.meta["amp"]
    nx, ny, nz = prob.grid
    E = int(prob.edge[0])
    h = float(prob.dx[0])
    out = []
    c = (np.arange(E) + 0.5) * h
    for sz in range(nz):
        for sy in range(ny):
            for sx in range(nx):
                zz, yy, xx = np.meshgrid(sz * E * h + c, sy * E * h + c, sx * E * h + c, indexing="ij")
                ph = kvec[0] * (xx - v[0] * t) + kvec[1] * (yy - v[1] * t) + kvec[2] * (zz - v[2] * t)
                out.append(1.0 + amp * np.sin(2.0 * math.pi * ph))
    return np.stack(out)


def uniform_state(nsub=(2, 2, 2), E: int = 8, n_species: int = 2, rho=1.3, v=(0.7, -0.4, 0.25), p=0.9,
                  periodic=True) -> Problem:
    """A uniform state (every cell identical) on a tiling, ghosts to be filled."""
    dims = [nsub[a] * E for a in range(3)]
    shape = (dims[2], dims[1], dims[0])
    one = np.ones(shape)
    fields = conserved(rho * one, v[0] * one, v[1] * one, v[2] * one, p * one,
                       [rho * (i + 1) / (n_species + 1) * one for i in range(n_species)])
    return _tile_global("uniform", fields, tuple(nsub), E, 1.0 / dims[0], 1 if periodic else 2, periodic)


WORKLOADS = {
    "sod_jump_8": sod_jump,
    "periodic_box_64": periodic_box,
    "mixed_levels": mixed_levels,
    "binary_star_128": lambda: binary_star(16),
    "binary_star_256": lambda: binary_star(32),
}


def sedov_blast(nsub: int = 8, E: int = 8, e_blast: float = 1.0, rho0: float = 1.0, p_amb: float = 1e-5,
                r_dep_cells: float = 2.0) -> Problem:
    """Sedov-Taylor point explosion (the paper's hydro-only test scenario,
    Sec. V-C): a uniform cold gas rho0, p_amb at rest in the unit box (outflow
    edges), with energy e_blast deposited as thermal energy, evenly, in the
    cells whose centres lie within r_dep_cells cells of the box centre."""
    N = nsub * E
    c = (np.arange(N) + 0.5) / N
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt((xx - 0.5) ** 2 + (yy - 0.5) ** 2 + (zz - 0.5) ** 2)
    hot = r < r_dep_cells / N
    vol = hot.sum() / N ** 3
    p = np.where(hot, (GAMMA - 1.0) * e_blast / vol, p_amb)
    z = np.zeros_like(r)
    fields = conserved(np.full_like(r, rho0), z, z, z, p, [np.where(hot, rho0, 0.0)])
    return _tile_global(f"sedov_{N}", fields, (nsub,) * 3, E, 1.0 / N, 2, False,
                        meta=dict(e_blast=e_blast, rho0=rho0))


def amr_wave(n_coarse: int = 4, E: int = 8, amp: float = 0.2) -> Problem:
    """The two-level geometry of amr_box (periodic) filled with a smooth
    density wave rho = 1 + amp sin 2 pi x advected at v = (1, 0, 0), p = 1,
    one species equal to rho: the wave crosses the coarse-fine faces.  Values
    are taken at cell centres.  meta as amr_box, plus amp."""
    q = amr_box(seed=1, n_coarse=n_coarse, E=E, n_species=1, periodic=True)
    B = E + 2 * NG
    i = np.arange(E)
    lev, org = q.meta["level"], q.meta["origin"]
    q.U[:] = 0.0
    for k in range(q.n_sub):
        h = float(q.dx[k])
        zz, yy, xx = np.meshgrid((org[k, 2] + i + 0.5) * h, (org[k, 1] + i + 0.5) * h, (org[k, 0] + i + 0.5) * h,
                                 indexing="ij")
        rho = 1.0 + amp * np.sin(2.0 * math.pi * xx)
        one = np.ones_like(rho)
        f = conserved(rho, one, 0.0 * one, 0.0 * one, one, [rho.copy()])
        q.U[q.off[k]: q.off[k] + q.nf * B ** 3].reshape(q.nf, B, B, B)[:, NG:NG + E, NG:NG + E, NG:NG + E] = f
    q.name = f"amr_wave_{n_coarse * E}"
    q.meta["amp"] = amp
    return q


def amr_box(seed: int = 1006, n_coarse: int = 4, E: int = 8, n_species: int = 5, periodic: bool = True) -> Problem:
    """Two refinement levels in the unit box (Sec. II "Data-Structure": an
    adaptive octree with a subgrid per leaf): n_coarse^3 level-0 subgrids of
    E^3 cells, the central 2x2x2 of which are each replaced by 8 level-1
    subgrids (dx halved).  The noisy gas law of the other batches is drawn
    for every interior cell, keyed on (level, cell of the level); ghosts are
    left to the ghost fill across levels.
    meta: level, origin ([n, 3], in cells of each subgrid's level), n0, periodic."""
    N0 = n_coarse * E
    c0 = n_coarse // 2 - 1
    subs = []
    for sz in range(n_coarse):
        for sy in range(n_coarse):
            for sx in range(n_coarse):
                if all(c0 <= v <= c0 + 1 for v in (sx, sy, sz)):
                    continue
                subs.append((0, sx * E, sy * E, sz * E))
    for fz in range(4):
        for fy in range(4):
            for fx in range(4):
                subs.append((1, 2 * c0 * E + fx * E, 2 * c0 * E + fy * E, 2 * c0 * E + fz * E))
    n = len(subs)
    nf = 6 + n_species
    edge = np.full(n, E, np.int32)
    off, total = layout_offsets(edge, nf)
    U = np.zeros(total)
    level = np.array([s[0] for s in subs], np.int32)
    origin = np.array([s[1:] for s in subs], np.int32)
    dx = 1.0 / (N0 * 2.0 ** level)
    B = E + 2 * NG
    i = np.arange(E)
    for k, (l, ox, oy, oz) in enumerate(subs):
        Nl = N0 << l
        cnt = ((np.uint64(l) << np.uint64(40)) +
               (((oz + i)[:, None, None] * Nl + (oy + i)[None, :, None]) * Nl + (ox + i)[None, None, :]).astype(np.uint64))
        f = _noisy_gas_law(seed, cnt.reshape(-1), GAMMA, n_species).reshape(nf, E, E, E)
        U[off[k]: off[k] + nf * B ** 3].reshape(nf, B, B, B)[:, NG:NG + E, NG:NG + E, NG:NG + E] = f
    return Problem(f"amr_box_{N0}", edge, off, dx, level, nf, U, bc=3, nbr=None, grid=(), gamma=GAMMA,
                   meta=dict(level=level, origin=origin, n0=N0, periodic=periodic))
