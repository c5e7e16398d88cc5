"""Pins of the oracle's same-level monopole gravity (reading R18: every cell
receives -G m_j / r and -G m_j (x_i - x_j) / r^3 from each cell j of its
level within r_s cell widths, m_j = rho_j dx^3 at the cell centre).

What fixes the result independently of the oracle's loops:
  - a single mass gives the textbook point-mass potential and field in
    exactly the cells within r_s (found across subgrid boundaries through
    the neighbour table), nothing elsewhere, and the field points at the
    mass (attraction);
  - Newton's third law: with every pair of massive cells within r_s of each
    other, the net self-force sum_i m_i g_i vanishes;
  - superposition: the potential and field are linear in the density;
  - a uniform sphere: the potential at its centre tends to that of the
    continuum sphere of equal volume, -2 pi G rho R^2 (less the centre cell's
    own share) under refinement, its interior field is -(4/3) pi G rho r, and
    outside it potential and field are those of a point mass of the sphere's
    mass (shell theorem; the discretised sphere's quadrupole vanishes by
    cubic symmetry).
"""
import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs

NF = 6
THETA_RS = 2.0 / 0.34  # the interaction radius of reading R18 for the paper's opening angle


def _box(rho, nsub, E, periodic=False):
    """A batch of nsub^3 subgrids of edge E tiling the density field rho
    [Z, Y, X] (other fields zero), with its neighbour table."""
    fields = np.zeros((NF,) + rho.shape)
    fields[0] = rho
    N = rho.shape[0]
    return inputs._tile_global("gravity", fields, (nsub,) * 3, E, 1.0 / N, 1 if periodic else 2, periodic)


def _grav(p, r_s=THETA_RS, G=1.0):
    E = int(p.edge[0])
    phi, g = oracle.gravity_monopole(E, p.off, p.nf, p.nbr, float(p.dx[0]), p.U, G=G, r_s=r_s)
    n = p.n_sub
    return phi.reshape(n, E, E, E), g.reshape(n, 3, E, E, E)


def _global(p, a, nsub):
    """[n, ..., E, E, E] per-subgrid arrays back to global [..., Z, Y, X]."""
    E = int(p.edge[0])
    lead = a.shape[1:-3]
    a = a.reshape((nsub, nsub, nsub) + lead + (E, E, E))
    perm = list(range(3, 3 + len(lead))) + [0, 3 + len(lead), 1, 4 + len(lead), 2, 5 + len(lead)]
    return a.transpose(perm).reshape(lead + (nsub * E,) * 3)


def test_single_mass_gives_the_point_mass_field_within_the_radius():
    nsub, E = 2, 8
    N = nsub * E
    rho = np.zeros((N, N, N))
    src = (7, 8, 6)  # a subgrid corner region: the stencil crosses into all neighbours
    rho[src] = 3.0
    p = _box(rho, nsub, E)
    phi, g = _grav(p, G=2.0)
    phi, g = _global(p, phi, nsub), _global(p, g, nsub)
    dx = 1.0 / N
    m = 3.0 * dx ** 3
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    d = np.stack([x - src[2], y - src[1], z - src[0]])  # x_i - x_j in cells
    d2 = np.sum(d * d, axis=0)
    inside = (d2 > 0) & (d2 <= THETA_RS ** 2)
    r = np.sqrt(d2) * dx
    with np.errstate(divide="ignore", invalid="ignore"):
        phi_ref = np.where(inside, -2.0 * m / r, 0.0)
        g_ref = np.where(inside, -2.0 * m * d * dx / r ** 3, 0.0)
    np.testing.assert_allclose(phi, phi_ref, rtol=4e-16, atol=0)
    np.testing.assert_allclose(g, g_ref, rtol=4e-16, atol=0)
    assert np.count_nonzero(phi) == np.count_nonzero(inside)
    # attraction: the field at every cell in range points at the mass
    assert np.all(np.sum(g * d, axis=0)[inside] < 0)


def test_newton_third_law_for_a_compact_cluster():
    """Random masses in a ball of radius 2.5 cells around a subgrid corner:
    every pair lies within r_s, so the forces cancel in pairs."""
    nsub, E = 2, 8
    N = nsub * E
    rng = np.random.default_rng(3)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    c = np.array([7.5, 7.5, 7.5])
    ball = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= 2.5 ** 2
    rho = np.where(ball, rng.uniform(0.1, 2.0, (N, N, N)), 0.0)
    p = _box(rho, nsub, E)
    phi, g = _grav(p)
    g = _global(p, g, nsub)
    dx = 1.0 / N
    m = rho * dx ** 3
    F = np.array([np.sum(m * g[a]) for a in range(3)])
    scale = np.sum(m * np.sqrt(np.sum(g * g, axis=0)))
    assert np.all(np.abs(F) <= 1e-14 * scale), F / scale
    # the potential energy is negative and every massive cell is bound
    assert np.all(_global(p, phi, nsub)[ball] < 0)


def test_superposition():
    nsub, E = 2, 8
    N = nsub * E
    rng = np.random.default_rng(4)
    r1 = rng.uniform(0, 1, (N, N, N))
    r2 = rng.uniform(0, 1, (N, N, N)) * (rng.uniform(0, 1, (N, N, N)) < 0.3)
    a = _grav(_box(r1, nsub, E))
    b = _grav(_box(r2, nsub, E))
    s = _grav(_box(r1 + r2, nsub, E))
    for k in range(2):
        np.testing.assert_allclose(s[k], a[k] + b[k], rtol=1e-13, atol=1e-13 * np.max(np.abs(s[k])))


def _sphere(R, E=16, nsub=3):
    """Uniform density 1 in the cells whose centres lie within R cell widths
    of the centre of the middle cell of a (nsub E)^3 box."""
    N = nsub * E
    c = N // 2
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    r2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    return (r2 <= R * R).astype(float), c, N


def _cube_self_integral():
    """The integral of 1/|x| over the unit cube centred at the origin: by
    symmetry 24 pyramids {0 <= y, z <= x <= 1/2}, each (1/8) int_0^1 int_0^1
    du dv / sqrt(1 + u^2 + v^2), so 3 times that double integral."""
    from scipy import integrate
    val, _ = integrate.dblquad(lambda v, u: 1.0 / np.sqrt(1.0 + u * u + v * v), 0.0, 1.0, 0.0, 1.0,
                               epsabs=1e-13, epsrel=1e-13)
    return 3.0 * val


def test_uniform_sphere_centre_converges():
    """The potential at the centre of a uniform sphere of cells against the
    continuum sphere of the same volume, -2 pi G rho R_eff^2, with the centre
    cell's own share (which a cell does not exert on itself) added back: the
    error falls as the sphere spans more cells."""
    pytest.importorskip("scipy")
    c_self = _cube_self_integral()
    assert abs(c_self - 2.3800773) < 1e-6  # the potential of a unit cube at its centre
    errs = []
    for R in (3, 6, 12):
        rho, c, N = _sphere(R)
        p = _box(rho, 3, 16)
        phi, _ = _grav(p, r_s=16.0)
        phi = _global(p, phi, 3)
        dx = 1.0 / N
        R_eff = (3.0 * np.sum(rho) / (4.0 * np.pi)) ** (1.0 / 3.0) * dx
        ref = -2.0 * np.pi * R_eff ** 2 + c_self * dx ** 2
        errs.append(abs(phi[c, c, c] - ref) / abs(ref))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-3, errs


@pytest.mark.parametrize("R", [3, 6])
def test_uniform_sphere_exterior_is_a_point_mass(R):
    """Outside the sphere, at points within r_s of every one of its cells:
    -G M / D and -G M / D^2 toward the centre, along an axis and a diagonal
    (the discretised sphere has no quadrupole moment by cubic symmetry)."""
    rho, c, N = _sphere(R)
    p = _box(rho, 3, 16)
    phi, g = _grav(p, r_s=16.0)
    phi, g = _global(p, phi, 3), _global(p, g, 3)
    dx = 1.0 / N
    M = np.sum(rho) * dx ** 3
    for off in ((R + 4, 0, 0), (7, 7, 0) if R == 6 else (5, 5, 0), (0, 4, 8) if R == 6 else (0, 3, 5)):
        o = np.array(off, float)
        D = np.sqrt(o @ o) * dx
        assert D / dx + R <= 16.0
        val = phi[c + off[2], c + off[1], c + off[0]]
        assert abs(val + M / D) / (M / D) < 3e-3, (off, val, -M / D)
        gv = g[:, c + off[2], c + off[1], c + off[0]]
        gref = -M / D ** 2 * o / np.sqrt(o @ o)
        assert np.linalg.norm(gv - gref) / np.linalg.norm(gref) < 1.5e-2, (off, gv, gref)


def test_uniform_sphere_interior_field():
    """Inside a uniform sphere the field is -(4/3) pi G rho r, toward the
    centre (every cell of the sphere within r_s of the points tested)."""
    R = 6
    rho, c, N = _sphere(R)
    p = _box(rho, 3, 16)
    _, g = _grav(p, r_s=16.0)
    g = _global(p, g, 3)
    dx = 1.0 / N
    for k in (2, 3, 4):
        r = k * dx
        gx = g[0, c, c, c + k]
        ref = -(4.0 / 3.0) * np.pi * r
        assert abs(gx - ref) / abs(ref) < 0.05, (k, gx, ref)
        # on the axis the other components cancel by symmetry
        assert abs(g[1, c, c, c + k]) <= 1e-13 * abs(gx) and abs(g[2, c, c, c + k]) <= 1e-13 * abs(gx)
    assert g[0, c, c, c] == 0.0 or abs(g[0, c, c, c]) < 1e-13 * abs(ref)


def test_mass_beyond_the_radius_is_not_seen_and_missing_neighbours_hold_none():
    nsub, E = 2, 8
    N = nsub * E
    rho = np.zeros((N, N, N))
    rho[0, 0, 0] = 1.0
    p = _box(rho, nsub, E)
    phi, _ = _grav(p, r_s=3.0)
    phi = _global(p, phi, nsub)
    # (3, 0, 0) is at distance 3 (inside); (2, 2, 2) at sqrt(12) > 3 (outside)
    assert phi[0, 0, 3] != 0.0 and phi[2, 2, 2] == 0.0 and phi[0, 0, 4] == 0.0
    # periodic: the mass is also seen across the wrapped edge, outflow: not
    pp = _box(rho, nsub, E, periodic=True)
    php, _ = _grav(pp, r_s=3.0)
    php = _global(pp, php, nsub)
    assert php[0, 0, N - 1] != 0.0 and phi[0, 0, N - 1] == 0.0
