"""Pins of the oracle's ghost fill across refinement levels (Sec. II
"Data-Structure": one subgrid per octree leaf, neighbours that may sit one
level coarser or finer).  Reading: a ghost cell takes the covering cell of
its own level, else the coarser cell that contains it (injection), else the
mean of the 8 finer cells it contains (restriction)."""
import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs

NG = 3


def _linear_fill(p, coef):
    """Every interior cell of field f gets coef[f] . (1, x, y, z), with
    (x, y, z) the cell centre in level-0 cell units.  Dyadic coefficients
    keep every value, and every mean of 8 of them, exact in binary."""
    E = int(p.edge[0])
    B = E + 2 * NG
    lev, org = p.meta["level"], p.meta["origin"]
    i = np.arange(E)
    for s in range(p.n_sub):
        h = 0.5 ** int(lev[s])
        z, y, x = np.meshgrid((org[s, 2] + i + 0.5) * h, (org[s, 1] + i + 0.5) * h, (org[s, 0] + i + 0.5) * h,
                              indexing="ij")
        blk = p.U[p.off[s]: p.off[s] + p.nf * B ** 3].reshape(p.nf, B, B, B)
        for f in range(p.nf):
            a, b, c, d = coef[f]
            blk[f, NG:NG + E, NG:NG + E, NG:NG + E] = a + b * x + c * y + d * z


def _coefs(nf):
    return [(1.0 + f, 0.25 * (f + 1), -0.5, 0.125 * (3 - f)) for f in range(nf)]


@pytest.mark.parametrize("periodic", [True, False])
def test_linear_field_closed_form(periodic):
    """Copies and restrictions of a linear field give its value at the ghost
    cell's own centre; injection gives it at the centre of the coarse parent.
    Which case applies follows from the geometry alone: the refined region is
    the central 2x2x2 block of level-0 subgrids."""
    p = inputs.amr_box(n_coarse=4, E=8, periodic=periodic)
    E, n0 = 8, p.meta["n0"]
    lev, org = p.meta["level"], p.meta["origin"]
    coef = _coefs(p.nf)
    _linear_fill(p, coef)
    oracle.amr_ghost_fill(E, p.off, p.nf, lev, org, n0, periodic, p.U)
    lo, hi = (n0 // E // 2 - 1) * E, (n0 // E // 2 + 1) * E  # refined block, level-0 cells
    B = E + 2 * NG
    r = np.arange(-NG, E + NG)
    gz, gy, gx = np.meshgrid(r, r, r, indexing="ij")
    ghost = ~((gx >= 0) & (gx < E) & (gy >= 0) & (gy < E) & (gz >= 0) & (gz < E))
    n_inj = 0
    for s in range(p.n_sub):
        l = int(lev[s])
        nl = n0 << l
        g = [org[s, 0] + gx, org[s, 1] + gy, org[s, 2] + gz]
        g = [np.mod(v, nl) if periodic else np.clip(v, 0, nl - 1) for v in g]
        if l == 1:
            inside = np.all([(v >= 2 * lo) & (v < 2 * hi) for v in g], axis=0)
            cen = [np.where(inside, (v + 0.5) / 2, (v // 2) + 0.5) for v in g]
            n_inj += int(np.sum(~inside & ghost))
        else:
            cen = [v + 0.5 for v in g]
        blk = p.U[p.off[s]: p.off[s] + p.nf * B ** 3].reshape(p.nf, B, B, B)
        for f in range(p.nf):
            a, b, c, d = coef[f]
            want = a + b * cen[0] + c * cen[1] + d * cen[2]
            np.testing.assert_array_equal(blk[f][ghost], want[ghost])
    assert n_inj > 0


@pytest.mark.parametrize("periodic", [True, False])
def test_single_level_reduces_to_tiling_fill(periodic):
    """With every subgrid on level 0 the fill across levels is the uniform
    tiling fill from the 26-neighbour table (periodic or zero-gradient)."""
    p = inputs.periodic_box(nsub=3, E=8)
    nbr = inputs.tiling_neighbours(3, 3, 3, periodic)
    org = np.array([((s % 3) * 8, ((s // 3) % 3) * 8, (s // 9) * 8) for s in range(p.n_sub)], np.int32)
    a, b = p.U.copy(), p.U.copy()
    oracle.ghost_fill(8, p.off, p.nf, nbr, a)
    oracle.amr_ghost_fill(8, p.off, p.nf, np.zeros(p.n_sub, np.int32), org, 24, periodic, b)
    assert np.array_equal(a, b)


def test_missing_source_is_an_error():
    """A ghost cell with no covering cell on its own, the coarser or the
    finer level (here: half of the root box has no subgrid) is rejected."""
    p = inputs.periodic_box(nsub=2, E=8)
    org = np.array([((s % 2) * 8, ((s // 2) % 2) * 8, (s // 4) * 8) for s in range(p.n_sub)], np.int32)
    lev = np.zeros(p.n_sub, np.int32)
    with pytest.raises(ValueError):
        oracle.amr_ghost_fill(8, p.off[:4], p.nf, lev[:4], org[:4], 16, True, p.U)


def test_uniform_state_is_steady_across_levels():
    """A uniform moving state is an exact steady solution.  With dyadic
    values (whose 8-cell means are exact) the RHS after the fill across
    levels is exactly zero on both levels; with general values one RK3 step
    changes no cell by more than the rounding of the restriction means and
    of the stage averages (3/4 a + 1/4 a), and the step is set by the finest
    cells (dx = 1/64)."""
    import math
    p = inputs.amr_box(n_coarse=4, E=8)
    E, B = 8, 14
    G = p.gamma
    m = p.meta

    def uniform(vals):
        for s in range(p.n_sub):
            blk = p.U[p.off[s]: p.off[s] + p.nf * B ** 3].reshape(p.nf, B, B, B)
            for f in range(p.nf):
                blk[f] = vals[f]

    # rho 1.25, v (0.75, -0.5, 0.25), p 0.5: E = 0.75 + 0.546875, tau 1, species 0.25
    uniform([1.25, 0.9375, -0.625, 0.3125, 1.296875, 1.0] + [0.25] * (p.nf - 6))
    oracle.amr_ghost_fill(E, p.off, p.nf, m["level"], m["origin"], m["n0"], m["periodic"], p.U)
    d, _, _ = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U)
    assert not np.any(d)

    rho, v, pr = 1.3, (0.7, -0.4, 0.2), 0.9
    e = pr / (G - 1)
    vals = [rho, rho * v[0], rho * v[1], rho * v[2], e + 0.5 * rho * sum(c * c for c in v), e ** (1 / G)]
    uniform(vals + [rho / 5] * (p.nf - 6))
    U0 = p.U.copy()
    dt, fired, st = oracle.rk3_step_amr(p.edge, p.off, p.dx, p.nf, p.U, m["level"], m["origin"], m["n0"],
                                        m["periodic"])
    assert st == 0 and fired == 0
    np.testing.assert_allclose(p.U, U0, rtol=1e-15, atol=0)
    c = math.sqrt(G * pr / rho)
    assert dt == pytest.approx(0.4 * (1.0 / 64) / (0.7 + c), rel=1e-14)
