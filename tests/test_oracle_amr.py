"""Pins of the oracle's ghost fill across refinement levels (Sec. II
"Data-Structure": one subgrid per octree leaf, neighbours that may sit one
level coarser or finer).  Reading: a ghost cell takes the covering cell of
its own level, else the coarser cell that contains it (injection), else the
mean of the 8 finer cells it contains (restriction)."""
import math

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


def _volume_totals(p, d):
    """Per field: sum over cells of dx^3 * d, and the same sum of |.|."""
    E = int(p.edge[0])
    dd = d.reshape(p.n_sub, p.nf, E ** 3)
    w = (p.dx ** 3)[:, None]
    return ([math.fsum((w * dd[:, f]).ravel()) for f in range(p.nf)],
            [math.fsum(np.abs(w * dd[:, f]).ravel()) for f in range(p.nf)])


def test_reflux_restores_conservation():
    """On a periodic two-level box the volume integral of dU/dt is a sum of
    face fluxes that cancel pairwise, except at coarse-fine faces where the
    coarse flux differs from the fine ones.  After the flux correction every
    field's integral vanishes to rounding; before it, it does not."""
    p = inputs.amr_box()
    m = p.meta
    oracle.amr_ghost_fill(8, p.off, p.nf, m["level"], m["origin"], m["n0"], m["periodic"], p.U)
    d, _, F, nb = oracle.rhs_faces(p.edge, p.off, p.dx, p.nf, p.U)
    assert nb == 0
    t, sc = _volume_totals(p, d)
    assert all(abs(a) > 1e-6 * b for a, b in zip(t, sc))
    oracle.amr_reflux(8, p.dx, p.nf, m["level"], m["origin"], m["n0"], m["periodic"], F, d)
    t, sc = _volume_totals(p, d)
    assert all(abs(a) <= 1e-14 * b for a, b in zip(t, sc)), [a / b for a, b in zip(t, sc)]


def test_reflux_takes_the_fine_mean_at_the_coarse_face_centre():
    """Coarse face fluxes 0, fine face fluxes a linear function of the face
    centre (distinct dyadic coefficients per axis and field): the
    correction of each coarse cell next to the refined block is +-F(centre of
    its coarse face)/dx, exactly, with + for its lower face; all other cells
    are untouched."""
    p = inputs.amr_box(n_coarse=4, E=8)
    E, n0 = 8, p.meta["n0"]
    lev, org = p.meta["level"], p.meta["origin"]
    nf = p.nf
    axes = [(1, 2), (0, 2), (0, 1)]
    coef = [(0.5 + f, 0.25 * (f + 1), -0.125 * (f + 2)) for f in range(nf)]

    def flux(f, k, lo, hi, pn):  # tangential positions lo, hi and normal position pn, level-0 units
        a, b, c = coef[f]
        return a + b * lo + c * hi + 0.375 * pn + 0.0625 * k

    F = np.zeros((p.n_sub, 6, nf, E, E))
    i = np.arange(E)
    for t in range(p.n_sub):
        if lev[t] != 1:
            continue
        for k in range(3):
            al, ah = axes[k]
            hi, lo = np.meshgrid((org[t, ah] + i + 0.5) / 2, (org[t, al] + i + 0.5) / 2, indexing="ij")
            for side in range(2):
                for f in range(nf):
                    F[t, 2 * k + side, f] = flux(f, k, lo, hi, (org[t, k] + side * E) / 2)
    d = np.zeros(p.n_sub * nf * E ** 3)
    oracle.amr_reflux(E, p.dx, nf, lev, org, n0, True, F, d)
    d = d.reshape(p.n_sub, nf, E, E, E)  # [s][f][z][y][x]
    lo_b, hi_b = (n0 // E // 2 - 1) * E, (n0 // E // 2 + 1) * E  # refined block, level-0 cells
    want = np.zeros_like(d)
    for s in range(p.n_sub):
        if lev[s] != 0:
            continue
        for z in range(E):
            for y in range(E):
                for x in range(E):
                    c = (org[s, 0] + x, org[s, 1] + y, org[s, 2] + z)
                    for k in range(3):
                        al, ah = axes[k]
                        for side, step in ((0, -1), (1, 1)):
                            if (c[k] - org[s, k]) != (E - 1 if side else 0):
                                continue
                            g = list(c)
                            g[k] = (g[k] + step) % n0
                            if not all(lo_b <= v < hi_b for v in g):
                                continue
                            for f in range(nf):
                                Fc = flux(f, k, c[al] + 0.5, c[ah] + 0.5, c[k] + side)
                                want[s, f, z, y, x] += (-Fc if side else Fc) / p.dx[s]
    assert np.count_nonzero(want) > 0
    np.testing.assert_array_equal(d, want)


def test_reflux_on_one_level_changes_nothing():
    p = inputs.periodic_box(nsub=2, E=8)
    org = np.array([((s % 2) * 8, ((s // 2) % 2) * 8, (s // 4) * 8) for s in range(p.n_sub)], np.int32)
    rng = np.random.default_rng(3)
    F = rng.standard_normal((p.n_sub, 6, p.nf, 8, 8))
    d = rng.standard_normal(p.n_sub * p.nf * 512)
    d0 = d.copy()
    oracle.amr_reflux(8, p.dx, p.nf, np.zeros(p.n_sub, np.int32), org, 16, True, F, d)
    assert np.array_equal(d, d0)


def test_amr_rk3_step_conserves():
    """One SSP-RK3 step across levels, with the flux correction, conserves
    mass, momentum and energy to 1e-14 on the periodic two-level box."""
    p = inputs.amr_box()
    m = p.meta
    oracle.amr_ghost_fill(8, p.off, p.nf, m["level"], m["origin"], m["n0"], m["periodic"], p.U)
    from tests.helpers import interior_layout
    before = interior_layout(p.U, p)
    dt, fired, st = oracle.rk3_step_amr(p.edge, p.off, p.dx, p.nf, p.U, m["level"], m["origin"], m["n0"],
                                        m["periodic"], gamma=p.gamma)
    assert st == 0 and fired == 0 and dt > 0
    after = interior_layout(p.U, p)
    t0, sc = _volume_totals(p, before)
    t1, _ = _volume_totals(p, after)
    for f in range(5):
        assert abs(t1[f] - t0[f]) <= 1e-14 * sc[f], (f, (t1[f] - t0[f]) / sc[f])


# ---------------------------------------------------------------------------
# Limited linear prolongation (order 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [True, False])
def test_order0_of_the_general_fill_is_the_injection_fill(periodic):
    p = inputs.amr_box(periodic=periodic)
    m = p.meta
    a, b = p.U.copy(), p.U.copy()
    oracle.amr_ghost_fill(8, p.off, p.nf, m["level"], m["origin"], m["n0"], periodic, a)
    lib = oracle.lib()
    lev, org = np.ascontiguousarray(m["level"], np.int32), np.ascontiguousarray(m["origin"], np.int32).reshape(-1)
    off = np.ascontiguousarray(p.off, np.int64)
    r = lib.oco_amr_ghost_fill_order(p.n_sub, 8, off.ctypes.data, p.nf, lev.ctypes.data, org.ctypes.data,
                                     int(m["n0"]), int(periodic), 0, b.ctypes.data)
    assert r == 0
    assert np.array_equal(a, b)


@pytest.mark.parametrize("periodic", [True, False])
def test_linear_prolongation_reproduces_a_linear_field(periodic):
    """With slopes from a linear field (equal one-sided differences, so the
    minmod keeps them) every ghost cell -- copy, restriction or prolongation --
    gets the field's value at its own centre, exactly (dyadic values)."""
    p = inputs.amr_box(n_coarse=4, E=8, periodic=periodic)
    E, n0 = 8, p.meta["n0"]
    lev, org = p.meta["level"], p.meta["origin"]
    coef = _coefs(p.nf)
    _linear_fill(p, coef)
    oracle.amr_ghost_fill(E, p.off, p.nf, lev, org, n0, periodic, p.U, order=1)
    B = E + 2 * NG
    r = np.arange(-NG, E + NG)
    gz, gy, gx = np.meshgrid(r, r, r, indexing="ij")
    ghost = ~((gx >= 0) & (gx < E) & (gy >= 0) & (gy < E) & (gz >= 0) & (gz < E))
    for s in range(p.n_sub):
        l = int(lev[s])
        nl = n0 << l
        g = [org[s, 0] + gx, org[s, 1] + gy, org[s, 2] + gz]
        g = [np.mod(v, nl) if periodic else np.clip(v, 0, nl - 1) for v in g]
        cen = [(v + 0.5) / (2 ** l) for v in g]
        blk = p.U[p.off[s]: p.off[s] + p.nf * B ** 3].reshape(p.nf, B, B, B)
        for f in range(p.nf):
            a, b, c, d = coef[f]
            want = a + b * cen[0] + c * cen[1] + d * cen[2]
            np.testing.assert_array_equal(blk[f][ghost], want[ghost])


def test_linear_prolongation_keeps_means_and_bounds():
    """On the noisy field: the prolonged children of a coarse cell lie within
    the range of that coarse cell and its six face neighbours (the minmod
    limiter adds no extremum), and where all 8 children of a coarse cell are
    ghost cells of one fine subgrid their mean is the coarse value."""
    p = inputs.amr_box()
    E, B, n0 = 8, 14, p.meta["n0"]
    lev, org = p.meta["level"], p.meta["origin"]
    oracle.amr_ghost_fill(E, p.off, p.nf, lev, org, n0, True, p.U, order=1)
    q = inputs.amr_box()  # the coarse values around, from the copies and restrictions of order 0
    oracle.amr_ghost_fill(E, q.off, q.nf, lev, org, n0, True, q.U, order=0)
    coarse = {}
    for s in range(p.n_sub):
        if lev[s] == 0:
            coarse[tuple(org[s] // E)] = s
    n_checked = n_means = 0
    for s in range(p.n_sub):
        if lev[s] != 1:
            continue
        blk = p.U[p.off[s]: p.off[s] + p.nf * B ** 3].reshape(p.nf, B, B, B)
        groups = {}
        for z in range(-NG, E + NG):
            for y in range(-NG, E + NG):
                for x in range(-NG, E + NG):
                    if 0 <= x < E and 0 <= y < E and 0 <= z < E:
                        continue
                    g = [(org[s, 0] + x) % (2 * n0), (org[s, 1] + y) % (2 * n0), (org[s, 2] + z) % (2 * n0)]
                    gc = [v >> 1 for v in g]
                    key = tuple(v // E for v in gc)
                    if key not in coarse:
                        continue  # a same-level copy
                    t = coarse[key]
                    cb = q.U[q.off[t]: q.off[t] + q.nf * B ** 3].reshape(q.nf, B, B, B)
                    lc = [gc[a] - org[t, a] + NG for a in range(3)]
                    nb = [cb[:, lc[2], lc[1], lc[0]]]
                    for a in range(3):
                        for st in (-1, 1):
                            ll = list(lc)
                            ll[a] += st
                            nb.append(cb[:, ll[2], ll[1], ll[0]])
                    nb = np.stack(nb)
                    v = blk[:, z + NG, y + NG, x + NG]
                    lo, hi = nb.min(axis=0), nb.max(axis=0)
                    tol = 1e-15 * np.maximum(np.abs(lo), np.abs(hi))
                    assert np.all(v >= lo - tol) and np.all(v <= hi + tol)
                    n_checked += 1
                    groups.setdefault(tuple(gc), []).append(v)
        for gc, vs in groups.items():
            if len(vs) == 8:
                t = coarse[tuple(v // E for v in gc)]
                cb = q.U[q.off[t]: q.off[t] + q.nf * B ** 3].reshape(q.nf, B, B, B)
                uc = cb[:, gc[2] - org[t, 2] + NG, gc[1] - org[t, 1] + NG, gc[0] - org[t, 0] + NG]
                np.testing.assert_allclose(np.mean(vs, axis=0), uc, rtol=1e-14,
                                           atol=1e-14 * float(np.max(np.abs(vs))))
                n_means += 1
    assert n_checked > 1000 and n_means > 10


def test_amr_rk3_step_with_linear_prolongation_conserves():
    p = inputs.amr_box()
    m = p.meta
    oracle.amr_ghost_fill(8, p.off, p.nf, m["level"], m["origin"], m["n0"], m["periodic"], p.U, order=1)
    from tests.helpers import interior_layout
    before = interior_layout(p.U, p)
    dt, fired, st = oracle.rk3_step_amr(p.edge, p.off, p.dx, p.nf, p.U, m["level"], m["origin"], m["n0"],
                                        m["periodic"], gamma=p.gamma, order=1)
    assert st == 0 and fired == 0 and dt > 0
    after = interior_layout(p.U, p)
    t0, sc = _volume_totals(p, before)
    t1, _ = _volume_totals(p, after)
    for f in range(5):
        assert abs(t1[f] - t0[f]) <= 1e-14 * sc[f], (f, (t1[f] - t0[f]) / sc[f])
