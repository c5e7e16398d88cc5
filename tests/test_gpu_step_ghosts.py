"""Ghost cells after an RK3 step on a uniform level, over the arrangements a
neighbour table can describe: the stepped state must match the oracle's
step, and its ghost cells must be exactly the oracle's ghost fill of its
interior (the copy of the matching neighbour cell, or of the nearest own cell
along axes without a face neighbour), bitwise.  Arrangements: one subgrid
wrapping onto itself; two and three subgrids along an axis (a two-wide
periodic axis links both faces to the same subgrid); non-cubic boxes;
periodic along some axes and open along the others; outflow on every side;
edges 8, 12 and 16; a table with a one-way link; and three graph-replayed
steps in a row.  Also the library's count of the kernels one step launches."""
import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.helpers import e3s, field_errors, interior_layout, oracle_filled

pytestmark = pytest.mark.gpu


def _box(nx, ny, nz, E=8, periodic=True, seed=7):
    n_cells = nx * ny * nz * E ** 3
    f = inputs._noisy_gas_law(seed, np.arange(n_cells, dtype=np.uint64))
    f = f.reshape(11, nz * E, ny * E, nx * E)
    bc = 1 if periodic is True else 2
    return inputs._tile_global("step_ghosts", f, (nx, ny, nz), E, 1.0 / (max(nx, ny, nz) * E), bc, periodic)


def _step_and_check(p, precision=0):
    import torch
    from paper_2210_06439_gb300 import binding
    ref = oracle_filled(p)
    U0 = ref.U.copy()
    dt_o, fired, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=p.bc, nbr=p.nbr)
    assert st == 0
    H = binding.Hydro.from_problem(p, precision=precision)
    # 3 RHS, each with the whole-subgrid uniform test (three kernels in the first stage,
    # two in the others) and, on edge 8 and 16, the work list after it; the dt
    # reduction, 3 combines, 3 ghost fills
    assert H.step_launches() == 3 + 7 + (3 if int(p.edge[0]) in (8, 16) else 0) + 1 + 3 + 3
    U = torch.from_numpy(U0).cuda()
    dt_g = H.rk_step(U)
    flags = H.error_flags()
    assert flags & ~binding.OCT_FLAG_FLOOR == 0, flags
    assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else 2e-6)
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs
    chk = p.copy()
    chk.U[:] = got
    oracle.ghost_fill(int(p.edge[0]), chk.off, chk.nf, chk.nbr, chk.U)
    assert np.array_equal(chk.U, got), np.flatnonzero(chk.U != got)[:10]
    return got


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 1), (3, 2, 1), (2, 2, 2), (1, 3, 2)])
def test_periodic_arrangements(shape):
    _step_and_check(_box(*shape, periodic=True))


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 1), (2, 3, 2), (3, 3, 3)])
def test_outflow_arrangements(shape):
    _step_and_check(_box(*shape, periodic=False))


@pytest.mark.parametrize("periodic", [(True, False, False), (False, True, True), (True, True, False)])
def test_periodic_along_some_axes(periodic):
    _step_and_check(_box(3, 2, 2, periodic=periodic))


@pytest.mark.parametrize("E", [12, 16])
@pytest.mark.parametrize("periodic", [True, False])
def test_larger_edges(E, periodic):
    _step_and_check(_box(2, 2, 1, E=E, periodic=periodic))


def test_mixed_form():
    _step_and_check(_box(3, 2, 2, periodic=(True, False, True)), precision=1)


def test_one_way_link():
    """Subgrid 1 of a 2x1x1 outflow row does not list subgrid 0 as its -x
    neighbour (so it clamps those ghosts to its own cells) while subgrid 0
    lists subgrid 1 as its +x neighbour."""
    p = _box(2, 1, 1, periodic=False)
    nbr = p.nbr.reshape(2, 26).copy()
    slot = inputs.nb_slot(-1, 0, 0)
    assert nbr[1, slot] == 0
    nbr[1, slot] = -1
    p.nbr = nbr.ravel()
    _step_and_check(p)


def test_steps_replay_and_match_the_oracle_over_several_steps():
    """Three graph-replayed steps on an outflow box against three oracle
    steps."""
    import torch
    from paper_2210_06439_gb300 import binding
    p = _box(3, 2, 2, periodic=False, seed=11)
    ref = oracle_filled(p)
    U = torch.from_numpy(ref.U.copy()).cuda()
    H = binding.Hydro.from_problem(p)
    for _ in range(3):
        dt_o, _, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=p.bc, nbr=p.nbr)
        assert st == 0
        dt_g = H.rk_step(U)
        assert dt_g == pytest.approx(dt_o, rel=1e-12)
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= 1e-12), errs
    chk = p.copy()
    chk.U[:] = got
    oracle.ghost_fill(8, chk.off, chk.nf, chk.nbr, chk.U)
    assert np.array_equal(chk.U, got)


def _uniform_box(tau_scale, periodic=False, n_species=5):
    """A 3x2x2 box (outflow, or periodic) of one moving gas state: rho = 1.3,
    v = (0.2, -0.1, 0.05), p = 0.7, species in fixed fractions, tau =
    tau_scale * e_int^(1/gamma)."""
    g = inputs.GAMMA
    nx, ny, nz, E = 3, 2, 2, 8
    rho, v, p = 1.3, (0.2, -0.1, 0.05), 0.7
    ei = p / (g - 1.0)
    f = np.zeros((6 + n_species, nz * E, ny * E, nx * E))
    f[0] = rho
    for a in range(3):
        f[1 + a] = rho * v[a]
    f[4] = ei + 0.5 * rho * sum(x * x for x in v)
    f[5] = tau_scale * ei ** (1.0 / g)
    for i in range(n_species):
        f[6 + i] = rho * (i + 1) / (n_species * (n_species + 1) / 2)
    return inputs._tile_global("uniform_box", f, (nx, ny, nz), E, 1.0 / 24, 1 if periodic else 2, periodic)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("tau_scale,periodic", [(1.0, False), (0.5, False), (0.5, True)])
def test_uniform_box_steps(precision, tau_scale, periodic):
    """Every subgrid holds one state, so every RHS is -0.0 and the combines
    take their per-subgrid pass: with tau = e_int^(1/gamma) the state is a
    fixed point of the step to within the re-synchronisation's rounding (the
    later stages find nothing changed and the ghost fills leave the ghosts
    alone); with tau halved, the first re-synchronisation changes every cell
    (written, and the ghosts refilled).  Three graph-replayed steps against
    the oracle's three, each subgrid's interior exactly uniform afterwards,
    and the ghosts exactly the oracle's ghost fill of the interior."""
    import torch
    from paper_2210_06439_gb300 import binding
    p = _uniform_box(tau_scale, periodic)
    ref = oracle_filled(p)
    U = torch.from_numpy(ref.U.copy()).cuda()
    H = binding.Hydro.from_problem(p, precision=precision)
    for _ in range(3):
        dt_o, _, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=p.bc, nbr=p.nbr)
        assert st == 0
        dt_g = H.rk_step(U)
        assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else 2e-6)
    assert H.error_flags() & binding.OCT_FLAG_NONPHYS == 0
    got = U.cpu().numpy()
    gi = interior_layout(got, p).reshape(p.n_sub, p.nf, -1)
    assert np.all(gi == gi[:, :, :1])  # one value per field in every subgrid
    assert np.all(gi == gi[:1, :, :1])  # and the same in all of them
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs
    chk = p.copy()
    chk.U[:] = got
    oracle.ghost_fill(8, chk.off, chk.nf, chk.nbr, chk.U)
    assert np.array_equal(chk.U, got)


@pytest.mark.parametrize("precision", [0, 1])
def test_binary_star_steps(precision):
    """Three graph-replayed steps of the 32^3 binary star (48 of its 64
    subgrids atmosphere, which the combines take as whole subgrids) against
    the oracle's three; ghosts exactly the oracle's ghost fill of the
    interior."""
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.binary_star(nsub=4)
    ref = oracle_filled(p)
    U = torch.from_numpy(ref.U.copy()).cuda()
    H = binding.Hydro.from_problem(p, precision=precision)
    for _ in range(3):
        dt_o, _, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=p.bc, nbr=p.nbr)
        assert st == 0
        dt_g = H.rk_step(U)
        assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else 2e-6)
    assert H.error_flags() & binding.OCT_FLAG_NONPHYS == 0
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-5)), errs
    chk = p.copy()
    chk.U[:] = got
    oracle.ghost_fill(8, chk.off, chk.nf, chk.nbr, chk.U)
    assert np.array_equal(chk.U, got)


@pytest.mark.parametrize("precision", [0, 1])
def test_uniform_box_steps_with_given_ghosts(precision):
    """The uniform box with its ghosts given (filled once, never refilled):
    the step's stage states carry the given ghosts, so their uniform test
    streams the blocks instead of reading the combines' record.  Three
    steps against the oracle's, the ghosts left as they were."""
    import torch
    from paper_2210_06439_gb300 import binding
    p = oracle_filled(_uniform_box(0.5))
    p.bc = 0
    ref = p.copy()
    U = torch.from_numpy(p.U.copy()).cuda()
    H = binding.Hydro.from_problem(p, precision=precision)
    for _ in range(3):
        dt_o, _, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=0)
        assert st == 0
        dt_g = H.rk_step(U)
        assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else 2e-6)
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs
    ghosts = interior_layout(np.arange(got.size, dtype=np.float64), p)  # interior indices
    mask = np.ones(got.size, bool)
    mask[ghosts.astype(np.int64)] = False
    assert np.array_equal(got[mask], p.U[mask])


def test_two_states_alternating_on_one_handle():
    """The handle's stage state W is shared by every state it steps, and its
    first combine compares with what the last step left there.  Two uniform
    boxes of the same layout and different values (the second with tau
    consistent and density, momenta, energy and species doubled), stepped
    in turn, twice each, each step against the oracle's; ghosts bitwise."""
    import torch
    from paper_2210_06439_gb300 import binding
    pa = _uniform_box(0.5)
    pb = _uniform_box(1.0)
    for s in range(pb.n_sub):
        b = pb.block(s)
        b[0] *= 2.0
        b[1:5] *= 2.0
        b[6:] *= 2.0
    refs = [oracle_filled(pa), oracle_filled(pb)]
    Us = [torch.from_numpy(r.U.copy()).cuda() for r in refs]
    H = binding.Hydro.from_problem(pa)
    for k in range(4):
        i = k % 2
        ref = refs[i]
        dt_o, _, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=ref.bc, nbr=ref.nbr)
        assert st == 0
        dt_g = H.rk_step(Us[i])
        assert dt_g == pytest.approx(dt_o, rel=1e-12)
        got = Us[i].cpu().numpy()
        errs = field_errors(interior_layout(got, pa), interior_layout(ref.U, pa), pa.nf, e3s(pa))
        assert np.all(errs <= 1e-12), (k, errs)
        chk = pa.copy()
        chk.U[:] = got
        oracle.ghost_fill(8, chk.off, chk.nf, chk.nbr, chk.U)
        assert np.array_equal(chk.U, got), k


@pytest.mark.parametrize("precision", [0, 1])
def test_state_changed_between_steps(precision):
    """The uniform box stepped once (which leaves the handle's record of its
    stage state), then one cell of U perturbed by the caller and the ghosts
    refilled, then stepped again: the second step must see the change (the
    disturbed subgrid and its neighbours are no longer uniform), against the
    oracle, with the ghosts bitwise."""
    import torch
    from paper_2210_06439_gb300 import binding
    p = _uniform_box(1.0)
    ref = oracle_filled(p)
    U = torch.from_numpy(ref.U.copy()).cuda()
    H = binding.Hydro.from_problem(p, precision=precision)
    oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=p.bc, nbr=p.nbr)
    H.rk_step(U)
    # perturb the density and energy of one interior cell of subgrid 5, on both sides
    B = 14
    for arr in (ref.U,):
        blk = arr[ref.off[5]: ref.off[5] + ref.nf * B ** 3].reshape(ref.nf, B, B, B)
        blk[0, 6, 5, 7] *= 1.25
        blk[4, 6, 5, 7] *= 1.25
    oracle.ghost_fill(8, ref.off, ref.nf, ref.nbr, ref.U)
    U.copy_(torch.from_numpy(ref.U))
    dt_o, _, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=p.bc, nbr=p.nbr)
    assert st == 0
    dt_g = H.rk_step(U)
    assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else 2e-6)
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-5)), errs
    gi = interior_layout(got, p).reshape(p.n_sub, p.nf, -1)
    assert not np.all(gi[5] == gi[5][:, :1])  # the disturbance is there
    chk = p.copy()
    chk.U[:] = got
    oracle.ghost_fill(8, chk.off, chk.nf, chk.nbr, chk.U)
    assert np.array_equal(chk.U, got)
