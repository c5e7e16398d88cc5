"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: FP64 form 1e-12 max relative error per field (error
normalised by the field's max |oracle| over the batch); mixed form 1e-5;
signal speeds and dt at the tolerance of a_q."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.helpers import e3s, field_errors, interior_layout, oracle_filled, MIXED_SPEED_RTOL

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def _torch():
    import torch
    return torch


def _hydro(prob, precision=0, **kw):
    from paper_2210_06439_gb300 import binding
    return binding.Hydro.from_problem(prob, precision=precision, **kw)


def _gpu_rhs(prob, precision=0, fill=True):
    torch = _torch()
    H = _hydro(prob, precision)
    U = torch.from_numpy(prob.U).cuda()
    if fill:
        H.fill_ghosts(U)
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    am = torch.zeros(prob.n_sub, dtype=torch.float64, device="cuda")
    H.rhs(U, d, am)
    torch.cuda.synchronize()
    flags = H.error_flags()
    return d.cpu().numpy(), am.cpu().numpy(), flags, H, U


def _check_rhs(prob, precision, tol=None):
    ref = oracle_filled(prob)
    d_o, am_o, nb = oracle.rhs(ref.edge, ref.off, ref.dx, ref.nf, ref.U, gamma=ref.gamma, nthreads=0)
    assert nb == 0
    d_g, am_g, flags, _, _ = _gpu_rhs(prob, precision)
    assert flags == 0
    errs = field_errors(d_g, d_o, prob.nf, e3s(prob))
    tol = TOL[precision] if tol is None else tol
    assert np.all(errs <= tol), errs
    np.testing.assert_allclose(am_g, am_o, rtol=1e-12 if precision == 0 else MIXED_SPEED_RTOL)
    return errs


@pytest.mark.parametrize("precision", [0, 1])
def test_sod_jump_single_subgrid(precision):
    _check_rhs(inputs.sod_jump(), precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_periodic_box_2x2x2(precision):
    _check_rhs(inputs.periodic_box(nsub=2), precision)


@pytest.mark.parametrize("edge", [12, 16])
@pytest.mark.parametrize("precision", [0, 1])
def test_periodic_box_larger_edges(edge, precision):
    _check_rhs(inputs.periodic_box(nsub=2, E=edge), precision)


def test_periodic_box_64_full_fp64():
    _check_rhs(inputs.periodic_box(), 0)


def test_uniform_state_exactly_zero_on_gpu():
    for prec in (0, 1):
        p = inputs.uniform_state(nsub=(2, 2, 1), v=(0.7, -0.4, 0.25))
        d, am, flags, _, _ = _gpu_rhs(p, prec)
        assert flags == 0
        assert np.all(d == 0.0)


def test_ghost_fill_bitwise():
    torch = _torch()
    for p in (inputs.periodic_box(nsub=2), inputs.binary_star(nsub=2)):
        ref = oracle_filled(p)
        H = _hydro(p)
        U = torch.from_numpy(p.U).cuda()
        H.fill_ghosts(U)
        assert np.array_equal(U.cpu().numpy(), ref.U)


def test_max_dt_matches_oracle():
    p = inputs.periodic_box(nsub=2)
    ref = oracle_filled(p)
    _, am, _ = oracle.rhs(ref.edge, ref.off, ref.dx, ref.nf, ref.U)
    dt_o = oracle.dt_from_amax(ref.dx, am, 0.4)
    torch = _torch()
    H = _hydro(p)
    U = torch.from_numpy(ref.U).cuda()
    dt_g = H.max_dt(U)
    assert dt_g == pytest.approx(dt_o, rel=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_rk3_step_periodic_matches_oracle_and_conserves(precision):
    torch = _torch()
    p = inputs.periodic_box(nsub=2)
    ref = oracle_filled(p)
    U0 = ref.U.copy()
    dt_o, fired, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=1, nbr=ref.nbr)
    assert st == 0 and fired == 0
    H = _hydro(p, precision)
    U = torch.from_numpy(U0).cuda()
    dt_g = H.rk_step(U)
    assert H.error_flags() == 0
    assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else MIXED_SPEED_RTOL)
    got = U.cpu().numpy()
    gi, ri = interior_layout(got, p), interior_layout(ref.U, p)
    errs = field_errors(gi, ri, p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs
    # ghosts refreshed consistently with the interior
    chk = p.copy()
    chk.U[:] = got
    oracle.ghost_fill(8, chk.off, chk.nf, chk.nbr, chk.U)
    assert np.array_equal(chk.U, got)
    # conservation of mass, momentum, energy
    g1 = interior_layout(got, p).reshape(p.n_sub, p.nf, -1)
    g0 = interior_layout(U0, p).reshape(p.n_sub, p.nf, -1)
    lim = 1e-14 if precision == 0 else 1e-13
    for f in range(5):
        scale = math.fsum(np.abs(g0[:, f]).ravel())
        assert abs(math.fsum(g1[:, f].ravel()) - math.fsum(g0[:, f].ravel())) <= lim * scale, f


def test_rk3_graph_replay_is_deterministic():
    torch = _torch()
    p = oracle_filled(inputs.periodic_box(nsub=2))
    H = _hydro(p)
    outs = []
    for _ in range(2):
        U = torch.from_numpy(p.U).cuda()
        for _ in range(3):
            H.rk_step(U, want_dt=False)
        torch.cuda.synchronize()
        outs.append(U.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_mixed_levels_sampled_cells():
    torch = _torch()
    p = inputs.mixed_levels(n=96)
    d_g, am_g, flags, _, _ = _gpu_rhs(p, 0, fill=False)
    assert flags == 0
    rng = np.random.default_rng(5)
    smp = np.stack([rng.integers(0, p.n_sub, 200), np.zeros(200, np.int64)], axis=1)
    smp[:, 1] = [rng.integers(0, int(p.edge[s]) ** 3) for s in smp[:, 0]]
    ref = oracle.rhs_cells(p.edge, p.off, p.dx, p.nf, p.U, smp)
    doff = np.concatenate([[0], np.cumsum(p.nf * p.edge.astype(np.int64) ** 3)])
    for i, (s, c) in enumerate(smp):
        E3 = int(p.edge[s]) ** 3
        g = d_g[doff[s] + c + E3 * np.arange(p.nf)]
        np.testing.assert_allclose(g, ref[i], rtol=1e-11, atol=1e-12 * np.max(np.abs(ref[i])))


@pytest.mark.parametrize("precision", [0, 1])
def test_binary_star_small(precision):
    _check_rhs(inputs.binary_star(nsub=4), precision)


def test_fp64_fields_of_one_value_are_skipped_exactly(tmp_path, monkeypatch):
    """The 32^3 binary star in FP64: in the subgrids the stellar surfaces cut
    through, some fields (z momentum, the species of the other star) hold one
    value over the whole ghosted block, and the handle's RHS reconstructs
    only the other fields. Every stencil of such a field is constant, so
    skipping it must change no bit. So the RHS of every launch shape equals,
    bitwise, that of the allocation-free call (whose kernel has no such
    record and reconstructs every field), and the oracle's within 1e-12."""
    torch = _torch()
    from paper_2210_06439_gb300 import binding
    p = oracle_filled(inputs.binary_star(nsub=4))
    nf, E = p.nf, 8
    skipped = 0
    for s in range(p.n_sub):
        b = p.block(s).reshape(nf, -1).view(np.int64)
        one = np.all(b == b[:, :1], axis=1)
        if not one.all():
            skipped += int(one.sum())
    assert skipped > 0
    U = torch.from_numpy(p.U).cuda()
    L = binding.load()
    dx = torch.from_numpy(np.ascontiguousarray(p.dx)).cuda()
    ref = torch.full((p.n_sub * nf * E ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = L.oct_hydro_rhs_dt_noalloc(p.n_sub, E, p.n_species, p.gamma, 0, 0.4, 1e-3, U.data_ptr(), dx.data_ptr(),
                                    ref.data_ptr(), dt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == binding.OCT_OK
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    d_o, _, _ = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U)
    assert np.all(field_errors(ref, d_o, nf, e3s(p)) <= TOL[0])
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("OCT_HYDRO_TUNE_CACHE", str(path))
    H = _hydro(p, 0)
    path.write_text("")
    H.autotune(U)
    key = path.read_text().split()[0]
    seen = set()
    for mode in range(4):
        path.write_text(f"{key} {mode} 1\n")
        H.autotune(U)
        if H.launch_info()[:2] != (mode, 1):
            continue
        seen.add(mode)
        d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
        H.rhs(U, d)
        torch.cuda.synchronize()
        assert H.error_flags() == 0
        got = d.cpu().numpy()
        assert np.array_equal(got.view(np.int64), ref.view(np.int64)), (mode, np.flatnonzero(got != ref)[:8])
    assert seen == {0, 1, 2, 3}, seen
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_uniform_subgrids_take_the_whole_block_test(precision):
    """The 32^3 binary star (64 subgrids, 48 of them atmosphere): the
    subgrids whose ghosted block holds one value per field (found here with
    numpy) get RHS -0.0, sign bit set, in every cell, as the oracle's full
    formula gives, and the oracle's a_max; the handle's RHS (whole-subgrid
    test ahead of the kernel) and the allocation-free call (the kernel's
    per-item test) agree on them bitwise and elsewhere within the form's
    tolerance."""
    torch = _torch()
    from paper_2210_06439_gb300 import binding
    p = oracle_filled(inputs.binary_star(nsub=4))
    nf, E = p.nf, 8
    blocks = [p.block(s) for s in range(p.n_sub)]
    uni = np.array([all(np.all(b[f].view(np.int64) == b[f].ravel()[0].view(np.int64)) for f in range(nf))
                    for b in blocks])
    assert 8 <= uni.sum() < p.n_sub
    d_o, am_o, _ = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U)
    H = _hydro(p, precision)
    U = torch.from_numpy(p.U).cuda()
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    am = torch.zeros(p.n_sub, dtype=torch.float64, device="cuda")
    H.rhs(U, d, am)
    L = binding.load()
    dx = torch.from_numpy(np.ascontiguousarray(p.dx)).cuda()
    d2 = torch.full((H.rhs_len,), float("nan"), dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = L.oct_hydro_rhs_dt_noalloc(p.n_sub, E, p.n_species, p.gamma, precision, 0.4, 1e-3, U.data_ptr(),
                                    dx.data_ptr(), d2.data_ptr(), dt.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == binding.OCT_OK
    torch.cuda.synchronize()
    g, g2 = d.cpu().numpy().reshape(p.n_sub, -1), d2.cpu().numpy().reshape(p.n_sub, -1)
    o = d_o.reshape(p.n_sub, -1)
    neg0 = np.array([-0.0]).view(np.int64)[0]
    assert np.all(o[uni].view(np.int64) == neg0)
    assert np.all(g[uni].view(np.int64) == neg0) and np.all(g2[uni].view(np.int64) == neg0)
    np.testing.assert_allclose(am.cpu().numpy()[uni], am_o[uni], rtol=1e-12 if precision == 0 else MIXED_SPEED_RTOL)
    errs = field_errors(g2.ravel(), g.ravel(), p.nf, e3s(p))
    assert np.all(errs <= TOL[precision]), errs


def test_nonphysical_input_sets_flag_without_trap():
    torch = _torch()
    p = oracle_filled(inputs.periodic_box(nsub=2))
    p.block(3)[0, 7, 7, 7] = -1.0  # negative density in one interior cell
    H = _hydro(p)
    U = torch.from_numpy(p.U).cuda()
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    H.rhs(U, d)
    torch.cuda.synchronize()
    assert H.error_flags() & 1
    assert H.error_flags() == 0  # read-and-clear


@pytest.mark.parametrize("precision", [0, 1])
def test_rk3_step_with_floor_firings_matches_oracle(precision):
    """The last species slightly below zero (-1e-9 rho) in the lower-x half
    of the periodic box: the floors (rho_i >= 0 after every stage) fire on
    both sides, the GPU raises the floor flag and no other, and the stepped
    state matches the oracle's."""
    torch = _torch()
    p = inputs.periodic_box(nsub=2)
    for s in range(p.n_sub):
        if s % 2 == 0:  # subgrids with x origin 0
            blk = p.block(s)
            blk[10] = -1e-9 * blk[0]
    ref = oracle_filled(p)
    U0 = ref.U.copy()
    dt_o, fired, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=1, nbr=ref.nbr)
    assert st == 0 and fired > 0
    H = _hydro(p, precision)
    U = torch.from_numpy(U0).cuda()
    dt_g = H.rk_step(U)
    flags = H.error_flags()
    assert flags & 2 and not flags & 1
    assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else MIXED_SPEED_RTOL)
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs
    assert np.all(interior_layout(got, p).reshape(p.n_sub, p.nf, -1)[:, 6:] >= 0.0)


def test_dt_cap_applies_to_replayed_graphs():
    """The cap lives in device memory: a captured step follows later changes
    of it, and removing it restores the CFL step of max_dt."""
    torch = _torch()
    p = oracle_filled(inputs.periodic_box(nsub=2))
    H = _hydro(p)
    st = torch.cuda.Stream()
    U = torch.from_numpy(p.U).cuda()
    dt_free = H.max_dt(U, stream=st)
    H.set_dt_cap(dt_free / 4)
    assert H.rk_step(U, stream=st) == dt_free / 4
    H.set_dt_cap(dt_free / 8)
    assert H.rk_step(U, stream=st) == dt_free / 8
    H.set_dt_cap(0.0)
    dt_now = H.max_dt(U, stream=st)
    assert H.rk_step(U, stream=st) == dt_now
    assert H.error_flags() == 0


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n_species", [0, 1, 3])
def test_species_counts(n_species, precision):
    """Field counts other than 11: no species (6 fields), one and three."""
    _check_rhs(inputs.periodic_box(nsub=2, n_species=n_species), precision)


@pytest.mark.parametrize("recon", [0, 1])
def test_dual_energy_switch_over_wide_tau_range(recon):
    """Velocities 2000 times those of the noisy gas law (kinetic energy about
    1e5 times the internal one), so that the dual-energy switch takes
    e_int = tau^gamma at (nearly) every point, with each subgrid's tau scaled
    by its own power of two from 2^-640 to 2^299: the
    cheap tau^(5/3) of the FP64 kernels against the oracle's pow, per
    subgrid, on both sides of the exponent limits of its fast path (2^+-600;
    beyond them the kernels call pow as well)."""
    torch = _torch()
    from paper_2210_06439_gb300 import binding
    p = inputs.mixed_levels(n=9)
    shifts = [-640, -601, -598, -200, -1, 0, 5, 150, 299]
    nf = p.nf
    for s in range(p.n_sub):
        B = int(p.edge[s]) + 6
        blk = p.U[p.off[s]: p.off[s] + nf * B ** 3].reshape(nf, -1)
        rho = blk[0]
        kin = 0.5 * (blk[1] ** 2 + blk[2] ** 2 + blk[3] ** 2) / rho
        eint = blk[4] - kin
        blk[1:4] *= 2000.0
        blk[4] = eint + 0.5 * (blk[1] ** 2 + blk[2] ** 2 + blk[3] ** 2) / rho
        assert np.mean(eint < 1e-3 * blk[4]) > 0.999
        blk[5] *= 2.0 ** shifts[s]
    d_o, am_o, nb = oracle.rhs(p.edge, p.off, p.dx, nf, p.U, nthreads=0, recon=recon)
    assert nb == 0
    H = binding.Hydro.from_problem(p, precision=0, recon=recon)
    U = torch.from_numpy(p.U).cuda()
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    am = torch.zeros(p.n_sub, dtype=torch.float64, device="cuda")
    H.rhs(U, d, am)
    torch.cuda.synchronize()
    assert H.error_flags() == 0
    d_g = d.cpu().numpy()
    o = 0
    for s in range(p.n_sub):
        E3 = int(p.edge[s]) ** 3
        errs = field_errors(d_g[o: o + nf * E3], d_o[o: o + nf * E3], nf, [E3])
        assert np.all(errs <= 1e-12), (s, shifts[s], errs)
        o += nf * E3
    np.testing.assert_allclose(am.cpu().numpy(), am_o, rtol=1e-12)


def _halo_case(case):
    """A uniform state with values changed in one subgrid's block only: a
    ramp of every field across the three ghost layers below x (two rows),
    below z or above y, tau alone in the interior, a species alone in the
    interior, or the block's far corner (read by no stencil).  Returns the
    problem and the changed fields."""
    p = oracle_filled(inputs.uniform_state(nsub=(2, 2, 1), v=(0.3, -0.2, 0.1), n_species=5))
    blk = p.block(1)
    e = 0.3
    fields = list(range(p.nf))
    if case == "x_ramp":
        for k in range(3):
            blk[:, 3, 3:5, k] *= 1 + e * (3 - k)
    elif case == "z_ramp":
        for k in range(3):
            blk[:, k, 5, 6] *= 1 + e * (3 - k)
    elif case == "y_ramp":
        for k in range(3):
            blk[:, 6, 13 - k, 4] *= 1 + e * (3 - k)
    elif case == "interior_tau":
        blk[5, 7, 6, 5] *= 1 + e
        fields = [5]
    elif case == "interior_species":
        blk[7, 7, 7, 7] *= 1 + e
        fields = [7]
    else:
        blk[:, 0, 0, 0] *= 1 + e
        fields = []
    return p, fields


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["x_ramp", "z_ramp", "y_ramp", "interior_tau", "interior_species", "corner"])
def test_uniform_column_test_sees_every_value_read(case, precision):
    """Work items whose column (the tile, its 3-cell halo, every field) holds
    one value per field write their RHS and signal speed without the
    reconstruction.  Here one subgrid's block is uniform but for a few
    values in its halo or interior: the items that read them must take the
    full path.  The changed fields match the oracle at the form's tolerance;
    the others (exactly zero in the oracle where only one field changed)
    stay within that tolerance of the changed fields' scale; the corner,
    read by no stencil, leaves the RHS exactly zero."""
    p, fields = _halo_case(case)
    d_o, am_o, nb = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U)
    assert nb == 0
    d_g, am_g, flags, _, _ = _gpu_rhs(p, precision, fill=False)
    assert flags == 0
    np.testing.assert_allclose(am_g, am_o, rtol=1e-12 if precision == 0 else MIXED_SPEED_RTOL)
    if not fields:
        assert not np.any(d_o) and not np.any(d_g)
        return
    errs = field_errors(d_g, d_o, p.nf, e3s(p))
    assert np.all(errs[fields] <= TOL[precision]), errs
    G = d_g.reshape(p.n_sub, p.nf, -1)
    O = d_o.reshape(p.n_sub, p.nf, -1)
    scale = max(float(np.max(np.abs(O[:, f]))) for f in fields)
    assert scale > 0
    for f in range(p.nf):
        assert np.max(np.abs(G[:, f] - O[:, f])) <= TOL[precision] * scale, f


def test_host_buffer_calls_match_device_calls_bitwise():
    """oct_hydro_rk_steps_host and oct_hydro_rhs_host on a pinned host state
    of 124 MB give the same bits as oct_hydro_rk_step and oct_hydro_rhs on a
    device copy of it."""
    torch = _torch()
    p = oracle_filled(inputs.periodic_box())
    H = _hydro(p)
    st = torch.cuda.Stream()
    U = torch.from_numpy(p.U.copy()).cuda()
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    H.rhs(U, d, stream=st)
    for _ in range(2):
        H.rk_step(U, want_dt=False, stream=st)
    torch.cuda.synchronize()
    Uh = torch.from_numpy(p.U.copy()).pin_memory()
    dh = torch.zeros(H.rhs_len, dtype=torch.float64).pin_memory()
    H.rhs_host(Uh, dh, stream=st)
    H.rk_steps_host(Uh, 2, stream=st)
    assert torch.equal(dh, d.cpu())
    assert torch.equal(Uh, U.cpu())
    assert H.error_flags() == 0


def test_host_step_copies_interior_planes_and_refills_ghosts():
    """On a uniform level in the contiguous layout, oct_hydro_rk_steps_host
    copies in only the interior z-planes of each field block and fills the
    ghosts on the device: a host state whose ghost cells hold NaN steps to
    the same bits as one with valid ghosts, and as oct_hydro_rk_step on the
    device.  Another layout (blocks in reverse order) copies the whole
    state."""
    torch = _torch()
    p = oracle_filled(inputs.periodic_box(nsub=2))
    H = _hydro(p)
    E, B = 8, 14
    h2d, d2h = H.host_copy_bytes()
    assert h2d == p.n_sub * p.nf * E * B * B * 8 and d2h == p.U.nbytes
    good = torch.from_numpy(p.U.copy()).pin_memory()
    bad = good.clone().pin_memory()
    for s in range(p.n_sub):
        blk = bad[p.off[s]: p.off[s] + p.nf * B ** 3].view(p.nf, B, B, B)
        blk[:, :3] = float("nan")
        blk[:, 3 + E:] = float("nan")
        blk[:, 3:3 + E, :3] = float("nan")
        blk[:, 3:3 + E, :, 3 + E:] = float("nan")
    H.rk_steps_host(good, 1)
    H.rk_steps_host(bad, 1)
    assert torch.equal(good, bad)
    U = torch.from_numpy(p.U.copy()).cuda()
    H.rk_step(U)
    assert torch.equal(good, U.cpu())
    assert H.error_flags() == 0
    q = p.copy()
    q.off = np.ascontiguousarray(p.off[::-1])
    Hq = _hydro(q)
    assert Hq.host_copy_bytes() == (p.U.nbytes, p.U.nbytes)
