"""Ghost exchange across refinement levels on the GPU (Sec. II
"Data-Structure": octree leaves one level coarser or finer than their
neighbours) against the oracle: the fill bit for bit, then the RHS with the
flux correction at coarse-fine faces and SSP-RK3 steps on the two-level box
with the fill inside the step, and their conservation."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.helpers import e3s, field_errors, interior_layout, MIXED_SPEED_RTOL

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def _oracle_fill(p):
    m = p.meta
    q = p.copy()
    oracle.amr_ghost_fill(int(p.edge[0]), q.off, q.nf, m["level"], m["origin"], m["n0"], m["periodic"], q.U)
    return q


@pytest.mark.parametrize("periodic", [True, False])
def test_amr_fill_bitwise(periodic):
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.amr_box(periodic=periodic)
    ref = _oracle_fill(p)
    H = binding.Hydro.from_problem(p)
    U = torch.from_numpy(p.U).cuda()
    for _ in range(2):  # a second fill from filled ghosts changes nothing
        H.fill_ghosts(U)
        torch.cuda.synchronize()
        assert np.array_equal(U.cpu().numpy(), ref.U)


@pytest.mark.parametrize("precision", [0, 1])
def test_amr_rhs_matches_oracle(precision):
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.amr_box()
    ref = _oracle_fill(p)
    m = p.meta
    d_o, am_o, F, nb = oracle.rhs_faces(ref.edge, ref.off, ref.dx, ref.nf, ref.U, gamma=ref.gamma)
    assert nb == 0
    oracle.amr_reflux(8, ref.dx, ref.nf, m["level"], m["origin"], m["n0"], m["periodic"], F, d_o)
    H = binding.Hydro.from_problem(p, precision=precision)
    U = torch.from_numpy(p.U).cuda()
    H.fill_ghosts(U)
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    am = torch.zeros(p.n_sub, dtype=torch.float64, device="cuda")
    H.rhs(U, d, am)
    torch.cuda.synchronize()
    assert H.error_flags() == 0
    errs = field_errors(d.cpu().numpy(), d_o, p.nf, e3s(p))
    assert np.all(errs <= TOL[precision]), errs
    np.testing.assert_allclose(am.cpu().numpy(), am_o, rtol=1e-12 if precision == 0 else MIXED_SPEED_RTOL)


@pytest.mark.parametrize("precision", [0, 1])
def test_amr_rk3_step_matches_oracle(precision):
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.amr_box()
    ref = _oracle_fill(p)
    U0 = ref.U.copy()
    m = p.meta
    dts = []
    for _ in range(2):
        dt, fired, st = oracle.rk3_step_amr(ref.edge, ref.off, ref.dx, ref.nf, ref.U, m["level"], m["origin"],
                                            m["n0"], m["periodic"], gamma=ref.gamma)
        assert st == 0 and fired == 0
        dts.append(dt)
    H = binding.Hydro.from_problem(p, precision=precision)
    U = torch.from_numpy(U0).cuda()
    st = torch.cuda.Stream()
    dg = [H.rk_step(U, stream=st) for _ in range(2)]
    torch.cuda.synchronize()
    assert H.error_flags() == 0
    np.testing.assert_allclose(dg, dts, rtol=1e-12 if precision == 0 else MIXED_SPEED_RTOL)
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs
    # ghosts left consistent with the interior by the fill inside the step
    chk = p.copy()
    chk.U[:] = got
    chk = _oracle_fill(chk)
    assert np.array_equal(chk.U, got)


@pytest.mark.parametrize("precision", [0, 1])
def test_amr_rk3_steps_conserve(precision):
    """Three RK3 steps on the periodic two-level box keep the volume
    integrals of mass, momentum and energy to 1e-14 (FP64) or 1e-13 (mixed)
    relative to the integral of their magnitudes."""
    import torch
    from paper_2210_06439_gb300 import binding
    p = _oracle_fill(inputs.amr_box())
    H = binding.Hydro.from_problem(p, precision=precision)
    U = torch.from_numpy(p.U).cuda()
    for _ in range(3):
        H.rk_step(U)
    torch.cuda.synchronize()
    assert H.error_flags() == 0
    w = (p.dx ** 3)[:, None]
    a = interior_layout(p.U, p).reshape(p.n_sub, p.nf, -1)
    b = interior_layout(U.cpu().numpy(), p).reshape(p.n_sub, p.nf, -1)
    lim = 1e-14 if precision == 0 else 1e-13
    for f in range(5):
        t0 = math.fsum((w * a[:, f]).ravel())
        t1 = math.fsum((w * b[:, f]).ravel())
        sc = math.fsum(np.abs(w * a[:, f]).ravel())
        assert abs(t1 - t0) <= lim * sc, (f, (t1 - t0) / sc)


def test_set_amr_rejects_unnested_layouts():
    from paper_2210_06439_gb300 import binding
    p = inputs.periodic_box(nsub=2, E=8)
    H = binding.Hydro.from_problem(p)
    org = np.array([((s % 2) * 8, ((s // 2) % 2) * 8, (s // 4) * 8) for s in range(p.n_sub)], np.int32)
    lev = np.zeros(p.n_sub, np.int32)
    H.set_amr(lev, org, 16, True)  # the uniform tiling is accepted
    with pytest.raises(binding.OctError):
        H.set_amr(lev, org, 32, True)  # 7/8 of the root box has no subgrid
    org2 = org.copy()
    org2[1] = org2[0]
    with pytest.raises(binding.OctError):
        H.set_amr(lev, org2, 16, True)  # two subgrids on one place


@pytest.mark.parametrize("precision", [0, 1])
def test_amr_rhs_primitive_reconstruction(precision):
    """The two variable choices compose with the levels: primitive
    reconstruction on the two-level box, flux correction included."""
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.amr_box()
    ref = _oracle_fill(p)
    m = p.meta
    d_o, am_o, F, nb = oracle.rhs_faces(ref.edge, ref.off, ref.dx, ref.nf, ref.U, gamma=ref.gamma, recon=1)
    assert nb == 0
    oracle.amr_reflux(8, ref.dx, ref.nf, m["level"], m["origin"], m["n0"], m["periodic"], F, d_o)
    H = binding.Hydro.from_problem(p, precision=precision, recon=binding.OCT_RECON_PRIMITIVE)
    U = torch.from_numpy(p.U).cuda()
    H.fill_ghosts(U)
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    am = torch.zeros(p.n_sub, dtype=torch.float64, device="cuda")
    H.rhs(U, d, am)
    torch.cuda.synchronize()
    assert H.error_flags() == 0
    errs = field_errors(d.cpu().numpy(), d_o, p.nf, e3s(p))
    assert np.all(errs <= TOL[precision]), errs
    np.testing.assert_allclose(am.cpu().numpy(), am_o, rtol=1e-12 if precision == 0 else MIXED_SPEED_RTOL)


@pytest.mark.parametrize("E", [12, 16])
def test_amr_fill_bitwise_larger_edges(E):
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.amr_box(n_coarse=4, E=E, n_species=1)
    ref = _oracle_fill(p)
    H = binding.Hydro.from_problem(p)
    U = torch.from_numpy(p.U).cuda()
    H.fill_ghosts(U)
    torch.cuda.synchronize()
    assert np.array_equal(U.cpu().numpy(), ref.U)


@pytest.mark.parametrize("periodic", [True, False])
def test_linear_prolongation_fill_bitwise(periodic):
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.amr_box(periodic=periodic)
    m = p.meta
    ref = p.copy()
    oracle.amr_ghost_fill(8, ref.off, ref.nf, m["level"], m["origin"], m["n0"], m["periodic"], ref.U, order=1)
    H = binding.Hydro.from_problem(p)
    H.set_prolongation(1)
    U = torch.from_numpy(p.U).cuda()
    for _ in range(2):
        H.fill_ghosts(U)
        torch.cuda.synchronize()
        assert np.array_equal(U.cpu().numpy(), ref.U)
    # back to injection: the plan is rebuilt
    H.set_prolongation(0)
    U = torch.from_numpy(p.U).cuda()
    H.fill_ghosts(U)
    torch.cuda.synchronize()
    assert np.array_equal(U.cpu().numpy(), _oracle_fill(p).U)
    with pytest.raises(binding.OctError):
        H.set_prolongation(2)


@pytest.mark.parametrize("precision", [0, 1])
def test_linear_prolongation_rk3_steps_match_oracle(precision):
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.amr_box()
    m = p.meta
    ref = p.copy()
    oracle.amr_ghost_fill(8, ref.off, ref.nf, m["level"], m["origin"], m["n0"], m["periodic"], ref.U, order=1)
    U0 = ref.U.copy()
    dts = []
    for _ in range(2):
        dt, fired, st = oracle.rk3_step_amr(ref.edge, ref.off, ref.dx, ref.nf, ref.U, m["level"], m["origin"],
                                            m["n0"], m["periodic"], gamma=ref.gamma, order=1)
        assert st == 0 and fired == 0
        dts.append(dt)
    H = binding.Hydro.from_problem(p, precision=precision)
    H.set_prolongation(1)
    U = torch.from_numpy(U0).cuda()
    st = torch.cuda.Stream()
    dg = [H.rk_step(U, stream=st) for _ in range(2)]
    torch.cuda.synchronize()
    assert H.error_flags() == 0
    np.testing.assert_allclose(dg, dts, rtol=1e-12 if precision == 0 else MIXED_SPEED_RTOL)
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs


def test_linear_prolongation_is_more_accurate_on_a_smooth_wave():
    """A smooth density wave advected through the coarse-fine faces for a
    quarter period: the limited linear prolongation gives a smaller L1
    density error (against the exact translated wave) than injection."""
    import math
    import torch
    from paper_2210_06439_gb300 import binding
    errs = {}
    for order in (0, 1):
        p = inputs.amr_wave()
        m = p.meta
        H = binding.Hydro.from_problem(p)
        H.set_prolongation(order)
        U = torch.from_numpy(p.U).cuda()
        st = torch.cuda.Stream()
        H.fill_ghosts(U, stream=st)
        t, t_end = 0.0, 0.25
        while t < t_end * (1 - 1e-12):
            H.set_dt_cap(t_end - t)
            t += H.rk_step(U, stream=st)
        torch.cuda.synchronize()
        assert H.error_flags() == 0
        got = interior_layout(U.cpu().numpy(), p).reshape(p.n_sub, p.nf, -1)
        E = 8
        i = np.arange(E)
        tot = vol = 0.0
        for s in range(p.n_sub):
            h = float(p.dx[s])
            xx = np.broadcast_to(((m["origin"][s, 0] + i + 0.5) * h)[None, None, :], (E, E, E)).ravel()
            exact = 1.0 + m["amp"] * np.sin(2.0 * math.pi * (xx - t_end))
            tot += np.sum(np.abs(got[s, 0] - exact)) * h ** 3
            vol += E ** 3 * h ** 3
        errs[order] = tot / vol
    print(f"\nL1(rho) after a quarter period: injection {errs[0]:.3e}, linear {errs[1]:.3e}")
    assert errs[1] < errs[0]
