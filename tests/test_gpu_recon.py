"""Primitive reconstruction on the GPU (the optional variable choice: PPM on
w = (rho, v, p, tau, X_i), points turned back into conserved fields) against
the oracle with the same choice, in both precisions."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.helpers import MIXED_SPEED_RTOL, e3s, field_errors, interior_layout, oracle_filled
from tests.test_oracle_recon import shear_flow

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def _gpu_rhs(p, precision):
    import torch
    from paper_2210_06439_gb300 import binding
    H = binding.Hydro.from_problem(p, precision=precision, recon=binding.OCT_RECON_PRIMITIVE)
    U = torch.from_numpy(p.U).cuda()
    if p.bc != 0:
        H.fill_ghosts(U)
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    am = torch.zeros(p.n_sub, dtype=torch.float64, device="cuda")
    H.rhs(U, d, am)
    torch.cuda.synchronize()
    return d.cpu().numpy(), am.cpu().numpy(), H.error_flags()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("make", [lambda: inputs.periodic_box(nsub=2), lambda: inputs.periodic_box(),
                                  lambda: inputs.binary_star(4), lambda: inputs.sod_jump()],
                         ids=["box16", "box64", "binary32", "sod_jump"])
def test_rhs_matches_oracle(make, precision):
    p = make()
    ref = oracle_filled(p)
    d_o, am_o, nb = oracle.rhs(ref.edge, ref.off, ref.dx, ref.nf, ref.U, gamma=ref.gamma, recon=1)
    assert nb == 0
    d_g, am_g, flags = _gpu_rhs(p, precision)
    assert flags == 0
    errs = field_errors(d_g, d_o, p.nf, e3s(p))
    assert np.all(errs <= TOL[precision]), errs
    np.testing.assert_allclose(am_g, am_o, rtol=1e-12 if precision == 0 else MIXED_SPEED_RTOL)


@pytest.mark.parametrize("precision", [0, 1])
def test_shear_flow_exact_zeros(precision):
    """The closed form the oracle is pinned to: in a pure shear flow the mass,
    x/z-momentum, tau and species RHS are exactly zero."""
    p = shear_flow()
    d_g, _, flags = _gpu_rhs(p, precision)
    assert flags == 0
    d = d_g.reshape(p.n_sub, p.nf, -1)
    for f in (0, 1, 3, 5, 6, 7, 8, 9, 10):
        assert not np.any(d[:, f]), f
    assert np.any(d[:, 2])


@pytest.mark.parametrize("precision", [0, 1])
def test_rk3_step_matches_oracle_and_conserves(precision):
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.periodic_box(nsub=2)
    ref = oracle_filled(p)
    U0 = ref.U.copy()
    dt_o, fired, st = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=1, nbr=ref.nbr, recon=1)
    assert st == 0 and fired == 0
    H = binding.Hydro.from_problem(p, precision=precision, recon=binding.OCT_RECON_PRIMITIVE)
    U = torch.from_numpy(U0).cuda()
    dt_g = H.rk_step(U)
    assert H.error_flags() == 0
    assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else MIXED_SPEED_RTOL)
    got = U.cpu().numpy()
    errs = field_errors(interior_layout(got, p), interior_layout(ref.U, p), p.nf, e3s(p))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs
    g1 = interior_layout(got, p).reshape(p.n_sub, p.nf, -1)
    g0 = interior_layout(U0, p).reshape(p.n_sub, p.nf, -1)
    lim = 1e-14 if precision == 0 else 1e-13
    for f in range(5):
        scale = math.fsum(np.abs(g0[:, f]).ravel())
        assert abs(math.fsum(g1[:, f].ravel()) - math.fsum(g0[:, f].ravel())) <= lim * scale, f


def test_switching_back_to_conserved_fields():
    import torch
    from paper_2210_06439_gb300 import binding
    p = oracle_filled(inputs.periodic_box(nsub=2))
    d_c, _, _ = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U)
    H = binding.Hydro.from_problem(p, recon=binding.OCT_RECON_PRIMITIVE)
    H.set_reconstruction(binding.OCT_RECON_CONSERVED)
    U = torch.from_numpy(p.U).cuda()
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    H.rhs(U, d)
    torch.cuda.synchronize()
    assert np.all(field_errors(d.cpu().numpy(), d_c, p.nf, e3s(p)) <= 1e-12)
    with pytest.raises(binding.OctError):
        H.set_reconstruction(2)
