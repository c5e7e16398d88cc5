"""Handles of different field counts alive at the same time.

The RHS kernel's dynamic shared memory depends on the field count, and its
launch limit is a process-wide attribute of each kernel instance.  Creating a
handle with fewer fields must not lower that limit under a live handle with
more fields: the 11-field handle's RHS and RK3 step, run after a 6-field
handle was created, still match the oracle."""
import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.helpers import e3s, field_errors, interior_layout, oracle_filled

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.mark.parametrize("precision", [0, 1])
def test_smaller_handle_created_later_leaves_the_larger_one_working(precision):
    import torch
    from paper_2210_06439_gb300 import binding

    big = inputs.periodic_box(nsub=2, n_species=5)
    small = inputs.periodic_box(nsub=2, n_species=0)
    H11 = binding.Hydro.from_problem(big, precision=precision)
    for mode_probe in range(2):  # the 6-field handle created after, and used in between
        H6 = binding.Hydro.from_problem(small, precision=precision)
        U6 = torch.from_numpy(small.U).cuda()
        H6.fill_ghosts(U6)
        d6 = torch.zeros(H6.rhs_len, dtype=torch.float64, device="cuda")
        H6.rhs(U6, d6)
        torch.cuda.synchronize()
        if mode_probe == 0:
            H6.close()
    # RHS of the 11-field handle
    ref = oracle_filled(big)
    d_o, am_o, nb = oracle.rhs(ref.edge, ref.off, ref.dx, ref.nf, ref.U)
    assert nb == 0
    U = torch.from_numpy(big.U).cuda()
    H11.fill_ghosts(U)
    d = torch.zeros(H11.rhs_len, dtype=torch.float64, device="cuda")
    H11.rhs(U, d)
    torch.cuda.synchronize()
    errs = field_errors(d.cpu().numpy(), d_o, big.nf, e3s(big))
    assert np.all(errs <= TOL[precision]), errs
    # and one RK3 step (graph captured now, after the 6-field handle exists)
    st = torch.cuda.Stream()
    U0 = ref.U.copy()
    dt_o, fired, rc = oracle.rk3_step(ref.edge, ref.off, ref.dx, ref.nf, ref.U, bc=1, nbr=ref.nbr)
    assert rc == 0 and fired == 0
    Ug = torch.from_numpy(U0).cuda()
    dt_g = H11.rk_step(Ug, stream=st)
    assert dt_g == pytest.approx(dt_o, rel=1e-12 if precision == 0 else 1e-5)
    errs = field_errors(interior_layout(Ug.cpu().numpy(), big), interior_layout(ref.U, big), big.nf, e3s(big))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-6)), errs
    assert H11.error_flags() == 0
    # the 6-field handle of the second round is still alive and still right
    ref6 = oracle_filled(small)
    d6_o, _, _ = oracle.rhs(ref6.edge, ref6.off, ref6.dx, ref6.nf, ref6.U)
    H6.rhs(U6, d6)
    torch.cuda.synchronize()
    errs6 = field_errors(d6.cpu().numpy(), d6_o, small.nf, e3s(small))
    assert np.all(errs6 <= TOL[precision]), errs6
    H6.close()
    H11.close()
