"""The allocation-free RHS + dt entry point (oct_hydro_rhs_dt_noalloc) gives
the same results as the handle-based oct_hydro_rhs and oct_hydro_max_dt.

It serves callers that cannot call cudaMalloc on their hot path (a host
program whose device memory is all owned by its own pool allocator, or one
that must avoid the implicit synchronisation cudaMalloc/cudaFree can cause):
its scratch is a fixed device array inside the library.  Two calls in a row,
with different batch shapes, check that the shared scratch left by one call
does not leak into the next; edge 12 (four 6x6 tiles per subgrid) is among
them.  A call made after a handle with fewer fields was created checks that
the kernels' launch limits stay large enough for 11 fields.  This file is
named to be collected last."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.helpers import e3s, field_errors, oracle_filled

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def test_noalloc_matches_handle_entry_points_on_two_calls_in_a_row():
    import torch
    from paper_2210_06439_gb300 import binding, inputs

    L = binding.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(1002, 2, 8, binding.OCT_FP64), (1005, 2, 16, binding.OCT_MIXED), (1004, 2, 12, binding.OCT_FP64),
             (1004, 2, 12, binding.OCT_MIXED)]
    for seed, nsub, E, prec in cases:
        p = inputs.periodic_box(seed=seed, nsub=nsub, E=E)
        H = binding.Hydro.from_problem(p, precision=prec)
        U = torch.from_numpy(p.U).cuda()
        H.fill_ghosts(U)
        ref = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
        H.rhs(U, ref)
        dt_ref = H.max_dt(U)
        dx = torch.from_numpy(np.ascontiguousarray(p.dx)).cuda()
        out = torch.full((H.rhs_len,), float("nan"), dtype=torch.float64, device="cuda")
        dt = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.oct_hydro_rhs_dt_noalloc(p.n_sub, E, p.n_species, p.gamma, prec, 0.4, 1e-3, U.data_ptr(),
                                        dx.data_ptr(), out.data_ptr(), dt.data_ptr(), stream)
        assert st == binding.OCT_OK, L.oct_hydro_last_error().decode()
        torch.cuda.synchronize()
        errs = field_errors(out.cpu().numpy(), ref.cpu().numpy(), p.nf, e3s(p))
        assert np.all(errs <= TOL[prec]), errs
        assert float(dt.item()) == pytest.approx(dt_ref, rel=TOL[prec])
        H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_after_a_smaller_handle_matches_oracle(precision):
    """A 6-field handle created (and used) first; then the allocation-free
    call with 11 fields, checked against the oracle itself."""
    import torch
    from paper_2210_06439_gb300 import binding

    L = binding.load()
    small = inputs.periodic_box(nsub=2, n_species=0)
    H6 = binding.Hydro.from_problem(small, precision=precision)
    U6 = torch.from_numpy(small.U).cuda()
    H6.fill_ghosts(U6)
    d6 = torch.zeros(H6.rhs_len, dtype=torch.float64, device="cuda")
    H6.rhs(U6, d6)
    p = oracle_filled(inputs.periodic_box(nsub=2, n_species=5))
    d_o, am_o, nb = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U)
    assert nb == 0
    dt_o = oracle.dt_from_amax(p.dx, am_o, 0.4)
    U = torch.from_numpy(p.U).cuda()
    dx = torch.from_numpy(np.ascontiguousarray(p.dx)).cuda()
    out = torch.full((p.rhs_len,), float("nan"), dtype=torch.float64, device="cuda")
    dt = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = L.oct_hydro_rhs_dt_noalloc(p.n_sub, 8, p.n_species, p.gamma, precision, 0.4, 1e-3, U.data_ptr(),
                                    dx.data_ptr(), out.data_ptr(), dt.data_ptr(), stream)
    assert st == binding.OCT_OK, L.oct_hydro_last_error().decode()
    torch.cuda.synchronize()
    errs = field_errors(out.cpu().numpy(), d_o, p.nf, e3s(p))
    assert np.all(errs <= TOL[precision]), errs
    assert float(dt.item()) == pytest.approx(dt_o, rel=1e-12 if precision == 0 else 1e-5)
    H6.close()


def test_noalloc_rejects_batches_beyond_its_scratch():
    from paper_2210_06439_gb300 import binding

    L = binding.load()
    st = L.oct_hydro_rhs_dt_noalloc(4097, 8, 5, 5.0 / 3.0, 0, 0.4, 1e-3, 16, 16, 4096, 16, None)
    assert st == binding.OCT_E_ARG
    assert "4096" in L.oct_hydro_last_error().decode()
