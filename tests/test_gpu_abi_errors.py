"""Host-side fault handling of the C ABI with a live handle: every bad
argument is rejected with OCT_E_ARG and a message before any launch, and the
handle keeps its previous, valid state (its RHS is unchanged afterwards).
Faults are made on the host only; nothing here can trap the GPU."""
import ctypes

import numpy as np
import pytest

from paper_2210_06439_gb300 import binding, inputs
from tests.helpers import oracle_filled

pytestmark = pytest.mark.gpu

E_ARG = binding.OCT_E_ARG


def _arr(a, t):
    a = np.ascontiguousarray(a, t)
    return a, a.ctypes.data


@pytest.fixture()
def live():
    import torch
    p = oracle_filled(inputs.periodic_box(nsub=2))
    H = binding.Hydro.from_problem(p)
    U = torch.from_numpy(p.U).cuda()
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    H.rhs(U, d)
    torch.cuda.synchronize()
    return H, p, U, d.cpu().numpy()


def _still_valid(H, U, ref):
    import torch
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    H.rhs(U, d)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), ref)
    assert H.error_flags() == 0


def _rejected(status):
    assert status == E_ARG
    assert binding.load().oct_hydro_last_error().decode()


def test_bad_layouts_are_rejected(live):
    H, p, U, ref = live
    L, h, n = H.L, H.h, p.n_sub
    edges, pe = _arr(p.edge, np.int32)
    offs, po = _arr(p.off, np.int64)
    dx, pd = _arr(p.dx, np.float64)
    nbr, pn = _arr(p.nbr, np.int32)
    bad_edge, pbe = _arr(np.where(np.arange(n) == 3, 10, p.edge), np.int32)
    _rejected(L.oct_hydro_set_layout(h, pbe, po, pd, None, pn, 1))
    odd_off, poo = _arr(p.off + np.where(np.arange(n) == 2, 2, 0), np.int64)
    _rejected(L.oct_hydro_set_layout(h, pe, poo, pd, None, pn, 1))
    overlap, pov = _arr(np.where(np.arange(n) == 1, p.off[0], p.off), np.int64)
    _rejected(L.oct_hydro_set_layout(h, pe, pov, pd, None, pn, 1))
    for v in (0.0, -1.0, float("nan")):
        bdx, pbd = _arr(np.where(np.arange(n) == 5, v, p.dx), np.float64)
        _rejected(L.oct_hydro_set_layout(h, pe, po, pbd, None, pn, 1))
    _rejected(L.oct_hydro_set_layout(h, pe, po, pd, None, None, 1))  # periodic without a table
    bnb, pbn = _arr(np.where(np.arange(nbr.size) == 7, n, p.nbr.reshape(-1)), np.int32)
    _rejected(L.oct_hydro_set_layout(h, pe, po, pd, None, pbn, 1))
    for bc in (-1, 3, 7):  # levels go through oct_hydro_set_amr
        _rejected(L.oct_hydro_set_layout(h, pe, po, pd, None, pn, bc))
    _still_valid(H, U, ref)


def test_bad_parameters_and_calls_are_rejected(live):
    import torch
    H, p, U, ref = live
    L, h = H.L, H.h
    for args in [(2, 0.4, 1e-12, 1e-3, 0.1), (0, 0.0, 1e-12, 1e-3, 0.1), (0, 1.5, 1e-12, 1e-3, 0.1),
                 (0, 0.4, -1.0, 1e-3, 0.1), (0, 0.4, 1e-12, 1.0, 0.1), (0, 0.4, 1e-12, 1e-3, -0.5)]:
        _rejected(L.oct_hydro_set_params(h, *args))
    _rejected(L.oct_hydro_set_dt_cap(h, float("nan")))
    _rejected(L.oct_hydro_set_reconstruction(h, 5))
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    _rejected(L.oct_hydro_rhs(h, None, d.data_ptr(), None, None))
    _rejected(L.oct_hydro_rhs(h, U.data_ptr(), None, None, None))
    _rejected(L.oct_hydro_rhs(h, U.data_ptr() + 8, d.data_ptr(), None, None))  # misaligned
    _rejected(L.oct_hydro_rhs(h, U.data_ptr(), U.data_ptr(), None, None))  # overlapping
    _rejected(L.oct_hydro_max_dt(h, U.data_ptr(), None, None))
    _rejected(L.oct_hydro_rk_steps_host(h, None, 1, None, None))
    host = np.zeros(H.state_len)
    _rejected(L.oct_hydro_rk_steps_host(h, host.ctypes.data, -1, None, None))
    _rejected(L.oct_hydro_get_error_flags(h, None))
    _still_valid(H, U, ref)


def test_bad_refinement_layouts_are_rejected(live):
    H, p, U, ref = live
    L, h, n = H.L, H.h, p.n_sub
    org = np.array([((s % 2) * 8, ((s // 2) % 2) * 8, (s // 4) * 8) for s in range(n)], np.int32)
    lev = np.zeros(n, np.int32)
    lv, pl = _arr(lev, np.int32)
    og, pg = _arr(org, np.int32)
    _rejected(L.oct_hydro_set_amr(h, None, pg, 16, 1))
    _rejected(L.oct_hydro_set_amr(h, pl, pg, 12, 1))  # root not a multiple of the edge
    neg, pneg = _arr(np.where(np.arange(n) == 2, -1, lev), np.int32)
    _rejected(L.oct_hydro_set_amr(h, pneg, pg, 16, 1))
    shifted, psh = _arr(org + np.array([4, 0, 0], np.int32), np.int32)
    _rejected(L.oct_hydro_set_amr(h, pl, psh, 16, 1))  # origins off the subgrid lattice
    _still_valid(H, U, ref)


def test_noalloc_rejects_bad_batches():
    import torch
    L = binding.load()
    U = torch.zeros(1024, dtype=torch.float64, device="cuda")
    dx = torch.ones(1, dtype=torch.float64, device="cuda")
    d = torch.zeros(1024, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    args = dict(edge=8, n_species=5, gamma=5.0 / 3.0, precision=0, cfl=0.4, de1=1e-3)
    for n, edge, ns, prec in [(0, 8, 5, 0), (4097, 8, 5, 0), (1, 9, 5, 0), (1, 8, 6, 0), (1, 8, 5, 3)]:
        st = L.oct_hydro_rhs_dt_noalloc(n, edge, ns, args["gamma"], prec, args["cfl"], args["de1"], U.data_ptr(),
                                        dx.data_ptr(), d.data_ptr(), dt.data_ptr(), None)
        _rejected(st)
    _rejected(L.oct_hydro_rhs_dt_noalloc(1, 8, 5, 5.0 / 3.0, 0, 0.4, 1e-3, U.data_ptr(), None, d.data_ptr(),
                                         dt.data_ptr(), None))
