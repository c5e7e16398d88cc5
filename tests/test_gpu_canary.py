"""Out-of-bounds detection without a sanitizer: every subgrid block sits
between guard regions filled with a NaN canary, and the RHS output between
guards holding a fixed pattern.  A kernel that read outside a block would
pull the NaN into its results (parity with the oracle fails); one that wrote
outside would change a guard.  Subgrids are also laid out in reverse order
with uneven gaps, so that no kernel can rely on packed, ordered blocks."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.helpers import e3s, field_errors, interior_layout

pytestmark = pytest.mark.gpu

CANARY = np.frombuffer(np.uint64(0x7FF8DEADBEEF0001).tobytes(), np.float64)[0]  # a quiet NaN
GUARD = 4096.5


def _spread(p, seed=3):
    """The same problem with its blocks in reverse order and NaN-filled gaps of
    4 to 256 doubles (multiples of 4) before, between and after them."""
    rng = np.random.default_rng(seed)
    sizes = [p.nf * (int(E) + 6) ** 3 for E in p.edge]
    order = list(range(p.n_sub))[::-1]
    off = np.zeros(p.n_sub, np.int64)
    o = int(rng.integers(1, 65)) * 4
    for s in order:
        off[s] = o
        o += (sizes[s] + 3) // 4 * 4 + int(rng.integers(1, 65)) * 4
    U = np.full(o + 256, CANARY)
    for s in range(p.n_sub):
        U[off[s]: off[s] + sizes[s]] = p.U[p.off[s]: p.off[s] + sizes[s]]
    q = dataclasses.replace(p, off=off, U=U)
    mask = np.ones(U.size, bool)
    for s in range(p.n_sub):
        mask[off[s]: off[s] + sizes[s]] = False
    return q, mask


def _run(q, precision, recon, amr):
    import torch
    from paper_2210_06439_gb300 import binding
    H = binding.Hydro.from_problem(q, precision=precision, recon=recon)
    U = torch.from_numpy(q.U).cuda()
    H.fill_ghosts(U)
    pad = 512
    dbuf = torch.full((H.rhs_len + 2 * pad,), GUARD, dtype=torch.float64, device="cuda")
    d = dbuf[pad: pad + H.rhs_len]
    H.rhs(U, d)
    dt = H.max_dt(U)
    U1 = U.clone()
    H.rk_step(U1)
    H.rk_step(U1)
    torch.cuda.synchronize()
    assert H.error_flags() == 0
    db = dbuf.cpu().numpy()
    assert np.all(db[:pad] == GUARD) and np.all(db[pad + H.rhs_len:] == GUARD)
    return U.cpu().numpy(), db[pad: pad + H.rhs_len], dt, U1.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("recon", [0, 1])
def test_uniform_level_guards(precision, recon):
    p = inputs.periodic_box(nsub=2)
    q, mask = _spread(p)
    Ug, d_g, dt_g, U1 = _run(q, precision, recon, False)
    # nothing outside the blocks was written, by the fill, the RHS or the steps
    gb = q.U.view(np.uint64)[mask]
    assert np.all(Ug.view(np.uint64)[mask] == gb)
    assert np.all(U1.view(np.uint64)[mask] == gb)
    # and nothing outside was read: the results are finite and match the oracle
    ref = q.copy()
    oracle.ghost_fill(8, ref.off, ref.nf, ref.nbr, ref.U)
    d_o, _, _ = oracle.rhs(ref.edge, ref.off, ref.dx, ref.nf, ref.U, recon=recon)
    errs = field_errors(d_g, d_o, q.nf, e3s(q))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-5)), errs
    assert np.all(np.isfinite(interior_layout(U1, q)))


@pytest.mark.parametrize("precision", [0, 1])
def test_two_level_guards(precision):
    p = inputs.amr_box()
    q, mask = _spread(p, seed=5)
    Ug, d_g, _, U1 = _run(q, precision, 0, True)
    gb = q.U.view(np.uint64)[mask]
    assert np.all(Ug.view(np.uint64)[mask] == gb)
    assert np.all(U1.view(np.uint64)[mask] == gb)
    m = q.meta
    ref = q.copy()
    oracle.amr_ghost_fill(8, ref.off, ref.nf, m["level"], m["origin"], m["n0"], m["periodic"], ref.U)
    d_o, _, F, _ = oracle.rhs_faces(ref.edge, ref.off, ref.dx, ref.nf, ref.U)
    oracle.amr_reflux(8, ref.dx, ref.nf, m["level"], m["origin"], m["n0"], m["periodic"], F, d_o)
    errs = field_errors(d_g, d_o, q.nf, e3s(q))
    assert np.all(errs <= (1e-12 if precision == 0 else 1e-5)), errs
    assert np.all(np.isfinite(interior_layout(U1, q)))
