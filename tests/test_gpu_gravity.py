"""Same-level monopole gravity on the GPU (oct_hydro_gravity_monopole)
against the oracle (reading R18), element by element: the potential and the
three acceleration components, each at 1e-12 of its max |oracle| over the
batch; edges 8, 12 and 16, several interaction radii (the stencil rebuilt
between calls), periodic and outflow layouts, and the 128^3 binary star in
full."""
import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs

pytestmark = pytest.mark.gpu

RS = 2.0 / 0.34


def _gpu(p, r_s, G=1.0, H=None):
    import torch
    from paper_2210_06439_gb300 import binding
    H = H or binding.Hydro.from_problem(p)
    U = torch.from_numpy(p.U).cuda()
    E3 = int(p.edge[0]) ** 3
    phi = torch.full((p.n_sub * E3,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full((3 * p.n_sub * E3,), float("nan"), dtype=torch.float64, device="cuda")
    H.gravity_monopole(U, phi, g, G=G, r_s=r_s)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), g.cpu().numpy(), H


def _check(p, r_s, G=1.0, H=None):
    E = int(p.edge[0])
    phi_o, g_o = oracle.gravity_monopole(E, p.off, p.nf, p.nbr, float(p.dx[0]), p.U, G=G, r_s=r_s)
    phi, g, H = _gpu(p, r_s, G, H)
    n, E3 = p.n_sub, E ** 3
    gg, go = g.reshape(n, 3, E3), g_o.reshape(n, 3, E3)
    errs = [np.max(np.abs(phi - phi_o)) / np.max(np.abs(phi_o))]
    errs += [np.max(np.abs(gg[:, a] - go[:, a])) / np.max(np.abs(go[:, a])) for a in range(3)]
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))
    assert max(errs) <= 1e-12, errs
    return H, errs


@pytest.mark.parametrize("E", [8, 12, 16])
def test_periodic_box_matches_oracle(E):
    _check(inputs.periodic_box(nsub=2, E=E), RS)


def test_outflow_binary_star_and_radius_changes():
    p = inputs.binary_star(4)
    H, _ = _check(p, RS, G=1.0)
    for r_s in (3.0, 8.0, 1.0, RS):  # the stencil is rebuilt for each
        _check(p, r_s, G=0.5, H=H)


def test_binary_star_128_every_cell():
    p = inputs.binary_star(16)
    _, errs = _check(p, RS)
    print("\nbinary_star_128 monopole gravity max rel err (phi, gx, gy, gz):", " ".join(f"{e:.2e}" for e in errs))


def test_rejects_bad_calls():
    import torch
    from paper_2210_06439_gb300 import binding
    p = inputs.periodic_box(nsub=2)
    H = binding.Hydro.from_problem(p)
    U = torch.from_numpy(p.U).cuda()
    out = torch.zeros(3 * p.n_sub * 512, dtype=torch.float64, device="cuda")
    for r_s in (0.5, 9.0, float("nan")):
        with pytest.raises(binding.OctError) as e:
            H.gravity_monopole(U, out, out, r_s=r_s)
        assert e.value.status == binding.OCT_E_ARG
    with pytest.raises(binding.OctError):
        H.gravity_monopole(U, out, out, G=-1.0)
    # ghosts given: no neighbour table
    q = inputs.mixed_levels(n=6)
    Hq = binding.Hydro.from_problem(q)
    Uq = torch.from_numpy(q.U).cuda()
    with pytest.raises(binding.OctError) as e:
        Hq.gravity_monopole(Uq, out, out)
    assert e.value.status == binding.OCT_E_STATE
