"""Pins of the oracle's primitive reconstruction (reading R16: PPM on
w = (rho, v, p, tau, X_i) of every cell, each point turned back into
conserved fields with its reconstructed v and p).  The method reconstructs
the conserved fields by default (reading R1); primitive reconstruction is
the optional variable choice."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.test_oracle_pins import _filled, _mirror, _mirror_rhs, _small_box

G = 5.0 / 3.0


def test_uniform_state_gives_exactly_zero_rhs():
    for v in [(0.0, 0.0, 0.0), (0.7, -0.4, 0.25), (-3.0, 2.0, 1.0)]:
        p = _filled(inputs.uniform_state(nsub=(2, 1, 1), v=v))
        d, amax, nb = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U, recon=1)
        assert nb == 0
        assert np.all(d == 0.0)
        c = math.sqrt(G * 0.9 / 1.3)
        assert np.allclose(amax, max(abs(x) for x in v) + c, rtol=1e-14)


def shear_flow(seed=5):
    """rho = 1, p = 1, v = (0, v_y(x), 0) with v_y a random multiple of 1/8
    per global x column, mass fractions (1/4, 1/4, 1/8, 1/8, 1/4): every
    conserved value and every recovered primitive is exact in binary."""
    p = inputs.periodic_box(nsub=2)
    E, N = 8, 16
    rng = np.random.default_rng(seed)
    vy = rng.integers(-8, 9, N) / 8.0
    X = [0.25, 0.25, 0.125, 0.125, 0.25]
    e_int = 1.0 / (G - 1.0)
    for s in range(p.n_sub):
        ox = (s % 2) * E
        blk = p.interior(s)
        v = np.broadcast_to(vy[ox:ox + E][None, None, :], (E, E, E))
        blk[0] = 1.0
        blk[1] = 0.0
        blk[2] = v
        blk[3] = 0.0
        blk[4] = e_int + 0.5 * v * v
        blk[5] = e_int ** (1.0 / G)
        for i in range(5):
            blk[6 + i] = X[i]
    return _filled(p)


def test_shear_flow_keeps_density_and_normal_momentum_exact():
    """In a pure shear flow (uniform rho and p, v_y varying across x) every
    point of the primitive reconstruction has p exactly uniform and v_x = 0,
    so the x-momentum flux through every x face is exactly p and the mass,
    x- and z-momentum, tau and species fluxes are the same on both faces of
    every cell: their dU/dt is exactly 0.  Reconstructing the conserved
    fields instead gives point pressures from PPM(E) - PPM(s_y)^2/(2 PPM(rho)),
    which vary, and a spurious d s_x/dt."""
    p = shear_flow()
    d, _, nb = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U, recon=1)
    assert nb == 0
    d = d.reshape(p.n_sub, p.nf, -1)
    for f in (0, 1, 3, 5, 6, 7, 8, 9, 10):
        assert not np.any(d[:, f]), f
    assert np.any(d[:, 2]) and np.any(d[:, 4])  # shear and energy diffuse
    dc, _, _ = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U, recon=0)
    assert np.max(np.abs(dc.reshape(p.n_sub, p.nf, -1)[:, 1])) > 1e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry_bitwise(axis):
    p = _small_box()
    d, amax, _ = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U, recon=1)
    q = _mirror(p, axis)
    dq, amq, _ = oracle.rhs(q.edge, q.off, q.dx, q.nf, q.U, recon=1)
    assert np.array_equal(dq, _mirror_rhs(p, d, axis))
    assert np.max(amq) == np.max(amax)


def test_total_conserved_on_periodic_box_after_one_rk3_step():
    p = _small_box(nsub=4)
    tot0 = [math.fsum(np.concatenate([p.interior(s)[f].ravel() for s in range(p.n_sub)])) for f in range(5)]
    mom_abs = [math.fsum(np.concatenate([np.abs(p.interior(s)[f]).ravel() for s in range(p.n_sub)]))
               for f in (1, 2, 3)]
    dt, fired, st = oracle.rk3_step(p.edge, p.off, p.dx, p.nf, p.U, bc=1, nbr=p.nbr, nthreads=8, recon=1)
    assert st == 0 and fired == 0 and dt > 0
    tot1 = [math.fsum(np.concatenate([p.interior(s)[f].ravel() for s in range(p.n_sub)])) for f in range(5)]
    assert abs(tot1[0] - tot0[0]) <= 1e-14 * abs(tot0[0])
    assert abs(tot1[4] - tot0[4]) <= 1e-14 * abs(tot0[4])
    for j, f in enumerate((1, 2, 3)):
        assert abs(tot1[f] - tot0[f]) <= 1e-14 * mom_abs[j]


def test_sod_l1_error_decreases_under_refinement():
    from tests.riemann_exact import density_profile
    errs = []
    for n in (64, 128, 256):
        p = inputs.sod_tube(n)
        oracle.ghost_fill(int(p.edge[0]), p.off, p.nf, p.nbr, p.U)
        t = 0.0
        while t < 0.2 * (1 - 1e-14):
            dt, fired, st = oracle.rk3_step(p.edge, p.off, p.dx, p.nf, p.U, bc=p.bc, nbr=p.nbr, gamma=p.gamma,
                                            dt_cap=0.2 - t, nthreads=8, recon=1)
            assert st == 0
            t += dt
        rho = np.concatenate([p.interior(s)[0, 0, 0, :] for s in range(p.n_sub)])
        x = (np.arange(n) + 0.5) / n
        exact = density_profile(x, 0.2, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G)
        errs.append(float(np.mean(np.abs(rho - exact))))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.01
