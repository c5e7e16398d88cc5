"""Pins of the oracle's floors and dual-energy re-synchronisation (readings
R6 and R7: after each RK stage rho >= rho_floor, rho_i >= 0, tau set to
e_int^(1/gamma) where e_int = E - |s|^2 / (2 rho) > eps2 E, then tau >= 0).

Every case is one interior cell of a single 8^3 subgrid with dyadic values,
so the expected result is a closed form; every other interior cell holds a
neutral state (rho = 1, s = 0, E = 16, gamma = 2: e_int = 16, tau = 4
exactly).  Each branch has a case that a plausible slip fails: pow(e, gamma)
for pow(e, 1/gamma), the re-sync threshold on the wrong side or not strict,
the floor applied after e_int is formed, -0 counted as negative, the tau
clamp applied before the re-sync, ghost cells touched."""
import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")

E = 8
NF = 8  # 2 species


def _batch(gamma=2.0):
    edge = np.array([E], np.int32)
    off, n = inputs.layout_offsets(edge, NF)
    U = np.full(n, 123.0)  # ghosts: a value no branch may produce
    blk = U[: NF * (E + 6) ** 3].reshape(NF, E + 6, E + 6, E + 6)
    inner = blk[:, 3:3 + E, 3:3 + E, 3:3 + E]
    inner[0] = 1.0
    inner[1:4] = 0.0
    inner[4] = 16.0
    inner[5] = 4.0 if gamma == 2.0 else 1.0
    inner[6] = 0.5
    inner[7] = 0.25
    return edge, off, U, blk, inner


def _set(inner, c, rho=None, s=None, Eg=None, tau=None, sp=None):
    z, y, x = c
    if rho is not None:
        inner[0, z, y, x] = rho
    if s is not None:
        inner[1:4, z, y, x] = s
    if Eg is not None:
        inner[4, z, y, x] = Eg
    if tau is not None:
        inner[5, z, y, x] = tau
    if sp is not None:
        inner[6:8, z, y, x] = sp


def test_neutral_state_is_a_fixed_point_and_ghosts_are_untouched():
    edge, off, U, blk, inner = _batch()
    before = U.copy()
    fired = oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=2.0 ** -40, eps2=0.25)
    assert fired == 0
    assert np.array_equal(U, before)  # tau = sqrt(16) = 4 exactly; ghosts (123) left alone


def test_density_floor_is_exact_and_counted_once():
    edge, off, U, blk, inner = _batch()
    _set(inner, (1, 2, 3), rho=2.0 ** -50)  # below the floor; s = 0, E = 16: e_int = 16
    _set(inner, (4, 4, 4), rho=-3.0)
    fired = oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=2.0 ** -40, eps2=0.25)
    assert fired == 2
    assert inner[0, 1, 2, 3] == 2.0 ** -40 and inner[0, 4, 4, 4] == 2.0 ** -40
    assert inner[5, 1, 2, 3] == 4.0  # re-synced from e_int = 16
    # a density equal to the floor is not raised and not counted
    edge, off, U, blk, inner = _batch()
    _set(inner, (0, 0, 0), rho=2.0 ** -40)
    assert oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=2.0 ** -40, eps2=0.25) == 0


def test_density_floor_comes_before_the_internal_energy():
    """rho = 2^-50 raised to 1/4; with s = (1, 0, 0), E = 6 the internal energy
    is 6 - 1/2 / (1/4) = 4 > E/4, so tau = 2.  Formed with the unfloored rho
    it would be hugely negative and tau would stay."""
    edge, off, U, blk, inner = _batch()
    _set(inner, (2, 5, 7), rho=2.0 ** -50, s=(1.0, 0.0, 0.0), Eg=6.0, tau=0.125)
    fired = oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=0.25, eps2=0.25)
    assert fired == 1
    assert inner[0, 2, 5, 7] == 0.25
    assert inner[5, 2, 5, 7] == 2.0


def test_species_floor():
    edge, off, U, blk, inner = _batch()
    _set(inner, (0, 1, 2), sp=(-2.0 ** -10, 2.0 ** -10))
    _set(inner, (3, 3, 3), sp=(-0.0, -5.0))
    fired = oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=2.0 ** -40, eps2=0.25)
    assert fired == 2  # -2^-10 and -5; -0 is not negative
    assert inner[6, 0, 1, 2] == 0.0 and inner[7, 0, 1, 2] == 2.0 ** -10
    assert inner[7, 3, 3, 3] == 0.0
    assert np.signbit(inner[6, 3, 3, 3])  # -0 kept as it is


def test_tau_resync_uses_one_over_gamma_and_the_kinetic_energy():
    """rho = 4, s = (4, 0, 0): |s|^2 / (2 rho) = 2; E = 18: e_int = 16,
    tau = 16^(1/2) = 4 (pow(16, gamma) would give 256)."""
    edge, off, U, blk, inner = _batch()
    _set(inner, (5, 6, 7), rho=4.0, s=(4.0, 0.0, 0.0), Eg=18.0, tau=0.5)
    _set(inner, (6, 6, 6), rho=0.5, s=(1.0, -1.0, 2.0), Eg=14.0, tau=0.5)  # 14 - 6/1 = 8: tau = sqrt(8)
    fired = oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=2.0 ** -40, eps2=0.25)
    assert fired == 0
    assert inner[5, 5, 6, 7] == 4.0
    assert inner[5, 6, 6, 6] == np.sqrt(8.0)


def test_tau_resync_gamma_five_thirds():
    """gamma = 5/3: e_int = 32 gives tau = 32^(3/5) = 8 (to the rounding of
    1/gamma and of pow); e_int = 2^-30 gives 2^-18."""
    edge, off, U, blk, inner = _batch(gamma=5.0 / 3.0)
    inner[4] = 32.0  # every cell: rho = 1, s = 0: e_int = 32
    _set(inner, (1, 1, 1), Eg=2.0 ** -30)
    fired = oracle.floors(edge, off, NF, U, gamma=5.0 / 3.0, rho_floor=2.0 ** -40, eps2=0.1)
    assert fired == 0
    tau = inner[5].copy()
    assert tau[1, 1, 1] == pytest.approx(2.0 ** -18, rel=4e-16)
    tau[1, 1, 1] = 8.0
    np.testing.assert_allclose(tau, 8.0, rtol=4e-16, atol=0)


def test_tau_resync_threshold_is_strict_and_on_the_right_side():
    """eps2 = 1/4.  rho = 2, s = (4, 4, 4): kinetic energy 12.
    E = 16: e_int = 4 = E/4, not above it: tau stays.
    E = 17: e_int = 5 > 17/4: tau = sqrt(5).
    E = 15: e_int = 3 < 15/4: tau stays."""
    edge, off, U, blk, inner = _batch()
    for c, Eg in (((0, 0, 1), 16.0), ((0, 0, 2), 17.0), ((0, 0, 3), 15.0)):
        _set(inner, c, rho=2.0, s=(4.0, 4.0, 4.0), Eg=Eg, tau=0.75)
    fired = oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=2.0 ** -40, eps2=0.25)
    assert fired == 0
    assert inner[5, 0, 0, 1] == 0.75
    assert inner[5, 0, 0, 2] == np.sqrt(5.0)
    assert inner[5, 0, 0, 3] == 0.75


def test_tau_clamp_after_the_resync():
    """A negative tau where the re-sync does not apply is clamped to 0 and
    counted; where it applies, tau comes from e_int and nothing fires."""
    edge, off, U, blk, inner = _batch()
    _set(inner, (7, 0, 0), rho=1.0, s=(4.0, 0.0, 0.0), Eg=8.5, tau=-0.5)  # e_int = 0.5 < 8.5/4
    _set(inner, (7, 0, 1), tau=-0.5)  # neutral e_int = 16: re-synced to 4
    fired = oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=2.0 ** -40, eps2=0.25)
    assert fired == 1
    assert inner[5, 7, 0, 0] == 0.0
    assert inner[5, 7, 0, 1] == 4.0


def test_every_branch_in_one_batch_counts_add_up():
    edge, off, U, blk, inner = _batch()
    _set(inner, (0, 0, 0), rho=-1.0)                                   # 1 firing
    _set(inner, (0, 0, 1), sp=(-1.0, -1.0))                            # 2
    _set(inner, (0, 0, 2), rho=1.0, s=(4.0, 0.0, 0.0), Eg=8.5, tau=-1.0)  # 1
    before = U.copy()
    fired = oracle.floors(edge, off, NF, U, gamma=2.0, rho_floor=2.0 ** -40, eps2=0.25)
    assert fired == 4
    changed = np.flatnonzero(U != before)
    assert changed.size == 4  # rho, two species, tau; the rest (ghosts included) unchanged
