"""Accuracy of the FP64 arithmetic helpers the kernels use in place of
division, square root and pow (FP64 arithmetic on this GPU issues at about
1/64 of the FP32 rate, so these start from FP32 hardware estimates and refine
them by Newton-Raphson / Heron steps in FP64):

  rcp_nr        1/x: rcp.approx estimate + two Newton-Raphson steps
  sqrt_nr       sqrt(q): rsqrt.approx estimate + two Heron corrections
  eint_of_tau   tau^gamma (gamma = 5/3): exponent split + lg2/ex2 estimate of
                m^(5/3) + two Newton steps on y^3 = m^5
  tau_of_eint   e^(1/gamma) (gamma = 5/3): exponent split + lg2/ex2 estimate of
                m^(3/5) + two chord-Newton steps on y^5 = m^3

Each is swept over the whole exponent range (random mantissas at every
binary exponent, both signs where defined, zeros, subnormals, infinities,
NaN) through oct_hydro_eval_math, and compared with the correctly rounded
result: numpy's division and sqrt (IEEE correctly rounded), and for the
powers the exact exponents 5/3 and 3/5 evaluated in the host's long double
(x87 extended or IEEE quad) and rounded once to double -- the helpers compute
the power of the exact fraction, where pow(x, gamma) takes gamma rounded to
double (the two differ by |ln x| * 7e-17 relative).  CUDA's own 1.0 / x,
sqrt and pow are evaluated on the device beside them.  Bounds: rcp_nr and
sqrt_nr within 1 ulp, tau^gamma and e^(1/gamma) within 2 ulp; outside their
fast ranges the helpers call CUDA's own functions and must equal them
bitwise."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

G53 = 5.0 / 3.0


def _ulp_diff(a, b):
    """|a - b| in units in the last place (same-sign finite values)."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def _sweep(lo, hi, per=24, seed=0, signs=(1.0,)):
    rng = np.random.default_rng(seed)
    e = np.repeat(np.arange(lo, hi + 1), per)
    m = 1.0 + rng.random(e.size)
    x = np.ldexp(m, e)
    out = [s * x for s in signs]
    return np.concatenate(out)


def _eval(which, x, gamma=G53):
    import torch
    from paper_2210_06439_gb300 import binding
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = torch.empty_like(xd)
    binding.eval_math(which, xd, yd, gamma=gamma)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _same_or_both_nan(a, b):
    return np.all((a.view(np.int64) == b.view(np.int64)) | (np.isnan(a) & np.isnan(b)))


def test_reciprocal_within_one_ulp_over_all_exponents():
    x = _sweep(-1022, 1023, signs=(1.0, -1.0))
    with np.errstate(over="ignore", divide="ignore"):
        ref = 1.0 / x
    got = _eval(0, x)
    cuda = _eval(16, x)
    assert _same_or_both_nan(cuda, ref)  # CUDA's division is correctly rounded
    fin = np.isfinite(ref) & (ref != 0) & (np.abs(ref) >= np.finfo(np.float64).tiny)
    u = _ulp_diff(got[fin], ref[fin])
    print(f"\nrcp_nr: max {u.max():.0f} ulp, {np.mean(u > 0):.2%} not correctly rounded")
    assert u.max() <= 1
    # results in the subnormal range, zeros, infinities, NaN: CUDA's division exactly
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.0 ** 1023 * 1.9, 2.0 ** -1074 * 7])
    with np.errstate(over="ignore", divide="ignore"):
        assert _same_or_both_nan(_eval(0, special), _eval(16, special))
    rest = ~fin
    assert _same_or_both_nan(got[rest], ref[rest])


def test_square_root_within_one_ulp_over_all_exponents():
    x = np.concatenate([_sweep(-1022, 1023), np.ldexp(1.0 + np.arange(64) / 64.0, -1060)])
    ref = np.sqrt(x)
    got = _eval(1, x)
    assert _same_or_both_nan(_eval(17, x), ref)  # CUDA's sqrt is correctly rounded
    u = _ulp_diff(got, ref)
    print(f"\nsqrt_nr: max {u.max():.0f} ulp, {np.mean(u > 0):.2%} not correctly rounded")
    assert u.max() <= 1
    special = np.array([0.0, -0.0, np.inf, np.nan, 5e-324, -1.0, -np.inf])
    with np.errstate(invalid="ignore"):
        assert _same_or_both_nan(_eval(1, special), _eval(17, special))


def _exact_power(x, num, den):
    """x^(num/den) with the exponent formed and the power taken in long
    double, rounded once to double."""
    xl = x.astype(np.longdouble)
    with np.errstate(over="ignore", under="ignore"):
        return np.power(xl, np.longdouble(num) / np.longdouble(den)).astype(np.float64)


def test_tau_to_the_gamma_within_two_ulp():
    """The fast path covers tau in [2^-600, 2^601); outside it, and for tau
    <= 0, infinities and NaN, the helper calls pow and must equal it."""
    x = _sweep(-600, 600, per=40)
    ref = _exact_power(x, 5, 3)
    got = _eval(2, x)
    cuda = _eval(18, x)
    u = _ulp_diff(got, ref)
    uc = _ulp_diff(cuda, ref)
    print(f"\ntau^gamma: max {u.max():.0f} ulp from the exact power (CUDA pow(x, gamma): {uc.max():.0f} ulp)")
    assert u.max() <= 2
    outside = np.concatenate([_sweep(-1022, -601, per=4), _sweep(601, 1023, per=4),
                              np.array([0.0, -0.0, -1.5, np.inf, np.nan, 5e-324])])
    assert _same_or_both_nan(_eval(2, outside), _eval(18, outside))
    # another gamma takes pow everywhere
    assert _same_or_both_nan(_eval(2, x[::7], gamma=1.4), _eval(18, x[::7], gamma=1.4))


def test_internal_energy_to_tau_within_two_ulp():
    """The fast path covers every positive normal e; zero, subnormals,
    negative values, infinities and NaN take pow and must equal it."""
    x = _sweep(-1022, 1023, per=24)
    ref = _exact_power(x, 3, 5)
    got = _eval(3, x)
    cuda = _eval(19, x)
    u = _ulp_diff(got, ref)
    uc = _ulp_diff(cuda, ref)
    print(f"\ne^(1/gamma): max {u.max():.0f} ulp from the exact power (CUDA pow(x, 1/gamma): {uc.max():.0f} ulp)")
    assert u.max() <= 2
    outside = np.array([0.0, -0.0, -2.5, np.inf, -np.inf, np.nan, 5e-324, 2.0 ** -1040])
    with np.errstate(invalid="ignore"):
        assert _same_or_both_nan(_eval(3, outside), _eval(19, outside))
    assert _same_or_both_nan(_eval(3, x[::7], gamma=1.4), _eval(19, x[::7], gamma=1.4))
