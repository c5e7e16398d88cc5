"""Integer identities the kernels rely on, checked exhaustively on the host
(no GPU): they are properties of the arithmetic, not of the device."""
import numpy as np


def test_division_by_multiply_high_is_exact():
    """The kernels divide index q by a small divisor d (tile widths, plane and
    ghost-shell cell counts, 2 <= d < 2^12) as the high 32 bits of q * m with
    m = floor((2^32 - 1) / d) + 1 = ceil(2^32 / d).  Every q < 2^16 gives
    floor(q / d) exactly, for every such d."""
    q = np.arange(1 << 16, dtype=np.uint64)
    for d in range(2, 1 << 12):
        m = np.uint64((0xFFFFFFFF // d) + 1)
        assert m == -(-(1 << 32) // d)  # ceil(2^32 / d)
        got = (q * m) >> np.uint64(32)
        assert np.array_equal(got, q // np.uint64(d)), d


def test_ghost_shell_enumeration_covers_the_shell_once():
    """The ghost kernels enumerate a subgrid's 3-deep shell as two z slabs,
    two y slabs inside the interior z range and two x slabs inside the
    interior y and z ranges; the decode (restated here with the same
    divisions) visits every ghost cell of the (E+6)^3 block exactly once and
    no interior cell."""
    NG = 3
    for E in (8, 12, 16):
        B = E + 2 * NG
        nzs, nys, nxs = NG * B * B, NG * B * E, NG * E * E
        seen = set()
        for q in range(2 * nzs + 2 * nys + 2 * nxs):
            if q < 2 * nzs:
                side, r = divmod(q, nzs)
                a, b = r // B, r // B // B
                g = (r - a * B - NG, a - b * B - NG, b + (E if side else -NG))
            elif q < 2 * nzs + 2 * nys:
                side, r = divmod(q - 2 * nzs, nys)
                a = r // B
                g = (r - a * B - NG, a % NG + (E if side else -NG), a // NG)
            else:
                side, r = divmod(q - 2 * nzs - 2 * nys, nxs)
                a = r // NG
                b = a // E
                g = (r - a * NG + (E if side else -NG), a - b * E, b)
            assert all(-NG <= c < E + NG for c in g), g
            assert not all(0 <= c < E for c in g), g
            seen.add(g)
        assert len(seen) == B ** 3 - E ** 3
