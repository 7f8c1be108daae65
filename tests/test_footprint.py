"""qnsch_footprint (host logic, no device) against the layout include/qnsch.h
and the design notes describe, recomputed here: per level one FP64 block of 59
arrays over the padded index space (row pitch m1 + 3 rounded up to 32
elements, m2 + 3 rows), one more block of 43 arrays per level for the error
equation (FP32 at precision 1, FP64 at precision 2), the committed state (5
arrays of the finest level's size), the two earlier states the predictor
extrapolates from (10 more), the reduction partials (10 doubles per
32 x 8 tile of the (m1 + 1) x (m2 + 1) points), a host-I/O staging array of
(m1 + 1)(m2 + 1) doubles, 128 scalars (norms, reductions and the
control block of the device-side outer-cycle loop) and the banded wavefront's
counters (a ticket and one count per band of 4 rows of the finest level,
4 bytes each, rounded up to 256 bytes)."""
import pytest

from paper_1703_06606_gb300 import qnsch


def _levels(m1, m2, px):
    n = 1
    while m1 % 2 == 0 and m2 % 2 == 0 and m2 // 2 >= 2 and (
            m1 // 2 >= 4 and (m1 // 2) % 2 == 0 if px else m1 // 2 >= 2):
        m1, m2, n = m1 // 2, m2 // 2, n + 1
    return n


def _bytes(m1, m2, px, levels, precision):
    lev = levels or _levels(m1, m2, px)
    total, a, b = 0, m1, m2
    for l in range(lev):
        n = -(-(a + 3) // 32) * 32 * (b + 3)
        if l == 0:
            n0 = n
        total += 59 * 8 * n + (43 * (4 if precision == 1 else 8) * n if precision else 0)
        a, b = a // 2, b // 2
    total += 5 * 8 * n0 + 10 * 8 * n0
    total += -(-(m1 + 1) // 32) * -(-(m2 + 1) // 8) * 10 * 8
    total += (m1 + 1) * (m2 + 1) * 8 + 128 * 8
    total += -(-(4 * (2 + -(-m2 // 4))) // 256) * 256
    return total


@pytest.mark.parametrize("m1,m2,px,levels", [(256, 512, False, 0), (1024, 4096, True, 0),
                                             (64, 64, True, 0), (37, 29, False, 0),
                                             (40, 24, True, 2), (2, 2, False, 0),
                                             (512, 512, False, 3)])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_footprint_matches_the_layout(m1, m2, px, levels, precision):
    assert qnsch.footprint(m1, m2, px, levels, precision) == _bytes(m1, m2, px, levels, precision)


def test_footprint_of_the_bench_workloads():
    """The sizes quoted for the droplet and Rayleigh-Taylor workloads."""
    mb = [qnsch.footprint(256, 512, False, 0, p) / 1e6 for p in (0, 1, 2)]
    gb = [qnsch.footprint(1024, 4096, True, 0, p) / 1e9 for p in (0, 1, 2)]
    assert [round(x, 1) for x in mb] == [117.5, 153.5, 189.4]
    assert [round(x, 2) for x in gb] == [3.32, 4.33, 5.34]


def test_footprint_rejects_what_create_rejects():
    for args in ((1, 8, False, 0, 0), (8, 8, False, 0, 3), (7, 8, True, 0, 0), (2, 8, True, 0, 0),
                 (64, 64, False, 9, 0)):
        with pytest.raises(qnsch.QnschError) as e:
            qnsch.footprint(*args)
        assert e.value.code == -1, args


def test_grids_beyond_32_bit_indexing_are_rejected():
    """(m1 + 3 rounded up to 32) x (m2 + 3) must fit a 32-bit index: 46304^2
    gives 46304 x 46307 < 2^31 - 1, 46336 x 46336 does not.  Rejected by
    qnsch_footprint and, before any device is looked for, by qnsch_create."""
    assert qnsch.footprint(46304, 46304) > 0
    for m1, m2 in ((46336, 46336), (1 << 29, 8), (8, 1 << 29)):
        with pytest.raises(qnsch.QnschError) as e:
            qnsch.footprint(m1, m2)
        assert e.value.code == -1
    with pytest.raises(qnsch.QnschError) as e:
        qnsch.Solver(46336, 46336)
    assert e.value.code == -1
