"""The ordering argument of the skewed-chunk smoothing schedule (k_skew), on
the CPU.  Launch d runs pass p on the rows
[1 + (d - p) H - p lag, 1 + (d - p + 1) H - p lag) of an m2-row level, clipped.
A visit of any smoother at row j reads rows j - 2 .. j + 1 and writes rows
j - 1 and j (plus the ghost row 0 from row 1 and m2 + 1 from row m2).  The
schedule is equivalent to running every pass over the whole level in order
if every (pass, row) runs exactly once and, for any two visits of different
passes where one writes a row the other reads, the earlier pass's visit runs
in an earlier launch and the later pass's in a later one.  This holds with
the lag of two rows the library uses and fails with one."""
import pytest

LAG = 2  # the library's SKEW_LAG


def schedule(m2, npass, H, lag):
    D = npass + (m2 - 1 + (npass - 1) * lag) // H
    when = {}
    for d in range(D):
        for p in range(npass):
            lo = max(1 + (d - p) * H - p * lag, 1)
            hi = min(1 + (d - p + 1) * H - p * lag, m2 + 1)
            for r in range(lo, hi):
                assert (p, r) not in when
                when[(p, r)] = d
    return when


def reads(r, m2):
    return set(range(r - 2, r + 2)) | ({0} if r == 1 else set()) | ({m2 + 1} if r == m2 else set())


def writes(r, m2):
    return {r - 1, r} | ({0} if r == 1 else set()) | ({m2 + 1} if r == m2 else set())


def violations(m2, npass, H, lag):
    when = schedule(m2, npass, H, lag)
    assert len(when) == npass * m2
    bad = 0
    for (p, r), d in when.items():
        rd = reads(r, m2)
        for p2 in range(npass):
            if p2 == p:
                continue
            for r2 in range(max(1, r - 3), min(m2, r + 3) + 1):
                if not writes(r2, m2) & rd:
                    continue
                d2 = when[(p2, r2)]
                if (p2 < p and d2 >= d) or (p2 > p and d2 <= d):
                    bad += 1
    return bad


@pytest.mark.parametrize("m2", [1, 2, 5, 17, 72, 130])
@pytest.mark.parametrize("npass", [1, 2, 7, 10, 20, 30])
@pytest.mark.parametrize("H", [1, 3, 8, 64, 1000])
def test_lag_two_orders_every_conflict(m2, npass, H):
    assert violations(m2, npass, H, LAG) == 0


@pytest.mark.parametrize("lag", [0, 1])
def test_a_shorter_lag_breaks_the_order(lag):
    assert violations(72, 10, 8, lag) > 0
