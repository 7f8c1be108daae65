"""The order of a level's arrays in the device code's list (QN_LV_ARRAYS,
csrc/qnsch_dev.cuh) is the order in which the library lays them out in the
level's block (alloc_all, csrc/solver.cu).  The fused coarse V-cycle's
shared-memory copy depends on it: the launcher checks each level pointer by
pointer and falls back to global memory if they differ, so a mismatch would
not fail any result, only lose the copy silently."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1703_06606_gb300", "csrc")


def _macro_order():
    txt = open(os.path.join(CSRC, "qnsch_dev.cuh")).read()
    body = txt[txt.index("#define QN_LV_ARRAYS(X)"):]
    body = body[:body.index("\n\n")]
    return re.findall(r"X\((\w+)\)", body)


def _alloc_order():
    txt = open(os.path.join(CSRC, "solver.cu")).read()
    start = txt.index("double** f[NFIELD] = {")
    body = txt[start:txt.index("};", start)]
    return re.findall(r"&L\.(\w+)", body)


def test_device_array_list_matches_the_allocation_order():
    macro, alloc = _macro_order(), _alloc_order()
    assert len(macro) == 59
    assert macro == alloc


def test_copy_back_indices_name_the_arrays_meant():
    """The copy writes back arrays 0..QN_LV_WRITTEN-1 and QN_LV_RHOC by index;
    those indices name the unknowns, the sources, the residuals, the kept
    restricted iterate and rho(c) of the list."""
    macro = _macro_order()
    txt = open(os.path.join(CSRC, "kernels.cu")).read()
    written = int(re.search(r"QN_LV_WRITTEN = (\d+);", txt).group(1))
    rhoc = int(re.search(r"QN_LV_RHOC = (\d+);", txt).group(1))
    assert macro[:written] == ["c", "mu", "p", "u", "v", "fc", "fmu", "fp", "fu", "fv", "rc",
                               "rmu", "rp", "ru", "rv", "sc", "smu", "sp", "su", "sv"]
    assert macro[rhoc] == "rhoc"
