"""The C ABI library builds, loads and exports every symbol include/qnsch.h
declares (no compute calls: this runs without a GPU); without a device,
qnsch_create reports QNSCH_ENODEV instead of falling back to the CPU."""
import ctypes
import os
import re

import pytest

from paper_1703_06606_gb300 import build as qbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "qnsch.h")).read()
    return sorted(set(re.findall(r"^int\s+(qnsch_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_paper_calls():
    names = declared_symbols()
    for must in ("qnsch_create", "qnsch_step", "qnsch_vcycle", "qnsch_mass", "qnsch_energy",
                 "qnsch_begin_step", "qnsch_commit_step", "qnsch_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(qbuild.build())
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_without_device_reports_enodev():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1703_06606_gb300 import qnsch
    with pytest.raises(qnsch.QnschError) as e:
        qnsch.Solver(16, 16)
    assert e.value.code == -2


def test_fma_probe_checks_arguments_then_device():
    """qnsch_fma_probe (libqnsch_probe.so) rejects out-of-range shapes with
    QNSCH_EINVAL before it touches the device, and reports QNSCH_ENODEV
    without one."""
    from paper_1703_06606_gb300 import probe, qnsch
    for bad in ((0, 16), (65, 16), (8, 0), (8, (1 << 24) + 1)):
        with pytest.raises(qnsch.QnschError) as e:
            probe.fma_probe(True, *bad)
        assert e.value.code == -1, bad
    import torch
    if torch.cuda.is_available():
        return
    with pytest.raises(qnsch.QnschError) as e:
        probe.fma_probe(True, 8, 16)
    assert e.value.code == -2


def test_fp64_issue_probe_checks_arguments_then_device():
    from paper_1703_06606_gb300 import probe, qnsch
    for bad in ((0, 32, 8, 16), (33, 32, 8, 16), (4, 0, 8, 16), (4, 33, 8, 16), (4, 32, 3, 16),
                (4, 32, 8, 0), (4, 32, 8, (1 << 20) + 1)):
        with pytest.raises(qnsch.QnschError) as e:
            probe.fp64_issue_probe(*bad)
        assert e.value.code == -1, bad
    import torch
    if torch.cuda.is_available():
        return
    with pytest.raises(qnsch.QnschError) as e:
        probe.fp64_issue_probe(4, 32, 8, 16)
    assert e.value.code == -2


def test_probes_are_not_in_the_solver_abi():
    """The probes are measurement tooling: libqnsch.so does not export them and
    include/qnsch.h does not declare them."""
    import ctypes
    from paper_1703_06606_gb300 import build, qnsch
    qnsch.lib()
    solver = ctypes.CDLL(build.LIB)
    for name in ("qnsch_fma_probe", "qnsch_fp64_issue_probe"):
        assert not hasattr(solver, name), name
    hdr = open(os.path.join(ROOT, "include", "qnsch.h")).read()
    assert "probe" not in hdr


def test_status_names_match_the_header():
    from paper_1703_06606_gb300 import qnsch
    text = open(os.path.join(ROOT, "include", "qnsch.h")).read()
    codes = {int(v): k for k, v in re.findall(r"#define QNSCH_(\w+) \((-?\d+)\)", text)}
    codes[0] = "OK"
    assert codes == qnsch.STATUS


def test_budget_refuses_creation_before_looking_for_a_device():
    """qnsch_create checks its arguments, then the budget, then the device."""
    from paper_1703_06606_gb300 import qnsch
    fp = qnsch.footprint(16, 16)
    try:
        qnsch.set_budget(fp - 1)
        assert qnsch.budget()[0] == fp - 1
        with pytest.raises(qnsch.QnschError) as e:
            qnsch.Solver(16, 16)
        assert e.value.code == -7
        with pytest.raises(qnsch.QnschError) as e:
            qnsch.Solver(16, 16, Re=-1.0)
        assert e.value.code == -1
        import torch
        if not torch.cuda.is_available():
            qnsch.set_budget(fp)
            with pytest.raises(qnsch.QnschError) as e:
                qnsch.Solver(16, 16)
            assert e.value.code == -2
    finally:
        qnsch.set_budget(0)
    assert qnsch.budget()[0] == 0


def test_create_rejects_nan_and_infinite_geometry_before_the_device():
    from paper_1703_06606_gb300 import qnsch
    for kw in (dict(Fr=float("nan")), dict(Lx=float("inf")), dict(Lx=float("nan")),
               dict(rho1=float("nan")), dict(Cn=0.0)):
        with pytest.raises(qnsch.QnschError) as e:
            qnsch.Solver(16, 16, **kw)
        assert e.value.code == -1, kw


C_PROGRAM = r"""
#include <stdio.h>
#include "qnsch.h"

typedef void (*any_fn)(void);
static const any_fn every_call[] = {
%s
};

int main(void) {
  qnsch_grid g = {256, 512, 1.0, 0, 0, 0};
  size_t fp = 0, b = 0, used = 0;
  qnsch_t* h = NULL;
  int rc_fp = qnsch_footprint(&g, 0, &fp);
  qnsch_set_budget(fp - 1);
  int rc_budget = qnsch_create(&g, 0.1, 1.0, 0.1, 1.0, 35.0, 10.0, 100.0, 0.01, 1.0, &h);
  qnsch_budget(&b, &used);
  qnsch_set_budget(0);
  int rc_create = qnsch_create(&g, 0.1, 1.0, 0.1, 1.0, 35.0, 10.0, 100.0, 0.01, 1.0, &h);
  if (rc_create == QNSCH_OK) qnsch_destroy(h);
  int ma = -1, mi = -1, pa = -1;
  qnsch_version(&ma, &mi, &pa);
  int same = ma == QNSCH_VERSION_MAJOR && mi == QNSCH_VERSION_MINOR && pa == QNSCH_VERSION_PATCH;
  printf("%%d %%zu %%d %%zu %%d %%d %%d\n", rc_fp, fp, rc_budget, b, rc_create,
         (int)(sizeof(every_call) / sizeof(every_call[0])), same);
  return 0;
}
"""


def test_header_is_plain_c_and_the_library_links_from_c(tmp_path):
    """A C99 program (-pedantic -Werror) takes the address of every declared
    call, links against libqnsch.so and runs the calls that need no device:
    qnsch_footprint, the budget, and qnsch_create's refusals."""
    import shutil
    import subprocess
    from paper_1703_06606_gb300 import qnsch
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    lib = qbuild.build()
    names = declared_symbols()
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM % ",\n".join("  (any_fn)%s" % n for n in names))
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True,
                         timeout=60).stdout.split()
    rc_fp, fp, rc_budget, b, rc_create, n, same_version = map(int, out)
    assert same_version == 1
    assert rc_fp == 0 and fp == qnsch.footprint(256, 512)
    assert rc_budget == -7 and b == fp - 1
    import torch
    assert rc_create == (0 if torch.cuda.is_available() else -2)
    assert n == len(names)


def test_binding_sets_argument_types_for_every_call():
    """Every call the header declares has its ctypes argument types set in the
    binding, so no Python value is passed by a guessed convention."""
    from paper_1703_06606_gb300 import qnsch
    L = qnsch.lib()
    missing = [n for n in declared_symbols() if getattr(L, n).argtypes is None]
    assert not missing, missing


def test_oracle_binding_sets_argument_types_for_every_call():
    from oracle import ref
    text = open(os.path.join(ROOT, "oracle", "qnsch_ref.h")).read()
    names = sorted(set(re.findall(r"^int\s+(qnsch_ref_\w+)\s*\(", text, flags=re.M)))
    L = ref.lib()
    assert names and not [n for n in names if getattr(L, n).argtypes is None]


def test_version_matches_the_header():
    from paper_1703_06606_gb300 import qnsch
    text = open(os.path.join(ROOT, "include", "qnsch.h")).read()
    want = tuple(int(re.search(r"#define QNSCH_VERSION_%s (\d+)" % k, text).group(1))
                 for k in ("MAJOR", "MINOR", "PATCH"))
    assert qnsch.version() == want
