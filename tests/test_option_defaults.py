"""The option defaults documented in include/qnsch.h are the ones the library
sets (csrc/solver.cu) and the autotuner starts from."""
import os
import re

from paper_1703_06606_gb300 import autotune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# option key -> member of the handle that holds it
MEMBERS = {"fuse_cells": "fuse64", "fuse_cells32": "fuse32", "vanka_team_max": "team_max",
           "ch_team_max": "ch_team_max", "vanka_team_max32": "team_max32",
           "ch_team_max32": "ch_team_max32", "coupled": "coupled", "scheme": "scheme",
           "precision": "precision", "diverge_cycles": "diverge", "device_loop": "device_loop",
           "wave_cells32": "wave_cells", "wave_rows": "wave_rows", "wave_stall": "wave_stall",
           "vanka_team8_max": "team8_max", "vanka_pair_max": "pair_max", "vanka_split": "vsplit", "coarse_smem": "coarse_smem", "nu1": "nu1", "nu2": "nu2", "nu_coarse": "nuc",
           "skew_cells32": "skew_cells", "skew_rows": "skew_rows", "predictor": "predictor",
           "nu1_fine": "nu1f", "nu2_fine": "nu2f", "fuse_ctas": "fuse_ctas"}


def _header_defaults():
    txt = open(os.path.join(ROOT, "include", "qnsch.h")).read()
    block = txt[txt.index("Options (key: default)"):txt.index("Unknown keys give")]
    return {k: v for k, v in re.findall(r'"(\w+)":\s*([0-9.e^-]+)', block)}


def _solver_defaults():
    txt = open(os.path.join(ROOT, "paper_1703_06606_gb300", "csrc", "solver.cu")).read()
    out = {}
    for member in MEMBERS.values():
        m = re.search(r"\b%s\s*=\s*(-?[0-9]+)\s*[,;]" % member, txt)
        assert m, member
        out[member] = int(m.group(1))
    return out


def test_header_and_library_agree():
    hdr, lib = _header_defaults(), _solver_defaults()
    for key, member in MEMBERS.items():
        assert key in hdr, key
        assert int(float(hdr[key])) == lib[member], (key, hdr[key], lib[member])


def test_autotuner_starts_from_the_library_defaults():
    lib = _solver_defaults()
    for key, cands in autotune.CANDIDATES.items():
        assert cands[0] == lib[MEMBERS[key]], (key, cands[0], lib[MEMBERS[key]])
