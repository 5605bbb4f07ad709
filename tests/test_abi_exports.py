"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/npcg.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "npcg.h")).read()
    return sorted(set(re.findall(r"NPCG_API\s+(?:npcg_status|const char\*)\s+(npcg_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2305_16432_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("npcg_assemble_system", "npcg_gnn_factor", "npcg_pcg_solve", "npcg_pcg_solve_batched",
                     "npcg_loss_and_grad", "npcg_ic0_factor", "npcg_create", "npcg_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (npcg_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_answers_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.npcg_status_string.restype = ctypes.c_char_p
    assert lib.npcg_status_string(0) == b"NPCG_OK"
    assert lib.npcg_status_string(7) == b"NPCG_ETIMEOUT"
    # argument validation happens before any CUDA call
    assert lib.npcg_destroy(None) == 1
    assert lib.npcg_pattern_free(None) == 1


def test_nparams_matches_layout(libpath):
    from paper_2305_16432_gb300 import inputs as I
    from paper_2305_16432_gb300 import npcg
    for cfg in (I.GnnConfig(2, 2, 2, 16), I.GnnConfig(6, 2, 2, 64), I.GnnConfig(3, 1, 3, 32)):
        assert npcg.gnn_nparams(cfg) == cfg.nparams


def test_builds_only_for_sm103a():
    from paper_2305_16432_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes mirrors of the ABI structs have the C layout: size and the
    # offset of every field, from a host C program compiled against the header
    from paper_2305_16432_gb300 import npcg as N
    mirrors = {"npcg_problem": N._Problem, "npcg_pattern_info": N._Info, "npcg_gnn_config": N._Cfg,
               "npcg_solve_stats": N._Stats, "npcg_solve_opts": N._Opts}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "npcg.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
