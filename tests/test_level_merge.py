"""The merged-level plan (csrc/level_merge.h, host C++) on the CPU: built and
evaluated by a small driver compiled with g++ against the header, for both
solve directions, groups of G = 1, 2, 4, 8 levels, against the oracle's
triangular solves; the structure (every M column in an earlier group, every
C column in the row's own group, C_ii = 1 / L_ii) is checked exactly."""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2305_16432_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2305_16432_gb300", "csrc")

DRIVER = r'''
#include <cstdio>
#include <vector>
#include "level_merge.h"
template <class T> static std::vector<T> rd(const char* dir, const char* name, size_t n) {
    std::vector<T> v(n);
    char path[4096];
    std::snprintf(path, sizeof(path), "%s/%s", dir, name);
    FILE* f = std::fopen(path, "rb");
    if (!f || std::fread(v.data(), sizeof(T), n, f) != n) { std::fprintf(stderr, "read %s\n", path); std::exit(2); }
    std::fclose(f);
    return v;
}
template <class T> static void wr(const char* dir, const char* name, const std::vector<T>& v) {
    char path[4096];
    std::snprintf(path, sizeof(path), "%s/%s", dir, name);
    FILE* f = std::fopen(path, "wb");
    std::fwrite(v.data(), sizeof(T), v.size(), f);
    std::fclose(f);
}
int main(int argc, char** argv) {
    const char* dir = argv[1];
    const long n = std::atol(argv[2]), nd = std::atol(argv[3]), nv = std::atol(argv[4]);
    const int G = std::atoi(argv[5]);
    auto dep_rp = rd<int64_t>(dir, "dep_rp", n + 1);
    auto dep_row = rd<int32_t>(dir, "dep_row", nd);
    auto dep_val = rd<int64_t>(dir, "dep_val", nd);
    auto diag = rd<int64_t>(dir, "diag", n);
    auto lev = rd<int32_t>(dir, "lev", n);
    auto Lv = rd<double>(dir, "Lv", nv);
    auto r = rd<double>(dir, "r", n);
    npcg::MergePlan p = npcg::build_merge_plan(n, dep_rp, dep_row, dep_val, diag, lev, G);
    std::vector<double> M, C, y(n, 0.0);
    npcg::eval_merge_plan(p, Lv.data(), M, C);
    npcg::solve_merge_plan(p, M, C, r.data(), y.data());
    wr(dir, "y", y);
    wr(dir, "grp", p.grp);
    wr(dir, "mrp", p.mrp);
    wr(dir, "mcol", p.mcol);
    wr(dir, "crp", p.crp);
    wr(dir, "ccol", p.ccol);
    wr(dir, "C", C);
    return 0;
}
'''


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("merge")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _direction(L, upper):
    """Dependencies of every row of L y = r (lower) or L^T z = y (upper):
    (row pointer, dependency rows, value index of the coefficient), the value
    index of the diagonal and the levels."""
    n, rp, ci = L.n, L.row_ptr, L.col_idx
    lev, _, levb, _ = O.levels(L)
    diag = np.array([rp[i + 1] - 1 for i in range(n)], np.int64)
    deps = [[] for _ in range(n)]
    for i in range(n):
        for k in range(rp[i], rp[i + 1] - 1):
            j = int(ci[k])
            if upper:
                deps[j].append((i, k))          # row j of L^T depends on row i > j through L_ij
            else:
                deps[i].append((j, k))
    for d in deps:
        d.sort()
    drp = np.zeros(n + 1, np.int64)
    drp[1:] = np.cumsum([len(d) for d in deps])
    drow = np.array([j for d in deps for j, _ in d], np.int32)
    dval = np.array([k for d in deps for _, k in d], np.int64)
    return drp, drow, dval, diag, (levb if upper else lev).astype(np.int32)


CASES = {
    "fem40": I.fem2d(40, sigma=1.0, seed=1),
    "heat36": I.heat2d(36, seed=2),
    "fd3d10": I.fd3d(10, 9, 8, sigma=1.5, corr_len=0.05, seed=3),
}


@pytest.mark.parametrize("G", [1, 2, 4, 8])
@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("name", list(CASES))
def test_merged_levels_reproduce_the_solve(driver, tmp_path, name, upper, G):
    A = O.assemble(CASES[name])
    L, _ = O.ic0(A)
    drp, drow, dval, diag, lev = _direction(L, upper)
    r = np.random.default_rng(4).standard_normal(A.n)
    for fname, arr in (("dep_rp", drp), ("dep_row", drow), ("dep_val", dval), ("diag", diag), ("lev", lev),
                       ("Lv", L.val.astype(np.float64)), ("r", r)):
        np.ascontiguousarray(arr).tofile(tmp_path / fname)
    subprocess.run([driver, str(tmp_path), str(A.n), str(len(drow)), str(L.nnz), str(G)], check=True)
    y = np.fromfile(tmp_path / "y", np.float64)
    yo = O.trsv_upper(L, r) if upper else O.trsv_lower(L, r)
    assert np.linalg.norm(y - yo) <= 1e-13 * np.linalg.norm(yo)
    # structure: M reads earlier groups only, C the row's own group, C_ii = 1 / L_ii
    grp = np.fromfile(tmp_path / "grp", np.int32)
    mrp, mcol = np.fromfile(tmp_path / "mrp", np.int64), np.fromfile(tmp_path / "mcol", np.int32)
    crp, ccol = np.fromfile(tmp_path / "crp", np.int64), np.fromfile(tmp_path / "ccol", np.int32)
    C = np.fromfile(tmp_path / "C", np.float64)
    assert np.array_equal(grp, lev // G)
    for i in range(A.n):
        mc, cc = mcol[mrp[i]:mrp[i + 1]], ccol[crp[i]:crp[i + 1]]
        assert np.all(grp[mc] < grp[i]) and np.all(grp[cc] == grp[i])
        assert np.all(np.diff(mc) > 0) and np.all(np.diff(cc) > 0)
        e = crp[i] + int(np.searchsorted(cc, i))
        assert ccol[e] == i and C[e] == 1.0 / L.val[diag[i]]
    if G == 1:
        # one level per group: M is the row's own dependencies over L_ii, C only the diagonal
        assert np.array_equal(np.diff(crp), np.ones(A.n, np.int64))
        assert np.array_equal(np.diff(mrp), np.diff(drp))
