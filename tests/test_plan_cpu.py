"""The batch's storage plan (paper_1809_04600_gb300/csrc/plan.h, host C++)
compiled with g++ and checked on cases whose answer follows from its rule:
systems by ascending pair count (ties by index), 12 bytes per stored nonzero;
all upper triangles when they fit, then both triangles while the rest of the
budget lasts; else upper triangles while they fit and the rest on the fly."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STORED, OTF, UPPER = 0, 1, 3

HARNESS = r'''
#include <cstdio>
#include "plan.h"
int main() {
    double budget; int n;
    if (std::scanf("%lf %d", &budget, &n) != 2) return 2;
    std::vector<int64_t> nnz(n);
    for (int s = 0; s < n; s++) { long long v; if (std::scanf("%lld", &v) != 1) return 2; nnz[s] = v; }
    for (int m : shci::storage_plan(nnz, budget)) std::printf("%d ", m);
    std::printf("\n");
    return 0;
}
'''


@pytest.fixture(scope="module")
def plan_exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("plan")
    src = d / "plan_main.cpp"
    src.write_text(HARNESS)
    exe = d / "plan_main"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1809_04600_gb300", "csrc"), str(src), "-o", str(exe)], check=True)
    return str(exe)


def plan(exe, nnz, budget):
    inp = "%r %d %s\n" % (float(budget), len(nnz), " ".join(str(int(v)) for v in nnz))
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    return [int(x) for x in out.split()]


@pytest.mark.parametrize("nnz,budget,want", [
    # all upper triangles fit (108 B); 48 B more upgrades the two smallest (12 + 36 B)
    ([5, 1, 3], 12 * 9 + 12 * 4, [UPPER, STORED, STORED]),
    # ... 47 B upgrades only the smallest
    ([5, 1, 3], 12 * 9 + 47, [UPPER, STORED, UPPER]),
    # exactly the upper triangles: no upgrade
    ([5, 1, 3], 12 * 9, [UPPER, UPPER, UPPER]),
    # equal counts: the lower index first
    ([2, 2, 2], 12 * 6 + 24, [STORED, UPPER, UPPER]),
    # the upper triangles do not all fit: smallest first while they fit, the rest on the fly
    ([5, 1, 3], 12 * 4, [OTF, UPPER, UPPER]),
    ([5, 1, 3], 12 * 4 - 1, [OTF, UPPER, OTF]),
    ([5, 1, 3], 11, [OTF, OTF, OTF]),
    # a system without pairs costs nothing
    ([0, 4], 0, [UPPER, OTF]),
    ([0, 0], 0, [STORED, STORED]),
    # room for everything
    ([7, 1, 9, 3], 1e18, [STORED, STORED, STORED, STORED]),
    # pair counts beyond 2^31 (bytes beyond 2^53 stay exact enough at this scale)
    ([3_000_000_000, 1_000_000_000], 12 * 4e9 + 12 * 1e9, [UPPER, STORED]),
])
def test_storage_plan_cases(plan_exe, nnz, budget, want):
    assert plan(plan_exe, nnz, budget) == want


def test_storage_plan_properties(plan_exe):
    """On seeded random batches: the stored bytes stay within the budget; when
    every upper triangle fits nothing is on the fly; the systems in both
    triangles are a prefix of the ascending order (no smaller system is left
    with less than a larger one); otherwise the upper-stored systems are a
    prefix and nothing is in both triangles."""
    import numpy as np
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = int(rng.integers(1, 20))
        nnz = [int(v) for v in rng.integers(0, 10_000, n)]
        budget = float(rng.uniform(0, 30 * sum(nnz) + 1))
        modes = plan(plan_exe, nnz, budget)
        used = sum(12 * v * (2 if m == STORED else 1 if m == UPPER else 0) for v, m in zip(nnz, modes))
        assert used <= budget + 1e-6
        order = sorted(range(n), key=lambda s: (nnz[s], s))
        ranked = [modes[s] for s in order]
        if 12 * sum(nnz) <= budget:
            assert OTF not in modes
            k = ranked.count(STORED)
            assert ranked[:k] == [STORED] * k
        else:
            assert STORED not in modes
            k = ranked.count(UPPER)
            assert ranked[:k] == [UPPER] * k
