"""Host ordering of the tile work list (csrc/rtlbfs_worklist.h), on the CPU.

spread_units reorders one cavity's part of the list so that its edge tiles
(those whose halo reaches past the mesh, which take the ghost-resolution
path) are spaced evenly among the interior ones.  The header is plain C++:
it is compiled here with g++ into a small driver that prints the reordered
unit ids.  Checked: the result is a permutation that leaves the units before
the range alone, each group keeps its order, consecutive edge units are
floor or ceil of n / ne apart, and with the 512 x 512 mesh's 592 tiles of
32 x 14 (102 on the edge) handed out round-robin to 152 SMs no SM gets two
edge tiles, where row-major order gives some SMs three.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_13449_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "rtlbfs_worklist.h"
struct Unit { int id; int edge; };
int main(int argc, char** argv)
{
    // argv[1]: start of the range; argv[2]: one '0'/'1' per unit (1: edge)
    const std::size_t b = (std::size_t)std::atoi(argv[1]);
    const char* f = argc > 2 ? argv[2] : "";
    std::vector<Unit> t;
    for (int k = 0; f[k]; ++k) t.push_back(Unit{k, f[k] == '1'});
    rtlbfs::spread_units(t, b, [](const Unit& u) { return u.edge != 0; });
    for (const Unit& u : t) std::printf("%d ", u.id);
    std::printf("\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    d = tmp_path_factory.mktemp("worklist")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def run(driver, b, flags):
    s = "".join("1" if x else "0" for x in flags)
    out = subprocess.run([driver, str(b), s] if s else [driver, str(b)], check=True,
                         capture_output=True, text=True).stdout.split()
    return [int(x) for x in out]


def check(order, b, flags):
    n_all = len(flags)
    assert sorted(order) == list(range(n_all))  # a permutation
    assert order[:b] == list(range(min(b, n_all)))  # the prefix is left alone
    rng = order[b:]
    edge = [u for u in rng if flags[u]]
    inner = [u for u in rng if not flags[u]]
    assert edge == sorted(edge) and inner == sorted(inner)  # each group keeps its order
    n, ne = len(rng), len(edge)
    if 0 < ne < n:
        pos = [k for k, u in enumerate(rng) if flags[u]]
        gaps = [q - p for p, q in zip(pos, pos[1:])]
        lo, hi = n // ne, -(-n // ne)
        assert all(lo <= g <= hi for g in gaps), (gaps, lo, hi)


def tiles_512():
    n, tx, th = 512, 32, 14
    tl = [(i * tx, j * th) for j in range(-(-n // th)) for i in range(n // tx)]
    return [not (i0 >= 2 and j0 >= 2 and i0 + tx + 2 <= n and j0 + th + 2 <= n) for i0, j0 in tl]


def test_cavity512_tiles_spread_over_the_sms(driver):
    flags = tiles_512()
    assert len(flags) == 592 and sum(flags) == 102
    order = run(driver, 0, flags)
    check(order, 0, flags)

    def max_edge_per_sm(o):
        c = {}
        for blk, u in enumerate(o):
            if flags[u]:
                c[blk % 152] = c.get(blk % 152, 0) + 1
        return max(c.values())

    assert max_edge_per_sm(list(range(592))) == 3  # row-major order
    assert max_edge_per_sm(order) == 1


@pytest.mark.parametrize("b,flags", [
    (0, [1, 1, 0, 0, 0, 0, 0, 0, 1, 1]),
    (3, [0, 1, 0, 1, 1, 1, 0, 0, 0, 0, 0, 1, 0]),
    (0, [0] * 7),            # no edge unit
    (0, [1] * 5),            # all edge units
    (2, [1, 0, 1]),          # one unit in the range
    (4, [0, 1, 0, 1]),       # empty range
    (0, []),                 # empty list
])
def test_spread_edge_cases(driver, b, flags):
    check(run(driver, b, flags), b, flags)


def test_random_lists(driver):
    import numpy as np
    rng = np.random.default_rng(7)
    for _ in range(40):
        n = int(rng.integers(1, 300))
        b = int(rng.integers(0, n + 1))
        flags = [bool(x) for x in rng.random(n) < rng.random()]
        check(run(driver, b, flags), b, flags)
