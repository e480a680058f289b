"""z-chunk lists of the fused kernels (csrc/chunks.h, host-only C++): every
list covers the column exactly once in increasing order; uniform lists are
chunks of the given depth; tapered lists keep that depth until at most two
chunks' worth remains and then shrink monotonically.  CPU only."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "chunks.h"
int main(int argc, char** argv) {
  const auto b = nlc::chunk_bounds(std::atoi(argv[1]), std::atoi(argv[2]), std::atoi(argv[3]) != 0);
  for (size_t i = 0; i < b.size(); i++) std::printf("%d ", b[i]);
  std::printf("\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def bounds(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("chunks")
    (d / "drv.cpp").write_text(DRIVER)
    exe = d / "drv"
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-I",
                           os.path.join(ROOT, "paper_1907_13415_gb300", "csrc"),
                           str(d / "drv.cpp"), "-o", str(exe)])

    def run(nz, tz, taper):
        out = subprocess.check_output([str(exe), str(nz), str(tz), str(int(taper))])
        return [int(v) for v in out.split()]
    return run


@pytest.mark.parametrize("nz", [1, 2, 3, 7, 8, 9, 23, 64, 100, 256, 257, 1000])
@pytest.mark.parametrize("tz", [0, 1, 4, 6, 16, 24, 48, 64, 128, 300])
def test_lists_cover_the_column_once(bounds, nz, tz):
    for taper in (False, True):
        b = bounds(nz, tz, taper)
        assert b[0] == 0 and b[-1] == nz
        sizes = [b[i + 1] - b[i] for i in range(len(b) - 1)]
        assert all(s > 0 for s in sizes), (nz, tz, taper, b)


@pytest.mark.parametrize("nz,tz", [(256, 24), (256, 48), (100, 7), (23, 4)])
def test_uniform_lists_are_chunks_of_the_depth(bounds, nz, tz):
    b = bounds(nz, tz, False)
    sizes = [b[i + 1] - b[i] for i in range(len(b) - 1)]
    assert all(s == tz for s in sizes[:-1]) and 0 < sizes[-1] <= tz


@pytest.mark.parametrize("nz,tz", [(256, 16), (256, 32), (256, 48), (256, 128),
                                   (1000, 24), (64, 8), (23, 4)])
def test_tapered_lists_shrink_at_the_end(bounds, nz, tz):
    b = bounds(nz, tz, True)
    sizes = [b[i + 1] - b[i] for i in range(len(b) - 1)]
    head = [s for s in sizes if s == tz]
    tail = sizes[len(head):]
    assert sizes[:len(head)] == head          # full chunks first
    assert sum(tail) <= 2 * tz                 # then at most two chunks' worth
    assert all(tail[i] >= tail[i + 1] for i in range(len(tail) - 2))
    assert min(sizes) >= min(4, nz)
    # the example the documentation gives: 256 planes at depth 48
    if (nz, tz) == (256, 48):
        assert sizes == [48, 48, 48, 48, 32, 16, 8, 8]
