"""The locality order of the GEMM modes (hilbert_index3, the order the fibers are counting-sorted
on and the centroid columns are laid out in) is a Hilbert curve through the cells of its
grid (2^LOC_BITS per axis): a bijection onto [0, 2^(3 LOC_BITS)) along which consecutive cells
share a face. Compiled from the library's
own header with the host compiler; no GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_11494_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <cstdio>
#include "seg_common.cuh"
int main() {
    const unsigned side = 1u << seg::LOC_BITS;
    std::printf("%u\n", side);
    for (unsigned x = 0; x < side; ++x)
        for (unsigned y = 0; y < side; ++y)
            for (unsigned z = 0; z < side; ++z) std::printf("%u\n", seg::hilbert_index3(x, y, z));
    return 0;
}
"""


def cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


@pytest.fixture(scope="module")
def keys(tmp_path_factory):
    d = tmp_path_factory.mktemp("hilbert")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(PROGRAM)
    subprocess.run(["g++", "-std=c++17", "-O1", str(src), "-I", CSRC, "-I", INCLUDE, "-I",
                    cuda_include(), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    v = np.array(out.split(), dtype=np.int64)
    side, k = int(v[0]), v[1:]
    assert side >= 32 and k.shape == (side ** 3,)
    return side, k  # k[(x * side + y) * side + z]


def test_hilbert_index_is_a_bijection(keys):
    side, k = keys
    assert k.min() == 0 and k.max() == side ** 3 - 1
    assert len(np.unique(k)) == side ** 3


def test_consecutive_cells_share_a_face(keys):
    side, k = keys
    cells = np.stack(np.meshgrid(np.arange(side), np.arange(side), np.arange(side),
                                 indexing="ij"), -1).reshape(-1, 3)
    keys = k
    path = cells[np.argsort(keys)]
    steps = np.abs(np.diff(path, axis=0)).sum(1)
    assert (steps == 1).all()
    assert (path[0] == 0).all()  # the curve starts in the corner cell
