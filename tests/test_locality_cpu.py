"""The locality order of the GEMM modes (hilbert_index3, the order the fibers are counting-sorted
on and the centroid columns are laid out in) is a Hilbert curve through the 64^3 cells: a
bijection onto [0, 2^18) along which consecutive cells share a face. Compiled from the library's
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
    for (unsigned x = 0; x < 64; ++x)
        for (unsigned y = 0; y < 64; ++y)
            for (unsigned z = 0; z < 64; ++z) std::printf("%u\n", seg::hilbert_index3(x, y, z));
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
    k = np.array(out.split(), dtype=np.int64)
    assert k.shape == (64 ** 3,)
    return k  # k[(x * 64 + y) * 64 + z]


def test_hilbert_index_is_a_bijection(keys):
    assert keys.min() == 0 and keys.max() == 64 ** 3 - 1
    assert len(np.unique(keys)) == 64 ** 3


def test_consecutive_cells_share_a_face(keys):
    cells = np.stack(np.meshgrid(np.arange(64), np.arange(64), np.arange(64), indexing="ij"),
                     -1).reshape(-1, 3)
    path = cells[np.argsort(keys)]
    steps = np.abs(np.diff(path, axis=0)).sum(1)
    assert (steps == 1).all()
    assert (path[0] == 0).all()  # the curve starts in the corner cell
