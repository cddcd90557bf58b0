"""Host logic of the mixed-precision Eq. 20 lists, on the CPU: a small C++
driver (tests/host/joint_lists_check.cpp) compiled against the library's host
precompute reads every tet pair's joint list the way the GPU kernel does
(groups of four entries, weights in two planes per block of 32 entries) and
checks that the sums equal the sums over each tet's own neighbour list, that
pads carry zero weight at positions the list already holds, and that the real
entries are exactly the unions of the pairs' neighbour sets (Eq. 20's
neighbourhoods r < R_d).  Cases: 128-tet tiles with a ragged last tile and an
odd tet count (a lone last tet), and a radius wide enough for 64-tet tiles.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from workloads import jitter, kuhn_box

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_14870_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    out = str(tmp_path_factory.mktemp("jl") / "joint_lists_check")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if os.path.isdir(os.path.join(cuda, "include")):
        inc += ["-I", os.path.join(cuda, "include")]
    subprocess.run([cxx, "-O2", "-std=c++17", *inc, os.path.join(ROOT, "tests", "host", "joint_lists_check.cpp"),
                    "-o", out, "-lpthread"], check=True)
    return out


def run(checker, tmp_path, nodes, tets, radius):
    path = tmp_path / "mesh.bin"
    with open(path, "wb") as f:
        np.array([len(nodes), len(tets)], np.int64).tofile(f)
        np.array([radius], np.float64).tofile(f)
        np.ascontiguousarray(nodes, np.float64).tofile(f)
        np.ascontiguousarray(tets, np.int32).tofile(f)
    r = subprocess.run([checker, str(path)], capture_output=True, text=True)
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert r.returncode == 0, out
    return out


def test_joint_lists_read_as_the_kernel_reads_them(checker, tmp_path):
    nodes, tets, _ = kuhn_box(6, 5, 7)
    nodes = jitter(nodes, 0.02, 1.0, 5)
    tets = tets[:-1]                       # odd count: the last pair holds one tet
    out = run(checker, tmp_path, nodes, tets, 1.5)
    assert out["tile"] == 128 and out["tets"] % 128 != 0
    assert out["bad"] == 0 and out["worst_rel"] <= 1e-12
    assert out["real"] == out["union_sizes"] and out["entries"] == out["real"] + out["pads"]
    assert out["entries"] % 4 == 0 and out["pads"] <= 3 * ((out["tets"] + 1) // 2)
    assert out["distinct_chunks"] >= 0.8 * out["chunks"]


def test_wide_radius_takes_64_tet_tiles(checker, tmp_path):
    nodes, tets, _ = kuhn_box(8, 8, 12)
    nodes = jitter(nodes, 0.02, 1.0, 9)
    out = run(checker, tmp_path, nodes, tets, 3.0)
    assert out["tile"] == 64
    assert out["bad"] == 0 and out["worst_rel"] <= 1e-12 and out["real"] == out["union_sizes"]
