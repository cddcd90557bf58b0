"""C ABI checks that need no GPU: the library builds, exports every entry point
declared in include/*.h with the struct layouts the binding assumes, and its
host precompute (gf_mesh_plan) agrees with the oracle's mesh graph."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2103_14870_gb300 as gf
from paper_2103_14870_gb300 import graphfem as gb
from oracle import mesh as omesh
from workloads import beam_config, bcc_ellipsoid, jitter, two_tet_fig4

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(gf_[a-z0-9_]+)\s*\(", txt))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_symbol_is_exported():
    lib = gf.load_library()
    names = declared_functions()
    assert "gf_step" in names and "gf_mesh_create" in names and len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "graphfem.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(gf_material), sizeof(gf_options), sizeof(gf_step_stats),'
                   ' sizeof(gf_mesh_info), offsetof(gf_options, stream), offsetof(gf_step_stats, rel_res));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(gb.Material), ctypes.sizeof(gb.Options), ctypes.sizeof(gb.StepStats),
            ctypes.sizeof(gb.MeshInfo), gb.Options.stream.offset, gb.StepStats.rel_res.offset]
    assert got == want


@pytest.mark.parametrize("radius", [0.0, 1.5])
def test_plan_matches_oracle_graph(radius):
    w = beam_config()
    mat = gf.material(w.young, w.poisson, w.density, w.threshold, radius)
    plan = gf.mesh_plan(w.nodes, w.tets, mat)
    edges, tet_edges = omesh.edges_of(w.tets)
    np.testing.assert_array_equal(plan["edges"], edges)
    assert plan["n_blocks"] == w.n_nodes + 2 * len(edges)
    nb = omesh.nonlocal_neighbours(w.nodes, w.tets, radius)
    np.testing.assert_array_equal(plan["nbr_count"], [len(x) for x in nb])
    assert plan["n_nbr_pairs"] == sum(len(x) for x in nb)


def test_colouring_is_conflict_free():
    nodes, tets = bcc_ellipsoid(6.0, 4.0, 3.0)
    nodes = jitter(nodes, 0.01, 1.0, 3)
    plan = gf.mesh_plan(nodes, tets, gf.material(1e5, 0.3, 1000.0))
    col = plan["colour"]
    assert col.min() == 0 and col.max() == plan["n_colours"] - 1
    for c in range(plan["n_colours"]):
        members = tets[col == c].ravel()
        assert len(np.unique(members)) == len(members), c


def test_plan_rejects_bad_meshes():
    nodes, tets = two_tet_fig4()
    mat = gf.material(1e6, 0.3, 1000.0)
    flat = nodes.copy()
    flat[3] = [0.5, 0.5, 0.0]          # A, B, C, D coplanar
    with pytest.raises(gf.GraphFEMError) as e:
        gf.mesh_plan(flat, tets, mat)
    assert e.value.status == 1 and "degenerate" in str(e.value)
    bad = tets.copy()
    bad[1, 2] = 99
    with pytest.raises(gf.GraphFEMError):
        gf.mesh_plan(nodes, bad, mat)
    with pytest.raises(gf.GraphFEMError):
        gf.mesh_plan(nodes, tets, gf.material(1e6, 0.6, 1000.0))
