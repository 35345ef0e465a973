"""Values the paper prints, kept as fixtures under tests/golden/ with their
citations: the number of basis functions N_p = (p+d)!/(d! p!) (Sec. 2) and
the 35 collocation nodes of a p = 4 tetrahedron (Sec. 5, Table 2
discussion), against the oracle's node sets and basis and the library's
host-side sizes."""
import json
import os
from math import factorial

import numpy as np
import pytest

import __graft_entry__
from oracle import basis, tet
from oracle.nodes import warp_blend_nodes

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "paper_sizes.json")))


@pytest.fixture(scope="module")
def B():
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding
    binding.load()
    return binding


def test_np_formula_and_node_sets():
    f = G["np_formula"]
    for d, p, n in zip(f["d"], f["p"], f["np"]):
        assert factorial(p + d) // (factorial(d) * factorial(p)) == n
        if d == 2:
            assert basis.n_modes(p) == n and len(warp_blend_nodes(p)[0]) == n
            assert basis.vandermonde(p, *warp_blend_nodes(p)).shape == (n, n)
        else:
            assert tet.n_modes(p) == n and len(tet.warp_blend_nodes_3d(p)[0]) == n
            assert tet.vandermonde(p, *tet.warp_blend_nodes_3d(p)).shape == (n, n)


def test_sphere_finest_level_nodes(B):
    s = G["sphere_finest_level"]
    assert s["d"] == 3
    r, _, _ = B.dg_tet_reference_nodes(s["p"])
    assert len(r) == s["collocation_nodes"] == B.dg_tet_sizes(s["p"])[0]
    ref = tet.ReferenceTet(s["p"])
    assert ref.Np == s["collocation_nodes"]
    assert np.linalg.matrix_rank(ref.V) == s["collocation_nodes"]
