"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every function include/dgcurved.h declares, its own reference nodes equal
the oracle's, and calls fail with status codes rather than crashing."""
import os
import re

import numpy as np
import pytest

import __graft_entry__
from oracle.operators import ReferenceElement
from oracle.quadrature import default_q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding
    binding.load()
    return binding


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dgcurved.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(B):
    lib = B.load()
    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_abi(B):
    for n in declared_functions():
        assert callable(getattr(B, n)), n


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_reference_nodes_match_oracle(B, N):
    r, s = B.dg_reference_nodes(N)
    ref = ReferenceElement(N)
    assert np.abs(r - ref.r).max() < 1e-14
    assert np.abs(s - ref.s).max() < 1e-14
    Np, Nq, Ng, q = B.dg_sizes(N)
    assert (Np, Nq, Ng, q) == (ref.Np, ref.Nq, ref.Ng, default_q(N))


def test_errors_are_status_codes(B):
    with pytest.raises(B.DgError) as e:
        B.dg_reference_nodes(0)
    assert e.value.status == B.DG_EINVAL
    with pytest.raises(B.DgError):
        B.dg_sizes(9)
    # no GPU here, or a bad device index on a GPU machine: EINVAL, not a crash
    with pytest.raises(B.DgError) as e:
        B.dg_create(10_000)
    assert e.value.status == B.DG_EINVAL
    assert "device" in B.dg_last_error(None)
    lib = B.load()
    assert lib.dg_destroy(None) == 0
    assert lib.dg_sync(None, 0.0) == B.DG_EINVAL


def test_params_struct_layout(B):
    import ctypes
    # the C layout of include/dgcurved.h: u_inf[5] at 40, prec at 80, cub_q at 84
    assert ctypes.sizeof(B.dg_params) == 88
    assert B.dg_params.u_inf.offset == 40 and B.dg_params.prec.offset == 80 and B.dg_params.cub_q.offset == 84


def test_autotune_argument_errors(B):
    """The autotuner rejects a missing context or output before touching a GPU."""
    import ctypes
    lib = B.load()
    out = ctypes.c_int32(0)
    assert lib.dg_autotune(None, 1, 5, ctypes.byref(out), None, None, None) == B.DG_EINVAL
    assert lib.dg_set_tc_config(None, 1, 12, None, None) == B.DG_EINVAL


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_tet_reference_nodes_match_oracle(B, N):
    from oracle import tet
    r, s, t = B.dg_tet_reference_nodes(N)
    R = tet.warp_blend_nodes_3d(N)
    assert max(np.abs(r - R[0]).max(), np.abs(s - R[1]).max(), np.abs(t - R[2]).max()) < 1e-14
    q = default_q(N)
    assert B.dg_tet_sizes(N) == (tet.n_modes(N), q ** 3, q ** 2, tet.n_face_nodes(N))


def test_mesh_prepare_on_host_threads(B):
    """dg_mesh_prepare is the host half of dg_mesh_upload: it needs no
    context or GPU, runs on several threads at once, and reports bad input
    as status codes (here a non-reciprocal neighbour and an inverted
    element)."""
    import concurrent.futures as cf
    from paper_1208_4772_gb300.inputs import curving, meshes, states

    def prep(N):
        r, s = B.dg_reference_nodes(N)
        m = meshes.cylinder_channel(n_t=24, n_r=4, seed=1002)
        xy, _ = curving.curve_mesh(m, N, r, s)
        return B.dg_mesh_prepare(N, m.EToE, m.EToF, m.bc, xy, B.make_params(u_inf=states.freestream(0.38, 0.0)))

    with cf.ThreadPoolExecutor(4) as ex:
        handles = list(ex.map(prep, [2, 3, 4, 5, 6, 4]))
    assert all(h for h in handles)
    for h in handles:
        B.dg_prepared_free(h)
    N = 2
    r, s = B.dg_reference_nodes(N)
    m = meshes.periodic_square(4, seed=1000)
    xy = meshes.straight_nodes(m.verts, r, s)
    bad = m.EToE.copy()
    bad[0, 0] = (bad[0, 0] + 1) % m.K
    with pytest.raises(B.DgError) as e:
        B.dg_mesh_prepare(N, bad, m.EToF, m.bc, xy, B.make_params())
    assert e.value.status == B.DG_EINVAL and "connectivity" in str(e.value)
    flipped = xy.copy()
    flipped[3, :, 0] = 2 * flipped[3, 0, 0] - flipped[3, :, 0]    # mirrored: clockwise, J < 0
    with pytest.raises(B.DgError) as e:
        B.dg_mesh_prepare(N, m.EToE, m.EToF, m.bc, flipped, B.make_params())
    assert e.value.status == B.DG_EINVAL
