"""Host state I/O: the staged path (host threads and one copy) and the
device path (a kernel on the caller's FP64 rows through coherent access to
pageable host memory) move the same values.

Bars:
  * set then get returns the input rounded to the mesh precision (FP32
    meshes: float32(U); DG_FP64_DEBUG: U itself), bit for bit, in either
    mode and across modes (set in one, get in the other);
  * dg_eval_rhs returns the same right-hand side bit for bit in both modes
    (the device work is the same; only the transfer differs).
The device mode is exercised where the device offers it; the staged mode
and the argument checks everywhere.
"""
import numpy as np
import pytest

import __graft_entry__
from cases import make_case, make_case3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def modes(B, ctx):
    out = ["staged"]
    try:
        B.dg_set_host_io(ctx, "device")
        out.append("device")
    except B.DgError:
        pass
    B.dg_set_host_io(ctx, "auto")
    return out


def tri_mesh(B, ctx, prec):
    r, s = B.dg_reference_nodes(4)
    case = make_case("cyl", 4, r, s, seed=5)   # curved walls: a non-trivial device order
    m = case["mesh"]
    p = B.make_params(u_inf=case["u_inf"], prec=prec)
    h = B.dg_mesh_upload(ctx, 4, m.EToE, m.EToF, m.bc, case["xy"], p)
    return case, h


@pytest.mark.parametrize("prec", ["fp32", "tf32", "fp64"])
def test_state_round_trip_in_every_mode(B, ctx, prec):
    case, h = tri_mesh(B, ctx, prec)
    U = case["U"]
    want = U if prec == "fp64" else U.astype(np.float32).astype(np.float64)
    ms = modes(B, ctx)
    try:
        for m_in in ms:
            for m_out in ms:
                B.dg_set_host_io(ctx, m_in)
                B.dg_set_state(ctx, h, U)
                B.dg_set_host_io(ctx, m_out)
                got = B.dg_get_state(ctx, h)
                assert np.array_equal(got, want), (m_in, m_out)
    finally:
        B.dg_set_host_io(ctx, "auto")
        B.dg_mesh_free(ctx, h)


def test_rhs_identical_in_every_mode(B, ctx):
    case, h = tri_mesh(B, ctx, "tf32")
    try:
        out = {}
        for mode in modes(B, ctx):
            B.dg_set_host_io(ctx, mode)
            B.dg_set_state(ctx, h, case["U"])
            out[mode] = B.dg_eval_rhs(ctx, h)
        ref = out["staged"]
        assert np.all(np.isfinite(ref))
        for mode, L in out.items():
            assert np.array_equal(L, ref), mode
    finally:
        B.dg_set_host_io(ctx, "auto")
        B.dg_mesh_free(ctx, h)


def test_tet_state_round_trip_in_every_mode(B, ctx):
    r, s, t = B.dg_tet_reference_nodes(2)
    case = make_case3("bump", 2, r, s, t, size="tiny")
    m = case["mesh"]
    h = B.dg_tet_mesh_upload(ctx, 2, m.EToV, m.bc, case["xyz"], B.make_params(u_inf=case["u_inf"], prec="fp32"))
    U = case["U"]
    want = U.astype(np.float32).astype(np.float64)
    try:
        for mode in modes(B, ctx):
            B.dg_set_host_io(ctx, mode)
            B.dg_set_state(ctx, h, U)
            assert np.array_equal(B.dg_get_state(ctx, h), want), mode
    finally:
        B.dg_set_host_io(ctx, "auto")
        B.dg_mesh_free(ctx, h)


def test_host_io_mode_arguments(B, ctx):
    auto = B.dg_host_io(ctx)
    assert auto in ("staged", "device")
    with pytest.raises(B.DgError):
        B.dg_set_host_io(ctx, 7)
    B.dg_set_host_io(ctx, "staged")
    assert B.dg_host_io(ctx) == "staged"
    B.dg_set_host_io(ctx, "auto")
    assert B.dg_host_io(ctx) == auto
