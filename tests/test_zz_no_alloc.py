"""The allocation-free residual-norm entry point, dg_residual_norms_noalloc.

It serves callers that cannot allocate device memory where they need the
norms (real-time loops that must stay off the allocator, hosts whose
framework owns every device byte through its own pool).  Its partial
results live in a fixed static device array; this test checks that two
calls in a row give the same norms as the allocating path (dg_residual)
on the same values, to FP64 round-off of a different summation order
(rtol 1e-12), and that sizes beyond the static limit are refused.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import __graft_entry__
from cases import make_case

pytestmark = pytest.mark.gpu


def test_noalloc_norms_match_dg_residual():
    torch = pytest.importorskip("torch")
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding as B
    B.load()
    ctx = B.dg_create(0)
    try:
        # two calls in a row, different sizes and fields
        for kind, N, av in (("naca", 3, True), ("vortex", 5, False)):
            r, s = B.dg_reference_nodes(N)
            case = make_case(kind, N, r, s, av=av)
            m = case["mesh"]
            p = B.make_params(u_inf=case["u_inf"], av_on=av, prec="fp32")
            h = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, case["xy"], p)
            B.dg_set_state(ctx, h, case["U"])
            linf, l2 = B.dg_residual(ctx, h)            # allocating path
            L = B.dg_eval_rhs(ctx, h, m.K, len(r))      # the same FP32 values
            B.dg_mesh_free(ctx, h)
            vals = torch.tensor(L.astype(np.float32), device="cuda")
            out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            B.dg_residual_norms_noalloc(vals.data_ptr(), m.K, len(r), out.data_ptr(), None)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.allclose(got[:4], linf, rtol=1e-12, atol=0), (got[:4], linf)
            assert np.allclose(got[4:], l2, rtol=1e-12, atol=0), (got[4:], l2)
            # the same on a stream of the caller's (ordered after the values
            # are written on it; the result read after that stream finishes)
            side = torch.cuda.Stream()
            out2 = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
            side.wait_stream(torch.cuda.current_stream())
            B.dg_residual_norms_noalloc(vals.data_ptr(), m.K, len(r), out2.data_ptr(), side.cuda_stream)
            side.synchronize()
            assert np.array_equal(out2.cpu().numpy(), got)
        # beyond the static scratch limit, and bad arguments: refused, nothing launched
        with pytest.raises(B.DgError) as e:
            B.dg_residual_norms_noalloc(vals.data_ptr(), 1 << 26, 28, out.data_ptr(), None)
        assert e.value.status == B.DG_EINVAL and "limit" in str(e.value)
        with pytest.raises(B.DgError) as e:
            B.dg_residual_norms_noalloc(0, 10, 6, out.data_ptr(), None)
        assert e.value.status == B.DG_EINVAL
    finally:
        B.dg_destroy(ctx)
