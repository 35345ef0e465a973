"""Mixed-precision products against the FP64 oracle on the workloads'
shapes, and the batched path against the oracle.

* Increments after 100 SSP-RK3 steps: || (U_100 - U_0)_gpu - (U_100 -
  U_0)_oracle || / || (U_100 - U_0)_oracle ||, per conserved variable.  The
  increment, not the state, is compared: the state is dominated by U_0,
  which both sides share.  The GPU state is FP32 and is rounded at every
  stage (2^-24 of U per value), which sets a floor under the increment's
  error of every GPU path, FP32 included; the bounds (BOUNDS, from GB300
  measurements with a margin) are stated per case and precision:
    - cylinder, N = 6, smoothly perturbed state, dt at CFL 0.3: the
      increment is 2.3e-2 of U and the floor about 1e-4;
    - periodic vortex, N = 4, artificial viscosity with a jump of all
      variables by half across x = 5 (troubled cells), dt at the viscous
      limit: increment 2e-2 of U;
    - NACA 0012, N = 4, artificial viscosity with a jump across x = 2: the
      viscous limit of the small wall elements makes dt so small that the
      increment is 4.5e-5 of U and the FP32 floor dominates (about 5e-2 for
      every precision); there the mixed products must stay within 10% of
      the FP32 path's error.
* The vortex convergence order and the mixed-precision errors at N = 4 and
  6 (N = 2, 3 in test_gpu_tensor.py).
* dg_batch_step on a batch of curved and periodic meshes of degrees 2..5
  with noisy states, ten SSP-RK3 steps, against the oracle on every
  element of every mesh: the state element by element at the single-mesh
  step tolerances, and the increment.
"""
import numpy as np
import pytest

import __graft_entry__
from oracle.dg import Oracle
from paper_1208_4772_gb300.inputs import states
from cases import make_case, rel_l2_per_var

pytestmark = pytest.mark.gpu

# largest relative L2 error of the 100-step increment, per case and
# precision of the products (measured on GB300 with margin; see DESIGN)
BOUNDS = {"naca4_av": {"fp32": 1e-1, "tf32": 1e-1, "bf16x3": 1e-1},
          "vortex4_av": {"fp32": 3e-4, "tf32": 1e-3, "bf16x3": 3e-4},
          "cyl6": {"fp32": 3e-4, "tf32": 4e-4, "bf16x3": 3e-4}}
_fp32_err = {}


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


def precision_case(B, name):
    if name in ("naca4_av", "vortex4_av"):
        N = 4
        r, s = B.dg_reference_nodes(N)
        if name == "naca4_av":
            case = make_case("naca", N, r, s, av=True, perturb=0.0)
            cut = 2.0
        else:
            case = make_case("vortex", N, r, s, av=True)
            cut = 5.0
        x = case["xy"][..., 0]
        case["U"] = case["U"] * np.where(x > cut, 1.5, 1.0)[:, None, :]
        dt = 0.5 * states.time_step(case["mesh"].verts, case["U"], N, eps0=0.3)
    else:
        N = 6
        r, s = B.dg_reference_nodes(N)
        case = make_case("cyl", N, r, s)
        dt = states.time_step(case["mesh"].verts, case["U"], N)
    case["U"] = case["U"].astype(np.float32).astype(np.float64)
    return case, dt


_oracle_cache = {}


def oracle_increment(name, case, dt, nsteps):
    if name not in _oracle_cache:
        m = case["mesh"]
        o = Oracle(case["N"], m.EToE, m.EToF, m.bc, case["xy"], u_inf=case["u_inf"], av=case["av"])
        U = case["U"].copy()
        for _ in range(nsteps):
            U = o.ssp_rk3_step(U, dt)
        eps = o.sensor(case["U"]) if case["av"] else None
        _oracle_cache[name] = (U - case["U"], eps)
    return _oracle_cache[name]


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
@pytest.mark.parametrize("name", ["naca4_av", "vortex4_av", "cyl6"])
def test_increment_100_steps_vs_oracle(B, ctx, name, prec):
    case, dt = precision_case(B, name)
    m = case["mesh"]
    nsteps = 100
    dU_o, eps = oracle_increment(name, case, dt, nsteps)
    p = B.make_params(u_inf=case["u_inf"], av_on=case["av"], prec=prec)
    h = B.dg_mesh_upload(ctx, case["N"], m.EToE, m.EToF, m.bc, case["xy"], p)
    B.dg_set_state(ctx, h, case["U"])
    if case["av"]:
        nv = B.dg_av_count(ctx, h)
        assert nv == int(np.sum(eps > 0)) and nv > 10, (nv, int(np.sum(eps > 0)))
    B.dg_step(ctx, h, dt, nsteps)
    U = B.dg_get_state(ctx, h, m.K, case["U"].shape[2])
    B.dg_mesh_free(ctx, h)
    err = rel_l2_per_var(U - case["U"], dU_o)
    rel = np.linalg.norm(dU_o) / np.linalg.norm(case["U"])
    print("\nincrement %s %s: rel L2 per variable %s; state %s (|dU|/|U| = %.2e)"
          % (name, prec, " ".join("%.3e" % x for x in err),
             " ".join("%.2e" % x for x in rel_l2_per_var(U, case["U"] + dU_o)), rel))
    assert np.all(np.isfinite(U))
    assert np.all(err <= BOUNDS[name][prec]), err
    if prec == "fp32":
        _fp32_err[name] = err
    elif name == "naca4_av" and name in _fp32_err:
        assert np.all(err <= 1.1 * _fp32_err[name]), (err, _fp32_err[name])


def _vortex_error(B, ctx, N, n, prec, T=0.2, length=10.0):
    from oracle import basis
    from oracle.operators import ReferenceElement
    from paper_1208_4772_gb300.inputs import meshes
    ref = ReferenceElement(N)
    r, s = B.dg_reference_nodes(N)
    Icub = ref.Vq @ np.linalg.inv(basis.vandermonde(N, r, s))
    m = meshes.periodic_square(n, length=length, seed=7)
    xy = meshes.straight_nodes(m.verts, r, s)
    U = states.vortex_state(xy, period=(length, length))
    dt0 = states.time_step(m.verts, U, N, cfl=0.3)
    nst = int(np.ceil(T / dt0))
    h = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, xy, B.make_params(u_inf=states.freestream(0.5, 45.0), prec=prec))
    B.dg_set_state(ctx, h, U)
    B.dg_step(ctx, h, T / nst, nst)
    Ug = B.dg_get_state(ctx, h, m.K, len(r))
    B.dg_mesh_free(ctx, h)
    Ue = states.vortex_state(xy, t=T, period=(length, length))
    e = (Ug - Ue)[:, 0, :] @ Icub.T
    v = m.verts
    J = 0.25 * np.abs((v[:, 1, 0] - v[:, 0, 0]) * (v[:, 2, 1] - v[:, 0, 1])
                      - (v[:, 2, 0] - v[:, 0, 0]) * (v[:, 1, 1] - v[:, 0, 1]))
    return np.sqrt(np.sum(J[:, None] * ref.wq[None, :] * e * e))


def test_vortex_order_and_mixed_precision_high_degree(B, ctx):
    """The isentropic vortex at T = 0.2 on periodic meshes (those of the
    oracle's convergence pins), density L2 error against the exact solution.

    N = 4, n = 8 -> 16: the FP64 oracle converges at order 4.55 here; the
    FP32 path and BF16 x3 products at 4.4 (the FP32 state's rounding adds
    about 10% to the fine-mesh error), order >= 4.3 is pinned, and BF16 x3
    stays within 5% of FP32.  TF32 products reach order 3.9 with a
    fine-mesh error 1.45 times FP32's (pinned: order >= 3.7, ratio <= 1.7).
    N = 6, n = 8 -> 12: the oracle converges at order 6.8, and so does the
    GPU's FP64 path (pinned >= 6.5), but every FP32-state path meets a floor
    near 1e-4 on the finer mesh (storage rounding alone gives 3.8e-5 in an
    oracle run that rounds to FP32 after every stage; the FP32 right-hand
    side's arithmetic adds the rest), so the order is not observable there:
    pinned are BF16 x3 within 5% of FP32, TF32 within 2.6 times FP32, and
    the FP32 fine-mesh error below 1.3e-4."""
    res = {}
    for N, n1, n2, precs in ((4, 8, 16, ("fp32", "tf32", "bf16x3")), (6, 8, 12, ("fp64", "fp32", "tf32", "bf16x3"))):
        for prec in precs:
            e1, e2 = _vortex_error(B, ctx, N, n1, prec), _vortex_error(B, ctx, N, n2, prec)
            res[(N, prec)] = (e1, e2, np.log(e1 / e2) / np.log(n2 / n1))
    print("\nvortex (N, products): (coarse error, fine error, order) %s"
          % {k: ("%.3e" % a, "%.3e" % b, "%.2f" % o) for k, (a, b, o) in res.items()})
    assert res[(4, "fp32")][2] >= 4.3 and res[(4, "bf16x3")][2] >= 4.3, res
    assert res[(4, "bf16x3")][1] <= 1.05 * res[(4, "fp32")][1], res
    assert res[(4, "tf32")][2] >= 3.7 and res[(4, "tf32")][1] <= 1.7 * res[(4, "fp32")][1], res
    assert res[(6, "fp64")][2] >= 6.5, res
    assert res[(6, "bf16x3")][1] <= 1.05 * res[(6, "fp32")][1], res
    assert res[(6, "tf32")][1] <= 2.6 * res[(6, "fp32")][1], res
    assert res[(6, "fp32")][1] <= 1.3e-4, res


# the batched path after ten steps against the oracle: the state element by
# element at the single-mesh step tolerances (relative to the element's
# state), and the increment relative to its norm plus the FP32 storage floor
# (3 x 2^-24 of the state per step).  On the airfoil meshes the FP32
# right-hand side itself differs from the oracle's by a few 1e-3 of L (the
# thin wall elements' cancellation; 1e-5 of the volume term, the single-mesh
# tolerance), which the increment bound leaves room for; an indexing error
# moves whole increments.
BATCH_STATE_TOL = {"fp32": 1e-5, "tf32": 1e-4, "bf16x3": 1e-5}
BATCH_INC_TOL = {"fp32": 1e-2, "tf32": 1e-2, "bf16x3": 1e-2}


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_batch_step_matches_oracle(B, ctx, prec):
    """Five meshes of degrees 2..5 (curved airfoil and cylinder meshes, a
    periodic vortex), noisy states, one persistent launch per stage over all
    of them, ten SSP-RK3 steps: every element of every mesh against the
    oracle."""
    nsteps = 10
    cases, dts = [], []
    for i, (kind, N) in enumerate((("naca", 2), ("cyl", 3), ("vortex", 4), ("naca", 5), ("cyl", 4))):
        r, s = B.dg_reference_nodes(N)
        c = make_case(kind, N, r, s, seed=10 + i)
        c["U"] = c["U"].astype(np.float32).astype(np.float64)
        cases.append(c)
        dts.append(0.5 * states.time_step(c["mesh"].verts, c["U"], N))
    hs = []
    for c in cases:
        m = c["mesh"]
        hs.append(B.dg_mesh_upload(ctx, c["N"], m.EToE, m.EToF, m.bc, c["xy"], B.make_params(u_inf=c["u_inf"], prec=prec)))
        B.dg_set_state(ctx, hs[-1], c["U"])
    B.dg_batch_step(ctx, hs, dts, nsteps)
    report = []
    for h, c, dt in zip(hs, cases, dts):
        m = c["mesh"]
        U1 = B.dg_get_state(ctx, h, m.K, c["U"].shape[2])
        B.dg_mesh_free(ctx, h)
        o = Oracle(c["N"], m.EToE, m.EToF, m.bc, c["xy"], u_inf=c["u_inf"])
        Uo = c["U"].copy()
        for _ in range(nsteps):
            Uo = o.ssp_rk3_step(Uo, dt)
        per_elt = np.linalg.norm(U1 - Uo, axis=(1, 2)) / np.linalg.norm(Uo, axis=(1, 2))
        dU, dU_o = U1 - c["U"], Uo - c["U"]
        floor = 3 * nsteps * 2.0 ** -24 * np.linalg.norm(c["U"].transpose(1, 0, 2).reshape(4, -1), axis=1)
        inc = np.linalg.norm((dU - dU_o).transpose(1, 0, 2).reshape(4, -1), axis=1) / (
            np.linalg.norm(dU_o.transpose(1, 0, 2).reshape(4, -1), axis=1) + floor)
        report.append((c["N"], "%.2e" % per_elt.max(), "%.2e" % inc.max()))
        assert np.all(np.isfinite(U1))
        assert per_elt.max() <= BATCH_STATE_TOL[prec], (c["N"], per_elt.max())
        assert np.all(inc <= BATCH_INC_TOL[prec]), (c["N"], inc)
    print("\nbatch %s: (N, max per-element state error, increment error) %s" % (prec, report))
