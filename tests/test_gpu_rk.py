"""GPU parity of the stage local operators (App. A) and of one IF-HERK step
(Schemes A, B and C of eq. ifherk_schemes, Sec. 3.2-3.3, xIF-HERK masks of
Sec. 5) against the FP64 oracle.

The GPU step uses a rearranged form with five (C: six) integrating-factor applications;
the oracle runs the paper's q/w recursions, so this also checks the
rearrangement.  Tolerances: operators relative L2 <= 1e-6; the step (three
FP32 Poisson solves, five integrating factors, three nonlinear terms)
relative L2 <= 2e-6 on the velocity change u_{k+1} - u_k.
"""
import numpy as np
import pytest

import oracle as O
from tests.helpers import built, rel_l2
from tests.rk_cases import from_blocks_dense, small_case, to_blocks_dense

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _plan(lgf, cs, dt, re, scheme=0):
    rk = lgf.RKPlan(cs["B"], cs["soln"], cs["dx"], dt, re, scheme=scheme)
    xs = rk.blocks(0)
    assert set(map(tuple, xs.tolist())) == set(map(tuple, cs["xsoln"].tolist()))
    return rk, xs


def test_local_operators():
    lgf = built()
    cs = small_case(B=8)
    B, n, org, dx = cs["B"], cs["n"], cs["origin"], cs["dx"]
    rk, xs = _plan(lgf, cs, 0.5, 10.0)
    rng = np.random.default_rng(3)
    xm = cs["masks"]["xsoln"]
    f = rng.standard_normal((3, n, n, n)) * xm
    c = rng.standard_normal((1, n, n, n)) * xm
    uinf = (0.3, -0.2, 0.1)
    cases = [
        (lgf.OP_CURL, f, O.op_C(f, dx), 3),
        (lgf.OP_CURL_T, f, O.op_Ct(f, dx), 3),
        (lgf.OP_DIV_T, f, O.op_Gt(f, dx)[None], 1),
        (lgf.OP_GRAD, c, O.op_G(c[0], dx), 3),
        (lgf.OP_NONLINEAR, f, -0.7 * O.op_N((f + np.reshape(uinf, (3, 1, 1, 1))) * xm, dx) * cs["masks"]["soln"], 3),
    ]
    for op, inp, ref, nout in cases:
        d_in = torch.from_numpy(to_blocks_dense(inp, B, xs, org)).cuda()
        d_out = torch.zeros((len(xs), nout, B, B, B), device="cuda")
        rk.op(op, d_in, d_out, coef=-0.7 if op == lgf.OP_NONLINEAR else 1.0, uinf=uinf)
        got = from_blocks_dense(d_out.cpu().numpy(), B, xs, org, (n, n, n))
        refm = ref * xm
        assert rel_l2(got, refm) < 1e-6, (op, rel_l2(got, refm))


@pytest.mark.parametrize("scheme,uinf", [("A", (0.0, 0.0, 0.0)), ("A", (0.05, -0.02, 0.1)),
                                         ("B", (0.05, -0.02, 0.1)), ("C", (0.05, -0.02, 0.1))])
def test_if_herk_step_matches_oracle(scheme, uinf):
    lgf = built()
    cs = small_case(B=8, amp=3.0)
    B, n, org, dx = cs["B"], cs["n"], cs["origin"], cs["dx"]
    dt, re = 0.5, 10.0
    rk, xs = _plan(lgf, cs, dt, re, scheme="ABC".index(scheme))
    u0 = cs["u0"]
    ref = O.if_herk_step(u0, dt, re, dx, uinf, cs["masks"], O.lgf_cube(64), nonlinear=True,
                         tab=O.SCHEMES[scheme])
    d_u0 = torch.from_numpy(to_blocks_dense(u0, B, xs, org)).cuda()
    d_u1 = torch.zeros_like(d_u0)
    rk.step(d_u0, d_u1, uinf)
    torch.cuda.synchronize()
    got = from_blocks_dense(d_u1.cpu().numpy(), B, xs, org, (n, n, n))
    assert rel_l2(got - u0, ref - u0) < 2e-6, rel_l2(got - u0, ref - u0)
    assert rel_l2(got, ref) < 1e-6


def test_step_divergence_free_on_gpu():
    """G^T u_{k+1} on the D_supp cells, computed by the GPU operator, is at FP32 roundoff."""
    lgf = built()
    cs = small_case(B=8, amp=3.0)
    B, n, org, dx = cs["B"], cs["n"], cs["origin"], cs["dx"]
    rk, xs = _plan(lgf, cs, 0.5, 10.0)
    d_u0 = torch.from_numpy(to_blocks_dense(cs["u0"], B, xs, org)).cuda()
    d_u1 = torch.zeros_like(d_u0)
    rk.step(d_u0, d_u1, (0.05, -0.02, 0.1))
    div = torch.zeros((len(xs), 1, B, B, B), device="cuda")
    rk.op(lgf.OP_DIV_T, d_u1, div)
    nsoln = len(cs["soln"])  # soln blocks come first in the field order
    d = div[:nsoln].abs().max().item()
    assert d < 1e-5 * d_u1.abs().max().item() / dx, d


def test_temporal_order_of_schemes():
    """Observed order of the velocity over T = 2 (Re = 10, the ring case at amplitude 10)
    against a 128-step reference: Scheme A 2, Schemes B and C 3 (the y-orders of the paper's
    table of scheme orders)."""
    lgf = built()
    cs = small_case(B=8, amp=10.0)
    B, org = cs["B"], cs["origin"]
    re, T, uinf = 10.0, 2.0, (0.05, -0.02, 0.1)
    want = {0: (1.7, 2.3), 1: (2.6, 3.4), 2: (2.6, 3.4)}
    for scheme, (lo, hi) in want.items():
        out = {}
        for nst in (4, 8, 16, 128):
            rk = lgf.RKPlan(B, cs["soln"], cs["dx"], T / nst, re, scheme=scheme)
            xs = rk.blocks(0)
            u = torch.from_numpy(to_blocks_dense(cs["u0"], B, xs, org)).cuda()
            v = torch.zeros_like(u)
            for _ in range(nst):
                rk.step(u, v, uinf)
                u, v = v, u
            torch.cuda.synchronize()
            out[nst] = u.double().cpu().numpy()
        err = [np.linalg.norm(out[n] - out[128]) / np.linalg.norm(out[128]) for n in (4, 8, 16)]
        orders = [np.log2(err[0] / err[1]), np.log2(err[1] / err[2])]
        assert all(lo <= o <= hi for o in orders), (scheme, err, orders)
