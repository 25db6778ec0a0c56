"""ifactor_apply_noalloc: the integrating factor for callers that cannot
allocate device memory (their memory is owned by another component, or they
run inside a framework that forbids cudaMalloc once started).  It must give
the same result as the plan-based ifactor_apply, call after call, while the
static scratch array inside the library is reused.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

from tests.helpers import built, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _holed_set(seed, n):
    rng = np.random.default_rng(seed)
    box = np.array([[x, y, z] for z in range(n) for y in range(n) for x in range(n)], dtype=np.int32)
    keep = rng.random(len(box)) < 0.7
    keep[len(box) // 2] = True
    return box[keep] - 1


def test_noalloc_matches_planned_ifactor_twice():
    lgf = built()
    # calls in a row on the shared scratch: B = 16 at R = 9 and 15, B = 8 at R = 7
    cases = [(16, 0.2, 2, _holed_set(1, 3)), (16, 1.0, 3, _holed_set(2, 4)), (8, 0.05, 1, _holed_set(3, 4))]
    for B, alpha, ncomp, blocks in cases:
        rng = np.random.default_rng(int(alpha * 10) + ncomp)
        x = torch.from_numpy(rng.standard_normal((len(blocks), ncomp, B, B, B)).astype(np.float32)).cuda()
        y_ref = torch.zeros_like(x)
        table = lgf.Table(lgf.IFACTOR, alpha=alpha)
        plan = lgf.Plan(table, [lgf.Solve(B, ncomp, blocks, None)])
        plan.ifactor(x, y_ref)
        y = torch.full_like(x, float("nan"))
        lgf.ifactor_apply_noalloc(alpha, B, ncomp, blocks, x, y)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert rel_l2(a, b) < 1e-6, (B, alpha)


def test_noalloc_binding_checks_sizes():
    lgf = built()
    blocks = _holed_set(1, 2)
    x = torch.zeros((len(blocks), 1, 16, 16, 16), device="cuda")
    y = torch.zeros((len(blocks) - 1, 1, 16, 16, 16), device="cuda")
    with pytest.raises(ValueError):
        lgf.ifactor_apply_noalloc(0.2, 16, 1, blocks, x, y)


def test_noalloc_rejects_oversize():
    lgf = built()
    B = 16
    blocks = np.array([[x, y, z] for z in range(12) for y in range(12) for x in range(12)], dtype=np.int32)
    x = torch.zeros((len(blocks), 3, B, B, B), device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(lgf.LGFError) as e:
        lgf.ifactor_apply_noalloc(0.2, B, 3, blocks, x, y)
    assert e.value.status == lgf.LGF_ERR_ARG and "scratch" in str(e.value)
