"""The allocation-free trace apply (hdg_trace_apply_noalloc) against hdg_trace_apply.

hdg_trace_apply_noalloc serves callers that must not allocate device memory once they run: hosts
whose device memory is handed to their own pool allocator, and time-critical loops that cannot
afford cudaMalloc's possible device-wide synchronisation. It must give the output of
hdg_trace_apply, the entry point it varies, on consecutive calls that share its static scratch,
for every degree and on meshes with walls as well as periodic ones, and refuse meshes whose
intermediate vectors do not fit that scratch. This file is collected last so that a run stopping
at its first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = a.cpu().numpy().ravel(), b.cpu().numpy().ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize('periodic_x', [True, False])
@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_trace_apply_noalloc_matches_trace_apply_on_consecutive_calls(k, periodic_x):
    import paper_2410_09790_gb300 as H
    ctx = H.Context(8, k, periodic_x=periodic_x)
    sL = ctx.shapes()[2]
    rng = np.random.default_rng(2024 + 10 * k + periodic_x)
    out = torch.empty(sL, dtype=torch.float64, device='cuda')
    for c in (2e-3, 2e-3, 1.0):                      # consecutive calls share the static scratch
        lam = torch.from_numpy(rng.standard_normal(sL)).cuda()
        got = ctx.hdg_trace_apply_noalloc(c, lam, out).clone()
        ref = ctx.hdg_trace_apply(c, lam)
        l2, mx = _rel(got, ref)
        assert l2 <= 1e-11 and mx <= 1e-10, (c, l2, mx)
    ctx.close()


def test_trace_apply_noalloc_rejects_wrong_sizes_and_large_meshes():
    import paper_2410_09790_gb300 as H
    ctx = H.Context(4, 2)
    sL = ctx.shapes()[2]
    lam = torch.zeros(sL, dtype=torch.float64, device='cuda')
    with pytest.raises(ValueError):
        ctx.hdg_trace_apply_noalloc(1.0, lam, torch.empty(ctx.nL - 1, dtype=torch.float64, device='cuda'))
    ctx.close()
    ctx = H.Context(190, 1)                          # 3 nlambda + 6 ncells > 2^20 doubles
    sL = ctx.shapes()[2]
    lam = torch.zeros(sL, dtype=torch.float64, device='cuda')
    out = torch.empty_like(lam)
    with pytest.raises(H.HdgError, match='maximum'):
        ctx.hdg_trace_apply_noalloc(1.0, lam, out)
    ctx.close()
