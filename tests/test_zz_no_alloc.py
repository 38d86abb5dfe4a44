"""helm6_residual_noalloc, the residual entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (an allocator or memory pool that must not
re-enter it, a runtime that owns all device memory, a real-time loop that must not block
on allocation).  Its output r = F - A u and ||r||^2 is checked against the existing
helm6_apply_A entry point, within the FP64 stencil tolerance of the other tests, on
consecutive calls (the calls share the library's static scratch array).

The file is named to be collected last: a run that stops at the first failure has then
already run every other test.
"""
import numpy as np
import pytest

import helm6_inputs as inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_1397_gb300 import build, helm6
    build.build()
    return helm6


def _reference(H, n, k, faces, F, u):
    """F - A u and its squared norm from the existing helm6_apply_A entry point."""
    with H.Solver(n, k, faces, precision=H.FP64) as s:
        r = F - s.apply_A(u)
    return r, float((r.abs() ** 2).sum())


def test_noalloc_residual_matches_apply_A_on_consecutive_calls(H):
    cases = [(37, 9.0 + 0.3j, "DDNNSS", 1), (21, 7.5, "NNDNNS", 2), (37, 9.0 + 0.3j, "DDNNSS", 3)]
    for n, k, faces, seed in cases:
        mx, my, mz = inputs.dims(n, faces)
        shape = (mz, my, mx)
        F = torch.from_numpy(inputs.complex_normal(10 + seed, shape)).cuda()
        u = torch.from_numpy(inputs.complex_normal(20 + seed, shape)).cuda()
        r_ref, ss_ref = _reference(H, n, k, faces, F, u)
        r = torch.full(shape, float("nan"), dtype=torch.complex128, device="cuda")
        ss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert H.residual_noalloc(n, k, faces, F, u, r, ss) == 0
        torch.cuda.synchronize()
        err = float((r - r_ref).abs().max() / r_ref.abs().max())
        assert err < 1e-12, (n, faces, err)
        assert abs(float(ss[0]) - ss_ref) <= 1e-12 * ss_ref, (n, faces, float(ss[0]), ss_ref)


def test_noalloc_rejects_grids_beyond_the_static_scratch(H):
    # 1000^3 needs more thread blocks than the static scratch has slots: rejected up front
    dummy = torch.zeros(1, dtype=torch.complex128, device="cuda")
    ss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(H.Helm6Error):
        H.residual_noalloc(1000, 10.0, "DDDDDD", dummy, dummy, dummy, ss)
    with pytest.raises(H.Helm6Error):
        H.residual_noalloc(16, 10.0, "SDDDDD", dummy, dummy, dummy, ss)
    assert np.isfinite(float(ss[0]))
