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


def test_noalloc_residual_matches_the_oracle(H):
    """One small case straight against the oracle's operator (FP64, elementwise)."""
    import oracle as O
    n, k, faces = 11, 6.0 + 0.2j, "DDNNSS"
    mx, my, mz = inputs.dims(n, faces)
    F = inputs.complex_normal(31, (mz, my, mx))
    u = inputs.complex_normal(32, (mz, my, mx))
    r_or = F - O.apply_A(O.Problem(n, k, faces), u)
    r = torch.empty((mz, my, mx), dtype=torch.complex128, device="cuda")
    ss = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert H.residual_noalloc(n, k, faces, torch.from_numpy(F).cuda(), torch.from_numpy(u).cuda(), r, ss) == 0
        torch.cuda.synchronize()
        got = r.cpu().numpy()
        assert np.abs(got - r_or).max() <= 1e-12 * np.abs(r_or).max()
        assert abs(float(ss[0]) - float((np.abs(r_or) ** 2).sum())) <= 1e-12 * float((np.abs(r_or) ** 2).sum())


def test_noalloc_rejects_grids_beyond_the_static_scratch(H):
    """ceil(mx/32) ceil(my/8) ceil(mz/16) <= 65,536 blocks: n = 640 (64,000 blocks) runs,
    n = 641 (69,741) is rejected before any device work, as is a Sommerfeld-like face off z."""
    ss = torch.zeros(1, dtype=torch.float64, device="cuda")
    z640 = torch.zeros((640, 640, 640), dtype=torch.complex128, device="cuda")
    assert H.residual_noalloc(640, 10.0, "DDDDDD", z640, z640, torch.empty_like(z640), ss) == 0
    torch.cuda.synchronize()
    assert float(ss[0]) == 0.0
    del z640
    e641 = torch.empty((641, 641, 641), dtype=torch.complex128, device="cuda")
    with pytest.raises(H.Helm6Error):
        H.residual_noalloc(641, 10.0, "DDDDDD", e641, e641, e641, ss)
    del e641
    torch.cuda.empty_cache()
    s16 = torch.zeros((16, 16, 17), dtype=torch.complex128, device="cuda")
    with pytest.raises(H.Helm6Error):
        H.residual_noalloc(16, 10.0, "SDDDDD", s16, s16, s16, ss)
    assert np.isfinite(float(ss[0]))
