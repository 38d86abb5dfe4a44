"""Batched solves and CUDA-graph replay of the Arnoldi steps, through the C-ABI.

* graph replay gives exactly the eager path's iterations and solution (same kernels, same
  order, replayed);
* helm6_solve_batch over heterogeneous problems (sizes, wavenumbers, faces, precisions) on
  several host threads and streams matches the oracle's solution of every problem and the
  one-by-one solves;
* options that graph replay needs are checked.
"""
import numpy as np
import pytest

import helm6_inputs as inputs
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_1397_gb300 import build, helm6
    build.build()
    return helm6


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _rhs(n, k, faces, seed):
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(seed, n, 1, margin_h=3)
    return prob, O.rhs(prob, O.sources.gaussians(src))


@pytest.mark.parametrize("precision,method", [("MIXED", "FGMRES"), ("FP64", "GMRES"), ("FP64", "FGMRES")])
def test_graph_replay_equals_eager(H, precision, method):
    n, k, faces = 21, 9.0 + 0.09j, "DNNDSN"
    _, F = _rhs(n, k, faces, 7)
    out = {}
    for graphs in (False, True):
        st_ = torch.cuda.Stream()
        with H.Solver(n, k, faces, precision=getattr(H, precision), method=getattr(H, method), max_restart=10,
                      stream=st_, use_graphs=graphs) as s:
            Fd = torch.from_numpy(F).cuda()
            torch.cuda.synchronize()
            u1, st1 = s.solve(Fd, tol=1e-9, restart=10, maxit=300)
            u2, st2 = s.solve(Fd, tol=1e-9, restart=10, maxit=300)  # replays the graphs
            out[graphs] = (u1.cpu().numpy(), st1, u2.cpu().numpy(), st2)
    e, g = out[False], out[True]
    assert e[1]["rc"] == 0 and g[1]["rc"] == 0
    assert e[1]["iters"] == g[1]["iters"] == g[3]["iters"]
    assert np.array_equal(e[0], g[0]) and np.array_equal(g[0], g[2])


def test_batch_matches_oracle_and_single_solves(H):
    specs = [(12, 6.0 + 0.06j, "DDDDDD"), (17, 9.5 + 0.1j, "NNDDSS"), (9, 4.0 + 0.04j, "DNNDDN"),
             (20, 12.0 + 0.12j, "NDDNNS"), (14, 7.0 + 0.07j, "DDNNSD"), (11, 5.5 + 0.05j, "NNNNNN")]
    solvers, Fs, us, refs = [], [], [], []
    for i, (n, k, faces) in enumerate(specs):
        prob, F = _rhs(n, k, faces, 20 + i)
        refs.append(O.solve(prob, F, tol=1e-12)[0])
        prec = H.MIXED if i % 2 == 0 else H.FP64
        meth = H.FGMRES if prec == H.MIXED else H.GMRES
        solvers.append(H.Solver(n, k, faces, precision=prec, method=meth, max_restart=20,
                                stream=torch.cuda.Stream(), use_graphs=True))
        Fs.append(torch.from_numpy(F).cuda())
        us.append(solvers[-1].empty())
    torch.cuda.synchronize()
    try:
        rc, stats = H.solve_batch(solvers, Fs, us, tol=1e-9, restart=20, maxit=400, nthreads=3)
        assert rc == 0, [st["status"] for st in stats]
        for u, ref, st in zip(us, refs, stats):
            assert st["relres"] <= 1e-9
            assert rel2(u.cpu().numpy(), ref) < 1e-6
        # one by one, on the same contexts: the same solutions and iteration counts
        for s, F, u, st in zip(solvers, Fs, us, stats):
            u1, st1 = s.solve(F, tol=1e-9, restart=20, maxit=400)
            assert st1["iters"] == st["iters"]
            assert np.array_equal(u1.cpu().numpy(), u.cpu().numpy())
    finally:
        for s in solvers:
            s.close()


def test_shared_streams_and_own_streams(H):
    """Contexts that share one stream (graph capture happens on each context's private
    stream) and contexts with their own streams give the one-by-one results."""
    specs = [(10, 5.0 + 0.05j, "DDNNSS"), (13, 6.5 + 0.07j, "NNDDDD"), (8, 4.0 + 0.04j, "DNDNSN")]
    shared = torch.cuda.Stream()
    for mode in ("shared", "own"):
        solvers, Fs, us, refs = [], [], [], []
        for i, (n, k, faces) in enumerate(specs):
            _, F = _rhs(n, k, faces, 40 + i)
            kw = dict(stream=shared) if mode == "shared" else dict(own_stream=True)
            solvers.append(H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=10,
                                    use_graphs=True, **kw))
            Fs.append(torch.from_numpy(F).cuda())
            us.append(solvers[-1].empty())
        torch.cuda.synchronize()
        try:
            rc, stats = H.solve_batch(solvers, Fs, us, tol=1e-9, restart=10, maxit=300, nthreads=3)
            assert rc == 0
            for s, F, u, st in zip(solvers, Fs, us, stats):
                u1, st1 = s.solve(F, tol=1e-9, restart=10, maxit=300)
                assert st1["iters"] == st["iters"]
                assert np.array_equal(u1.cpu().numpy(), u.cpu().numpy())
        finally:
            for s in solvers:
                s.close()


@pytest.mark.parametrize("n,k,faces", [(21, 9.0 + 0.09j, "DNNDSN"), (33, 14.0, "DDNNSS")])
def test_device_driven_solve_equals_host_driven(H, n, k, faces):
    """use_graphs = 2: the whole mixed FGMRES solve as one graph launch, every convergence
    decision on the device (conditional nodes): the same iterations, cycles and solution as
    the host-driven solve (same kernels, no wasted step), twice in a row (graph reused), and
    the oracle's solution."""
    prob, F = _rhs(n, k, faces, 11)
    ref = O.solve(prob, F, tol=1e-12)[0]
    Fd = torch.from_numpy(F).cuda()
    out = {}
    for mode in (0, 2):
        with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=12,
                      stream=torch.cuda.Stream(), use_graphs=mode) as s:
            torch.cuda.synchronize()
            u1, st1 = s.solve(Fd, tol=1e-9, restart=12, maxit=400)
            u2, st2 = s.solve(Fd, tol=1e-9, restart=12, maxit=400)
            out[mode] = (u1.cpu().numpy(), st1, u2.cpu().numpy(), st2)
    h, d = out[0], out[2]
    assert h[1]["rc"] == 0 and d[1]["rc"] == 0 and d[3]["rc"] == 0
    assert d[1]["iters"] == h[1]["iters"] == d[3]["iters"] and d[1]["outer"] == h[1]["outer"]
    assert np.array_equal(d[0], h[0]) and np.array_equal(d[0], d[2])
    assert abs(d[1]["relres"] - h[1]["relres"]) <= 1e-12 * h[1]["relres"]
    assert np.allclose(d[1]["history"], h[1]["history"], rtol=1e-12, atol=0)
    assert rel2(d[0], ref) < 1e-6


def test_device_driven_batch_is_one_launch_and_matches(H):
    """helm6_solve_batch over device-driven contexts of different sizes, wavenumbers and faces
    (one graph launch for the whole batch): every solution equals the host-driven solve of
    the same problem (bitwise) and the oracle's, per-problem device times are reported, and
    a second call reuses the batch graph."""
    specs = [(12, 6.0 + 0.06j, "DDDDDD"), (17, 9.5 + 0.1j, "NNDDSS"), (9, 4.0 + 0.04j, "DNNDDN"),
             (20, 12.0 + 0.12j, "NDDNNS"), (14, 7.0 + 0.07j, "DDNNSD"), (24, 11.0, "DDNNSS")]
    solvers, Fs, us, refs, host = [], [], [], [], []
    for i, (n, k, faces) in enumerate(specs):
        prob, F = _rhs(n, k, faces, 60 + i)
        refs.append(O.solve(prob, F, tol=1e-12)[0])
        solvers.append(H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=16,
                                own_stream=True, use_graphs=2))
        Fs.append(torch.from_numpy(F).cuda())
        us.append(solvers[-1].empty())
        with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=16) as s0:
            uh, sth = s0.solve(Fs[-1], tol=1e-9, restart=16, maxit=400)
            host.append((uh.cpu().numpy(), sth))
    torch.cuda.synchronize()
    try:
        for call in range(2):
            for u in us:
                u.zero_()
            rc, stats = H.solve_batch(solvers, Fs, us, tol=1e-9, restart=16, maxit=400, nthreads=4)
            assert rc == 0, [st["status"] for st in stats]
            for u, ref, st, (uh, sth) in zip(us, refs, stats, host):
                assert st["relres"] <= 1e-9 and st["iters"] == sth["iters"], (st["iters"], sth["iters"])
                assert np.array_equal(u.cpu().numpy(), uh)
                assert rel2(u.cpu().numpy(), ref) < 1e-6
                assert st["t_total_ms"] > 0
    finally:
        for s in solvers:
            s.close()


def test_block_options_are_checked(H):
    with pytest.raises(H.Helm6Error):
        H.Solver(8, 3.0, "DDDDDD", dot_blocks=-1)
    with pytest.raises(H.Helm6Error):
        H.Solver(8, 3.0, "DDDDDD", update_blocks=-1)
