"""bench.py's N > 1 path on the CPU: two `gloo` ranks (world size 2) run the bench's own
rank helpers -- the barrier, the max over ranks of the timed values, the per-rank replica
seeds -- and the reference arm's rank gating (rank 0 alone prints)."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [5.0, 7.5][rank]
    bench.sync_all(dist, cuda=False)
    worst = bench.reduce_max(local_ms, dist)
    seeds = bench.replica_seeds(rank)
    # reference arm: only rank 0 runs and prints (the oracle's unit costs and its recorded
    # complete solve are replaced by stubs: 0.1 s per unit, 40 iterations)
    bench.oracle_problem = lambda cfg, seed: (None, None, None)
    bench.oracle_unit_costs = lambda O, prob, x: dict(setup=0.1, precond=0.1, apply_A=0.1, proj=0.1)
    bench.ORACLE_FULL[bench.WORKLOAD] = dict(iters=40, cycles=2, seconds=1.0)
    args = type("A", (), dict(warmup=0, steps=1, gpus=world, workload=bench.WORKLOAD))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, dict(bench.inputs.WORKLOADS[bench.WORKLOAD]), rank, world)
    bench.sync_all(dist, cuda=False)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(dict(worst=worst, seeds=seeds, printed=buf.getvalue()), f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert res[0]["worst"] == res[1]["worst"] == 7.5
    assert res[0]["seeds"] != res[1]["seeds"]
    assert res[1]["printed"] == ""
    line = json.loads(res[0]["printed"])
    # 0.1 s x (set-up + initial A + 40 (A_p^-1 + A) + 2 cycles (A_p^-1 + A)
    # + (465 + 30) + (55 + 10) projections) = 0.1 s x 646
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert abs(line["value"] - 64600.0) < 1e-6, line["value"]


def test_oracle_projection_counts_the_gmres_work():
    """The projection of the oracle's GMRES(m) from its unit costs: per column j of a cycle
    j + 1 projections, per cycle one more per column (V y), A_p^-1 and A per iteration and
    per cycle, plus the set-up and the initial residual."""
    import bench
    u = dict(setup=1.0, precond=10.0, apply_A=100.0, proj=1000.0)
    ms, cyc = bench.oracle_projection(u, 35, 30)
    assert cyc == 2
    proj = (30 * 31 // 2 + 30) + (5 * 6 // 2 + 5)
    assert ms == 1e3 * (1.0 + 100.0 + 35 * 110.0 + 2 * 110.0 + proj * 1000.0)


def test_metric_names_the_workload():
    """The headline workload keeps its metric string; the others name their own size,
    wavenumber, faces and tolerance."""
    import bench
    assert bench.metric_for(bench.WORKLOAD) == bench.METRIC
    m = bench.metric_for("mixed_n256_k80c")
    assert "256^3" in m and "k=80+0.8i" in m and "DDNNSS" in m and "1e-8" in m
    assert "1e-10" in bench.metric_for("dirichlet_n32_k10")
