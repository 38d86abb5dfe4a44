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
    # reference arm: only rank 0 runs and prints (the oracle sample is replaced by a stub)
    bench.oracle_sample = lambda cfg, iters: (123.0, 0.5)
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
    assert line["impl"] == "reference" and line["value"] == 123.0 and line["n_gpus"] == 2


def test_metric_names_the_workload():
    """The headline workload keeps its metric string; the others name their own size,
    wavenumber, faces and tolerance."""
    import bench
    assert bench.metric_for(bench.WORKLOAD) == bench.METRIC
    m = bench.metric_for("mixed_n256_k80c")
    assert "256^3" in m and "k=80+0.8i" in m and "DDNNSS" in m and "1e-8" in m
    assert "1e-10" in bench.metric_for("dirichlet_n32_k10")
