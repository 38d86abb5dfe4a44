"""Host-side helpers of the package that need no GPU: the learned stage's parameter layout
and initialisation, and the batched solve's summary and tuning cache."""
import json
import math
import os

import numpy as np

import helm6_inputs as inputs


def test_init_theta_layout_and_scale():
    """Four 3x3x3 layers 2-16-16-16-2: weights N(0, 1/(27 c_in)) from the shared normal
    draws, each layer's biases (after its weights) zero, 15,602 parameters in all."""
    from paper_1212_1397_gb300 import learned, helm6 as H
    th = learned.init_theta(5)
    assert th.dtype == np.float32 and th.size == H.CNN_NPARAMS == 15602
    z = inputs.standard_normal(5, H.CNN_NPARAMS)
    o = 0
    for ci, co in zip((2, 16, 16, 16), (16, 16, 16, 2)):
        nw = 27 * ci * co
        w = th[o:o + nw]
        np.testing.assert_allclose(w, (z[o:o + nw] / math.sqrt(27.0 * ci)).astype(np.float32))
        assert abs(float(w.std()) * math.sqrt(27.0 * ci) - 1.0) < 0.15
        assert not np.any(th[o + nw:o + nw + co])
        o += nw + co
    assert o == th.size


def test_batch_summary():
    from paper_1212_1397_gb300 import batch
    items = [dict(N=10), dict(N=20), dict(N=30), dict(N=40)]
    stats = [dict(t_total_ms=t, status=s, iters=i) for t, s, i in
             [(1.0, "OK", 5), (2.0, "OK", 6), (3.0, "NOT_CONVERGED", 7), (4.0, "OK", 8)]]
    out = batch.summary(items, 0.5, stats)
    assert out["solves"] == 4 and out["solves_per_s"] == 8.0 and out["converged"] == 3
    assert out["iters_total"] == 26 and out["unknowns_total"] == 100
    assert out["p50_ms"] == 2.5 and abs(out["p99_ms"] - 3.97) < 1e-12


def test_tuning_cache(tmp_path):
    from paper_1212_1397_gb300 import batch
    assert batch.load_tuning(None) == batch.default_tuning()
    assert batch.load_tuning(str(tmp_path / "absent.json")) == batch.default_tuning()
    path = os.path.join(os.path.dirname(batch.__file__), "tuning", "batch_gb300.json")
    tun = batch.load_tuning(path)
    with open(path) as f:
        assert tun == json.load(f)
    assert set(tun["blocks"]) == {str(n) for n in inputs.BATCH_SIZES}
    for b in tun["blocks"].values():
        assert b["dot_blocks"] > 0 and b["update_blocks"] > 0
    assert tun["schedule"]["nthreads"] >= 1 and tun["schedule"]["order"] in ("as_drawn", "largest_first")
