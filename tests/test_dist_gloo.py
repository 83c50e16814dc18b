"""The multi-process path of bench.py on CPU: world size 2 over gloo.

The solver does not shard across GPUs (one GPU holds every subdomain; several
GPUs run independent replicas), so the only cross-rank logic is the bench's
timing aggregation: barrier, max over ranks of the step time, sum of the
kernel-launch counts, and rank 0 alone printing.  The reference arm prints
only on rank 0 and the other ranks exit without work."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench

    d = bench.Dist(backend="gloo")
    d.barrier()
    mx = d.max(10.0 * (rank + 1))
    sm = d.sum(rank + 1)
    d.barrier()
    d.close()
    with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as f:
        f.write("%r %r\n" % (mx, sm))


def test_gloo_world2_max_and_sum(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        mx, sm = open(tmp_path / ("r%d.txt" % r)).read().split()
        assert float(mx) == 20.0 and float(sm) == 3.0


def test_reference_arm_nonzero_rank_exits_quietly(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""


def test_algorithmic_bytes_formula():
    sys.path.insert(0, ROOT)
    import bench

    class S:
        nnz, nloc, ncopies, ngamma = 14581760, 2244608, 291483, 144027

    # 12 nnz + 4 (nloc+1) + 16 nloc + 4 ncopies + 4 (ngamma+1)
    assert bench.spmv_algorithmic_bytes(S) == 221615328


def test_reference_arm_line(capsys, monkeypatch):
    """Rank 0 of the reference arm: one JSON line with the contract's keys,
    a complete FP64 oracle solve of the 128^3 system to 1e-8 timed on the
    host cores (about 8 s here), the headline's workload and unit."""
    import json

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is False and d["dtype"] == "f64"
    assert d["config"]["workload"] == "fv3d_7pt_128^3_kappa=exp(N(0,1))_4x4x4_subdomains"
    assert d["config"]["mode"] == "fp64" and d["config"]["rtol"] == 1e-8
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert abs(cb["iters"] - 1055) <= 0.03 * 1055 and cb["true_relres"] <= 1.01e-8
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
