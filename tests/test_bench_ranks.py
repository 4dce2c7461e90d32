"""The benchmark's multi-rank path on CPU: two gloo ranks read their
rank, world size and rendezvous from the environment the way torchrun sets
it, the whole-job figures are the slowest rank's time and the sum of all
ranks' updates, and the oracle arm runs on rank 0 alone."""
import argparse
import contextlib
import io
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, what):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        if what == "batch":
            # each rank advances its share of 256 independent instances;
            # the whole job is the sum of the shares' work over the
            # slowest rank's time
            r, ws, local, dist = bench.dist_setup()
            mine = bench.partition(256, r, ws)
            res = {"rank": r, "mine": mine,
                   "fig": bench.over_ranks(dist, 10.0 + 5.0 * r, sum(i + 1 for i in mine))}
            dist.barrier()
            print(json.dumps(res))
        elif what == "reduce":
            r, ws, local, dist = bench.dist_setup()
            res = {"rank": r, "ws": ws, "local": local,
                   "fig": bench.over_ranks(dist, 10.0 + 5.0 * r, 100 * (r + 1))}
            dist.barrier()
            print(json.dumps(res))
        else:
            args = argparse.Namespace(workload="shock_tube", mode="multi", steps=2, warmup=3)
            bench.run_reference(args)
    import torch.distributed as d
    if d.is_initialized():
        d.barrier()
        d.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(buf.getvalue())


def _spawn(tmp_path, what, world=2):
    port = _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path), what), nprocs=world, join=True)
    outs = []
    for r in range(world):
        with open(tmp_path / f"rank{r}.txt") as f:
            outs.append(f.read())
    return outs


def test_two_ranks_report_max_time_and_summed_updates(tmp_path):
    outs = _spawn(tmp_path, "reduce")
    for r, text in enumerate(outs):
        res = json.loads(text)
        assert (res["rank"], res["ws"], res["local"]) == (r, 2, r)
        assert res["fig"] == [15.0, 300.0]


def test_oracle_arm_runs_on_rank_zero_only(tmp_path):
    outs = _spawn(tmp_path, "reference")
    assert outs[1] == ""
    lines = [ln for ln in outs[0].splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["config"]["workload"] and line["steps"] == 2 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["ms_per_step"] > 0


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.over_ranks(None, 7.5, 12) == (7.5, 12.0)


def test_two_ranks_split_the_batch_and_merge_its_work(tmp_path):
    outs = [json.loads(t) for t in _spawn(tmp_path, "batch")]
    assert outs[0]["mine"] + outs[1]["mine"] == list(range(256))
    assert len(outs[0]["mine"]) == len(outs[1]["mine"]) == 128
    for res in outs:
        assert res["fig"] == [15.0, float(256 * 257 // 2)]
