"""The benchmark's multi-rank host logic on CPU: two gloo ranks (one process
per rank, as torchrun launches them) initialise the process group from the
environment, agree on the maximum of their per-rank times, meet at the
barrier, and shard the work as independent replicas (rank r draws the pair
of seed + r, so no data-path collective is needed)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench

    r, w, local = bench.dist_info()
    assert (r, w, local) == (rank, world, rank)
    dist = bench.dist_init(w, use_cuda=False)
    bench.barrier(dist)
    # per-rank "times": the job's time is the slowest rank's
    t = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)
    # replica sharding: each rank its own seed, no exchange of points
    A, B = bench.make_pair(seed=3 + rank, n=64)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{t} {float(A[0, 0])}\n")
    bench.barrier(dist)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_agree_on_the_max_time(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    vals = [open(os.path.join(tmp_path, f"rank{r}.txt")).read().split() for r in range(2)]
    assert float(vals[0][0]) == float(vals[1][0]) == 15.0
    # the two replicas drew different pairs
    assert vals[0][1] != vals[1][1]


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        seed = 0
        n = 1000
        warmup = 3
        steps = 1

    bench.reference_arm(Args())
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_a_small_pair(monkeypatch, capsys):
    # rank 0 times the oracle and prints one JSON line with the contract's keys
    import json

    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class Args:
        seed = 0
        n = 20_000
        warmup = 3
        steps = 1

    bench.reference_arm(Args())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "20,000" in line["config"]["workload"]
    # the step time is what was measured; the full-pair figure is labelled as extrapolated
    assert line["extrapolated"] is True and line["cpu_baseline"]["extrapolated"] is True
    assert line["ms_per_step"] <= line["ms_per_full_pair_extrapolated"]
    assert set(line["scale_factors"]) == {"covariance", "subset_hd"}
