"""bench.py with more than one rank, on CPU ranks over gloo (world size 2).

The solver does not shard: with N ranks each rank builds and solves its own
independent problem (replicas, weak scaling), so the only cross-rank steps are
the barriers, the maximum of the ranks' timings, the whole-job rate over the
slowest rank, and rank 0 alone printing the JSON line.  Those steps run here
with CPU ranks; each rank's device work is the same as at one rank.
"""
import json
import os
import socket
import subprocess
import sys
import textwrap
from pathlib import Path

import numpy as np
import pytest

from paper_1307_2665_gb300.build import build

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, cwd, timeout=300):
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONPATH=str(ROOT))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), *args]
    return subprocess.run(cmd, cwd=cwd, env=env, capture_output=True, text=True, timeout=timeout)


RANK_SCRIPT = textwrap.dedent("""
    import json, os, sys
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, {root!r})
    import bench
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    # timings that differ by rank: every rank must see the slowest one
    t_build, t_solve = bench.max_over_ranks([10.0 + rank, 5.0 - rank], dist, "cpu")
    W = bench.make_workload("convdiff64", 2, rank)
    out = {{"rank": rank, "world": world, "t": [t_build, t_solve],
           "rate": bench.job_rate(world, W.dof, 3, t_build + t_solve)}}
    np.save(os.path.join({out!r}, f"f{{rank}}.npy"), W.probs[0]["f"])
    np.save(os.path.join({out!r}, f"c{{rank}}.npy"), W.probs[0]["coeffs"]["c1"])
    with open(os.path.join({out!r}, f"r{{rank}}.json"), "w") as fh:
        json.dump(out, fh)
    dist.barrier()
    dist.destroy_process_group()
""")


def test_two_ranks_share_the_slowest_time_and_solve_distinct_data(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(RANK_SCRIPT.format(root=str(ROOT), out=str(tmp_path)))
    r = _torchrun([str(script)], cwd=tmp_path)
    assert r.returncode == 0, r.stdout + r.stderr
    res = [json.loads((tmp_path / f"r{k}.json").read_text()) for k in range(2)]
    for k, d in enumerate(res):
        assert d["rank"] == k and d["world"] == 2
        assert d["t"] == [11.0, 5.0]  # max over ranks of (10 + r, 5 - r)
        # 2 ranks x (2 x 2 leaves x 16^2 nodes) x 3 steps over 16 ms
        assert d["rate"] == pytest.approx(2 * 1024 * 3 / 0.016)
    f0, f1 = (np.load(tmp_path / f"f{k}.npy") for k in range(2))
    c0, c1 = (np.load(tmp_path / f"c{k}.npy") for k in range(2))
    assert f0.shape == f1.shape == (16, 2 * (2 + 2) * 14)
    assert not np.allclose(f0, f1)  # each rank its own boundary data (seeds 16 r + 0..15)
    assert np.array_equal(c0, c1)  # on the same coefficient field


def test_max_over_ranks_is_the_identity_on_one_rank():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
    assert bench.job_rate(1, 100, 2, 1000.0) == 200.0


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    """`bench.py --impl reference` launched as two ranks: rank 0 times the
    oracle on its bounded sample and prints one JSON line, rank 1 exits 0
    without work."""
    r = _torchrun([str(ROOT / "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                   "--warmup", "0", "--ref-leaves", "2"], cwd=tmp_path)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["unit"] == "DOF/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # the same workload name as the native arm's line
    sys.path.insert(0, str(ROOT))
    import bench
    assert line["config"]["workload"] == bench.describe_workload("helmholtz256", 0)[0]["workload"]
