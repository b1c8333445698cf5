"""Host-side logic of bench.py (no GPU): the aggregation over ranks that --gpus N uses, run as
two gloo ranks on CPU, and the reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r pretends its timed region took (r + 1) seconds; the job time is the slowest rank's
    t = bench.max_over_ranks(float(rank + 1), world)
    bench.barrier(world)
    q.put((rank, t, bench.aggregate_mlups(1_000_000, 10, t, world)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_cells():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]
    # 2 ranks x 1e6 cells x 10 steps in 2 s = 10 MLUPS whole-job
    assert out[0][2] == pytest.approx(10.0) and out[1][2] == pytest.approx(10.0)


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--steps", "3", "--warmup", "3",
                        "--ref-seconds", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["metric"].startswith("MLUPS") and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_bench_rejects_too_few_warmup_steps():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--warmup", "2"], capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode != 0 and "warmup" in r.stderr


@pytest.mark.parametrize("steps,want", [(20, 20), (10000, 20), (7, 0), (64, 64), (66, 22), (3, 0), (30, 30),
                                       (2, 2), (100, 20), (4096, 32)])
def test_headline_graph_steps(steps, want):
    """The headline's graph length: the whole timed region when --steps is even and at most 64,
    else the largest even divisor of --steps up to 32; 0 (direct launches) when none exists."""
    sys.path.insert(0, str(ROOT))
    import bench
    gs = bench.headline_graph_steps(steps)
    assert gs == want
    if gs:
        assert gs % 2 == 0 and steps % gs == 0 and (gs <= 32 or gs == steps)


def test_summary_rounding_keeps_significant_digits():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.sig(21688.43) == 21690.0
    assert bench.sig(0.000123456, 2) == 0.00012
    assert bench.sig(0.0) == 0.0 and bench.sig(None) is None
    assert bench.sig(float("inf")) == float("inf")


@pytest.mark.parametrize("warmup,want", [(3, 32), (5, 32), (50, 50), (51, 52), (64, 64)])
def test_leg_warmup_covers_a_whole_graph_and_is_even(warmup, want):
    """Legs other than the headline warm up for at least one whole 32-step graph and an even
    count, so that their timed regions start from a buffer whose graph is already captured."""
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.leg_warmup(warmup) == want


def test_bench_rejects_unknown_legs():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--legs", "surrogate,nope"], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode != 0 and "unknown legs" in r.stderr


def test_kernel_hash_ignores_comments_and_whitespace_but_not_code():
    """The profile's source hash: comments and whitespace runs do not change the stripped text,
    code and string literals do."""
    sys.path.insert(0, str(ROOT))
    import bench
    a = bench.strip_comments('int a = 1; // one\n/* two\n lines */ float b = "//x";')
    assert a == 'int a = 1; float b = "//x";'
    assert bench.strip_comments("int  a =\n 1;") == bench.strip_comments("int a = 1; /* c */")
    assert bench.strip_comments("int a = 1;") != bench.strip_comments("int a = 2;")
    assert bench.strip_comments("x = '/'; // c") == "x = '/';"
