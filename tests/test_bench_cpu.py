"""bench.py on the CPU: the step runs on one GPU, so a launch that asks for
more (several ranks or --gpus above 1) is refused before any GPU work, and
the reference arm runs on rank 0 only."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                          text=True, env=env, timeout=300)


def test_several_ranks_are_refused():
    r = run_bench(["--gpus", "2", "--steps", "3", "--warmup", "3"], {"WORLD_SIZE": "2"})
    assert r.returncode != 0
    assert "one GPU" in r.stderr


def test_more_gpus_on_one_rank_is_refused():
    r = run_bench(["--gpus", "4"], {})
    assert r.returncode != 0
    assert "one GPU" in r.stderr


def test_reference_arm_other_ranks_exit_without_work():
    r = run_bench(["--impl", "reference", "--gpus", "2"], {"WORLD_SIZE": "2", "RANK": "1"})
    assert r.returncode == 0
    assert r.stdout.strip() == ""
