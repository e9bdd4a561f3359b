"""The benchmark's command-line contract, checked on the CPU without running a
benchmark: the flags the launcher passes exist, the reference arm is offered,
and a warm-up below 3 steps is refused."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=120)


def test_help_lists_the_contract_flags():
    r = _run("--help")
    assert r.returncode == 0
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--split", "--workload"):
        assert flag in r.stdout
    assert "reference" in r.stdout


def test_warmup_below_three_is_refused():
    r = _run("--steps", "1", "--warmup", "2")
    assert r.returncode != 0
    assert "--warmup must be >= 3" in r.stderr
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "1")
    assert r.returncode != 0
