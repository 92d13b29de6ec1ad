"""The strong-scaling launch (one molecule split over ranks, NCCL all-gather of the Q-vector
shares) end to end through bench.py under torchrun.  This pool gives one GPU per run, so it runs
as a group of one rank; the split itself is covered by the shard tests (several shards in turn on
one GPU) and by the gloo ranks of tests/test_dist_cpu.py."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("exact", [False, True])
def test_strong_launch_over_nccl_matches_unsharded(exact):
    """The FP64 shares all-gathered (within 1e-12 of the unsplit profile), or on deterministic
    contexts the exact shard sums all-reduced as limbs over NCCL (the unsplit profile bit for bit)."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "1",
           "--master-addr", "127.0.0.1", "--master-port", str(29563 + exact), "bench.py", "--scaling", "strong",
           "--steps", "2", "--warmup", "1"] + (["--exact"] if exact else [])
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [l for l in out.stdout.splitlines() if l.startswith("{")][-1]
    d = json.loads(line)
    assert d["scaling"] == "strong" and d["n_gpus"] == 1
    assert d["value"] > 0 and d["rel_diff_vs_unsharded"] <= 1e-12
    if exact:
        assert d["identical_to_unsharded"] and d["config"]["exact"]
