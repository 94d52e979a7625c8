"""Host-side fault injection (no GPU fault): MT_FAULT_INJECT=alloc:<n> makes the
n-th device allocation fail; scene creation must return MT_ERR_OUT_OF_MEMORY
and release everything it had allocated."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, torch
sys.path.insert(0, {root!r})
from paper_2510_25660_gb300 import api, scenes
api.load()
torch.cuda.init()
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
try:
    api.Scene(scenes.cornell_box())
    print("NOFAIL")
except api.MtError as e:
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    print("STATUS", e.status, "LEAK", free0 - free1)
"""


@pytest.mark.parametrize("n", [1, 3, 9, 20])
def test_injected_allocation_failure(n):
    from gpu_util import build_and_load
    build_and_load()
    env = dict(os.environ, MT_FAULT_INJECT=f"alloc:{n}")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    out = r.stdout.split()
    assert out[0] == "STATUS", r.stdout
    assert int(out[1]) == 2  # MT_ERR_OUT_OF_MEMORY
    assert abs(int(out[3])) < (4 << 20), r.stdout  # nothing kept (allocator granularity aside)
