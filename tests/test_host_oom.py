"""A host allocation failure during space creation becomes FE_ERR_OOM: no C++
exception crosses the C ABI and the process does not abort, also when the
failure happens on one of the setup's worker threads or when those threads
cannot be started. A child process caps its address space (RLIMIT_AS) a little
above what it already uses, asks for a host-only space whose setup needs far
more, gets FE_ERR_OOM, lifts the cap and then creates a space normally; under
a cap too tight for the worker threads' stacks a small space is still created
(or refused with FE_ERR_OOM), never aborted."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import resource, sys
sys.path.insert(0, sys.argv[1])
from paper_1708_01773_gb300 import feasm, inputs
feasm.lib()
big = inputs.small_problem((36, 36, 36), 2, 1, seed=1)      # ~3.4e8 contributions
small = inputs.small_problem((3, 3, 3), 1, 1, seed=2)
def vm_bytes():
    for line in open("/proc/self/status"):
        if line.startswith("VmSize:"):
            return int(line.split()[1]) * 1024
soft, hard = resource.getrlimit(resource.RLIMIT_AS)
resource.setrlimit(resource.RLIMIT_AS, (vm_bytes() + (192 << 20), hard))
try:
    feasm.FESpace(big, host_only=True)
    result = "created"
except feasm.FEError as e:
    result = "code %d" % e.code
resource.setrlimit(resource.RLIMIT_AS, (soft, hard))
sp = feasm.FESpace(small, host_only=True)
# a cap that leaves room for the setup's arrays but not for the 8 MB stacks of
# its worker threads: the chunks run on the calling thread instead
mid = inputs.small_problem((8, 8, 8), 1, 1, seed=3)
resource.setrlimit(resource.RLIMIT_AS, (vm_bytes() + (6 << 20), hard))
try:
    result2 = "created %d" % feasm.FESpace(mid, host_only=True).n_dofs
except feasm.FEError as e:
    result2 = "code %d" % e.code
resource.setrlimit(resource.RLIMIT_AS, (soft, hard))
print(result, "then", sp.n_dofs, "|", result2)
"""


@pytest.mark.skipif(not os.path.exists("/proc/self/status"), reason="needs /proc")
def test_host_setup_out_of_memory_is_a_status_code():
    from paper_1708_01773_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    first, second = r.stdout.strip().split("|")
    assert first.split() == ["code", "-3", "then", "192"], r.stdout
    assert second.split() in (["created", "2187"], ["code", "-3"]), r.stdout
