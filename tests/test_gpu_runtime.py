"""Runtime hygiene around the build, on the GPU: kernel attributes (dynamic
shared memory above 48 KB) are set per CUDA context and thread-safely, so
many host threads may start building at once, and a process may build on
every visible device."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu

_SCRIPT = r"""
import sys, threading
sys.path.insert(0, {root!r})
import numpy as np, torch
import gen, oracle
import paper_1610_03007_gb300 as gbsa
lib = gbsa.load()
devices = {devices}
texts = [gen.text(("zipf_repeats", "markov", "dna")[k % 3], 700 + k, 150000 + 997 * k)
         for k in range(16)]
want = [oracle.get().pd_sa(t)[0] for t in texts]
errors = []
start = threading.Barrier(16)

def work(k):
    try:
        dev = devices[k % len(devices)]
        torch.cuda.set_device(dev)
        s = torch.cuda.Stream(device=dev)
        d = torch.from_numpy(texts[k]).to(f"cuda:{{dev}}")
        n = d.numel()
        ws = torch.empty(int(lib.sa_workspace_bytes(n)), dtype=torch.uint8, device=d.device)
        torch.cuda.synchronize(dev)
        start.wait()
        for rep in range(2):
            out = torch.full((n,), -1, dtype=torch.int32, device=d.device)
            rc = lib.sa_build_ex(d.data_ptr(), n, out.data_ptr(), None, ws.data_ptr(),
                                 ws.numel(), None, None, s.cuda_stream)
            s.synchronize()
            if rc != 0:
                errors.append((k, rep, "rc", rc))
            elif not np.array_equal(out.cpu().numpy().view(np.uint32), want[k]):
                errors.append((k, rep, "differs"))
    except Exception as e:
        errors.append((k, repr(e)))

th = [threading.Thread(target=work, args=(k,)) for k in range(16)]
for t in th: t.start()
for t in th: t.join()
print("ERRORS", errors)
sys.exit(1 if errors else 0)
"""


def _run(devices):
    import __graft_entry__
    __graft_entry__.build()
    code = _SCRIPT.format(root=ROOT, devices=devices)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


def test_sixteen_threads_build_at_once_in_a_fresh_process():
    """The first builds of a fresh process run from 16 threads at once, two
    each, on the current device: every SA equals the oracle's."""
    _run([0])


def test_one_build_per_device_in_one_process():
    """One process builds on every visible device (threads spread over
    them); skipped with fewer than two GPUs."""
    import torch
    n = torch.cuda.device_count()
    if n < 2:
        pytest.skip(f"{n} GPU visible: the per-device attribute path needs two")
    _run(list(range(n)))
