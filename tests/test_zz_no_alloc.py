"""dbscan_run_static: the entry point that allocates nothing.

Some callers cannot call cudaMalloc (code inside another framework's memory
pool, hosts that forbid device allocation after start-up); dbscan_run_static
serves them from a fixed device array of the library.  These tests call it
through the C ABI and check its core flags and labels against dbscan_run and
against the CPU oracle on the same input, on two calls in a row (the array
keeps the previous call's contents, so the second call shows that the run
clears what it must), and once in a fresh process whose first call (the one
that sets the array up) runs on a non-blocking stream.
This file is named to be collected last.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1912_06255_gb300 import DBSCAN, _lib, build, synth  # noqa: E402


def _static(lib, X, eps, mp):
    n, d = X.shape
    core = torch.empty(n, dtype=torch.uint8, device="cuda")
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    dtype = _lib.F32 if X.dtype == torch.float32 else _lib.F64
    st = lib.dbscan_run_static(X.data_ptr(), n, d, dtype, float(eps), int(mp), core.data_ptr(),
                               labels.data_ptr(), s.cuda_stream)
    assert st == 0, _lib.STATUS.get(st, st)
    torch.cuda.synchronize()
    return core.cpu().numpy(), labels.cpu().numpy()


def test_static_entry_matches_dbscan_run_twice():
    build.build()
    lib = _lib.load()
    cases = [
        (synth.random_small(901, 12000, 3, dtype=np.float32), 0.3, 8),
        (synth.random_small(902, 16384, 2, dtype=np.float64), 0.2, 5),
    ]
    for X, eps, mp in cases:
        t = torch.from_numpy(X).cuda()
        ref = DBSCAN(len(X), X.shape[1]).run(t, eps, mp, border=False)
        ref_core, ref_labels = ref.core.cpu().numpy(), ref.labels.cpu().numpy()
        exp = oracle.dbscan(X, eps, mp)
        assert np.array_equal(ref_core, exp[0]) and np.array_equal(ref_labels, exp[1])
        for _ in range(2):
            core, labels = _static(lib, t, eps, mp)
            assert np.array_equal(core, ref_core)
            assert np.array_equal(labels, ref_labels)


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
import oracle
from paper_1912_06255_gb300 import _lib, synth
lib = _lib.load()
s = torch.cuda.Stream()  # a pooled stream: created non-blocking
X = synth.random_small(903, 9000, 3, dtype=np.float32)
with torch.cuda.stream(s):
    t = torch.from_numpy(X).to("cuda", non_blocking=False)
    core = torch.empty(len(X), dtype=torch.uint8, device="cuda")
    labels = torch.empty(len(X), dtype=torch.int32, device="cuda")
s.synchronize()
exp = oracle.dbscan(X, 0.3, 8)
for k in range(2):
    core.fill_(7)
    labels.fill_(-7)
    torch.cuda.synchronize()
    st = lib.dbscan_run_static(t.data_ptr(), len(X), 3, _lib.F32, 0.3, 8, core.data_ptr(), labels.data_ptr(),
                               s.cuda_stream)
    assert st == 0, _lib.STATUS.get(st, st)
    s.synchronize()
    assert np.array_equal(core.cpu().numpy(), exp[0]), k
    assert np.array_equal(labels.cpu().numpy(), exp[1]), k
print("static entry ok")
"""


def test_static_entry_fresh_process_nonblocking_stream():
    """The set-up call on a non-blocking stream in a new process, then a second
    call, both against the oracle."""
    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=root)], capture_output=True, text=True,
                       timeout=600, cwd=root)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "static entry ok" in r.stdout


def test_static_entry_rejects_oversize():
    lib = _lib.load()
    X = torch.zeros((16385, 3), device="cuda")
    out8 = torch.empty(16385, dtype=torch.uint8, device="cuda")
    out32 = torch.empty(16385, dtype=torch.int32, device="cuda")
    st = lib.dbscan_run_static(X.data_ptr(), 16385, 3, _lib.F32, 1.0, 3, out8.data_ptr(), out32.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 5  # DBSCAN_ERR_CAPACITY
    st = lib.dbscan_run_static(X.data_ptr(), 100, 4, _lib.F32, 1.0, 3, out8.data_ptr(), out32.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 2  # DBSCAN_ERR_UNSUPPORTED_DIM
