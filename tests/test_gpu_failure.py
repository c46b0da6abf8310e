"""Failure detection without a GPU fault: the tensor-core contraction bounds
every wait.  With BS_INJECT_MMA_STALL=1 the MMA thread waits on a barrier
nothing arrives at; after its (shortened, 50 ms) limit the kernel sets the
plan's error word, every role winds down, TMEM is freed, and the next
synchronising call returns BS_ERR_TIMEOUT.  The context stays usable: a
normal run in the same process afterwards matches the FP32 path.  Runs in a
child process so the environment switch cannot leak into other tests."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import os, sys, numpy as np, torch
    sys.path.insert(0, ROOT)
    import paper_2506_10526_gb300 as bs, synth
    vis = torch.from_numpy(synth.sky_visibilities(32, 4, seed=1)[None]).cuda()
    edges = synth.edges_linear(4, 16)
    out = torch.empty((1, 20, 7, 7), dtype=torch.float64, device="cuda")
    plan = bs.Plan(32, 4, edges, precision=bs.PREC_SPLIT_BF16)
    plan.grid_load(vis)
    os.environ["BS_INJECT_MMA_STALL"] = "1"
    plan.mabs()
    try:
        plan.mabs_delta(out)
        print("NO_TIMEOUT")
    except bs.BsError as e:
        print("STATUS", e.status)
    os.environ["BS_INJECT_MMA_STALL"] = "0"
    plan.grid_load(vis)
    plan.mabs()
    plan.mabs_delta(out)
    ref = bs.Plan(32, 4, edges)
    ref.grid_load(vis)
    ref.mabs()
    out2 = torch.empty_like(out)
    ref.mabs_delta(out2)
    torch.cuda.synchronize()
    a, b = out.cpu().numpy(), out2.cpu().numpy()
    ok = ~np.isnan(b)
    rel = np.abs(a[ok] - b[ok]).max() / np.abs(b[ok]).max()
    print("RECOVERED", rel < 1e-3, rel)
""").replace("ROOT", repr(ROOT))


def test_bounded_wait_timeout_is_reported_and_recoverable():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "STATUS 6" in r.stdout, r.stdout  # BS_ERR_TIMEOUT
    assert "RECOVERED True" in r.stdout, r.stdout
