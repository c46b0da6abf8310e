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


CHILD_ALLOC = textwrap.dedent("""
    import sys, numpy as np, torch
    sys.path.insert(0, ROOT)
    import paper_2506_10526_gb300 as bs, synth, oracle
    edges = synth.edges_linear(4, 16)
    vis_h = synth.sky_visibilities(32, 4, seed=3)
    vis = torch.from_numpy(vis_h[None]).cuda()
    # the plan's own workspace allocation fails cleanly
    p = bs.Plan(32, 4, edges, torch_workspace=False)
    try:
        p.grid_load(vis)
        print("WS_LOADED")
    except bs.BsError as e:
        print("WS_STATUS", e.status)
    p.close()
    # the other allocations
    for name, make in (("MC", lambda: bs.Ensemble([dict(nt=32, nchan=4, edges=edges, batch=1)])),
                       ("SKY", lambda: bs.SkyGenerator(32, 4)),
                       ("MLP", lambda: bs.Surrogate(bs.MLP_FEATURES, 32, seed=1))):
        try:
            make().close()
            print(name, "CREATED")
        except bs.BsError as e:
            print(name, "STATUS", e.status)
    g = bs.Plan(32, 4, edges, general=True)
    g.grid_load(vis)
    try:
        full = torch.empty((1, g.ntrip, 4, 4, 4), dtype=torch.complex128, device="cuda")
        g.mabs(out_full=full)
        print("SCRATCH_OK")
    except bs.BsError as e:
        print("SCRATCH_STATUS", e.status)
    g.close()
    # a plan on a caller-owned (torch) workspace still computes correctly
    q = bs.Plan(32, 4, edges)
    q.grid_load(vis)
    full = torch.empty((1, q.ntrip, 4, 4, 4), dtype=torch.float64, device="cuda")
    q.mabs(out_full=full)
    torch.cuda.synchronize()
    ref = oracle.mabs_full(vis_h.astype(np.complex128), edges)["B"].real
    got = full[0].cpu().numpy()
    ok = ~np.isnan(ref)
    print("AFTER", bool(np.array_equal(np.isnan(got), ~ok)),
          float(np.abs(got[ok] - ref[ok]).max() / np.abs(ref[ok]).max()))
    q.close()
""").replace("ROOT", repr(ROOT))


def test_injected_allocation_failures_are_reported_cleanly():
    """BS_INJECT_FAIL on the device allocations: the plan workspace, the Monte
    Carlo buffers, the sky generator, the surrogate and the general plans'
    scratch each fail with BS_ERR_OOM and nothing else; a plan on a torch
    workspace in the same process then computes correctly."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ)
    env["BS_INJECT_FAIL"] = "workspace_alloc,mc_alloc,sky_alloc,mlp_alloc,scratch_alloc"
    r = subprocess.run([sys.executable, "-c", CHILD_ALLOC], capture_output=True, text=True,
                       timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    out = r.stdout
    for tag in ("WS_STATUS 4", "MC STATUS 4", "SKY STATUS 4", "MLP STATUS 4", "SCRATCH_STATUS 4"):
        assert tag in out, out
    line = [l for l in out.splitlines() if l.startswith("AFTER")][0].split()
    assert line[1] == "True" and float(line[2]) < 1e-5, out
