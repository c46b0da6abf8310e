"""The benchmark's reference arm (the FP64 CPU oracle, timed on the host)
prints one JSON line with the keys the benchmark contract asks for; it runs
on the CPU, so it is checked here on the tiny workload.  The roofline's FLOP
count of a channel-symmetric cube is checked against a brute-force count."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "tiny", "--steps", "2", "--warmup", "1", "--cpu-seconds", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "mabs_bin_triple_x_channel_evals_per_s"
    assert d["unit"] == "evals/s" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "evals/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("tiny")


def test_contracted_flops_count_one_ordering_of_repeated_rings():
    """The roofline's FLOP count of a channel-symmetric cube: brute-force count of
    the channel triples contracted (nu1 <= nu2 for (i, i, l), nu2 <= nu3 for
    (i, j, j), i < j, every triple otherwise) against bench.contracted_flops."""
    import itertools

    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    nb, n = 3, 5
    trips = [(i, j, l) for i in range(nb) for j in range(i, nb) for l in range(j, nb)]
    rng = np.random.default_rng(3)
    tri = rng.integers(0, 2, len(trips))
    sides = rng.choice([8, 12, 16], len(trips))
    want_sym = want_all = 0.0
    for k, (i, j, l) in enumerate(trips):
        if tri[k] == 0:
            continue
        for a, b, c in itertools.product(range(n), repeat=3):
            f = 2.0 * sides[k] ** 2
            want_all += f
            if (i == j and a > b) or (i < j == l and b > c):
                continue
            want_sym += f
    assert bench.contracted_flops(tri, sides, nb, (n, n, n), False) == want_all
    assert bench.contracted_flops(tri, sides, nb, (n, n, n), True) == want_sym


def test_batched_monte_carlo_shapes_follow_the_configuration():
    """The batched Monte Carlo workload draws its realisation shapes inside the
    configuration's ranges (grids 128^2, 256^2 or 512^2; 384-768 channels,
    each a 2^a 3^b 5^c length the sky generator's FFTs take; 12-24 log
    rings), reproducibly by seed; the candidate channel blocks hold equal
    numbers of channel triples and fit the tiles' 32 x 16 pair rectangle."""
    sys.path.insert(0, ROOT)
    import bench
    shapes = bench.cfg4_shapes()
    assert shapes == bench.cfg4_shapes() and len(shapes) == 8
    assert bench.cfg4_shapes(seed=4001) != shapes
    for nt, nc, nb in bench.cfg4_shapes(n=200):
        assert nt in (128, 256, 512) and 384 <= nc <= 768 and 12 <= nb <= 24
        m = nc
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        assert m == 1, nc
    assert len({nt for nt, _, _ in bench.cfg4_shapes(n=200)}) == 3
    for b in (32, 64):
        blocks = bench.cfg4_block_shapes(b)
        assert all(x * y * z == b ** 3 for x, y, z in blocks)
        assert all(x % 32 == 0 and y % 16 == 0 for x, y, _ in blocks)
