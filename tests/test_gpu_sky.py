"""GPU Monte Carlo sky generator (bs_sky_*) against the double-precision
restatement of the same definition (synth.philox_sky_visibilities): same
Philox counters, same recipe, element by element; plus the batching rules
(odd batch, realisation offsets) and an ensemble driven by it."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 2e-5  # of max |V|: FP32 Box-Muller and FP32 FFTs of a few thousand points


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("nt,nc,batch,seed,r0,f_ng", [
    (32, 12, 3, 77, 5, 0.5),      # odd batch: the last pair has one realisation
    (48, 10, 2, 1, 0, 0.5),       # radices 3 and 5
    (40, 1, 4, 2**40 + 3, 2**33, 1.0),  # one channel; 64-bit seed and realisation words
    (64, 16, 2, 9, 100, 0.0),     # Gaussian sky
    # register-FFT line passes: x / y lines of 128 and 256, z lines of 256,
    # 384, 768 and of the odd channel counts 540, 675, 729, 750
    (128, 4, 2, 5, 7, 0.5),
    (256, 2, 2, 6, 8, 0.5),
    (8, 256, 2, 11, 1, 0.5),
    (8, 384, 1, 12, 2, 0.5),
    (8, 768, 2, 13, 3, 0.5),
    (8, 540, 2, 14, 4, 0.5),
    (8, 675, 2, 15, 5, 0.5),
    (8, 729, 1, 16, 6, 0.5),
    (8, 750, 2, 17, 7, 0.5),
])
def test_generator_matches_reference(nt, nc, batch, seed, r0, f_ng):
    _torch()
    import paper_2506_10526_gb300 as bs
    gen = bs.SkyGenerator(nt, nc, slope=-2.0, sigma=0.5, f_ng=f_ng, max_batch=batch)
    v = gen.generate(seed, r0).cpu().numpy()
    gen.close()
    for b in range(batch):
        ref = synth.philox_sky_visibilities(nt, nc, seed, r0 + b, f_ng=f_ng)
        err = np.abs(v[b] - ref).max() / np.abs(ref).max()
        assert err < TOL, (b, err)


def test_batches_are_slices_of_one_sequence():
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    gen = bs.SkyGenerator(32, 8, max_batch=6)
    a = gen.generate(3, 10, batch=6)
    b = gen.generate(3, 12, batch=2)
    torch.cuda.synchronize()
    assert torch.equal(a[2:4], b)  # same pairs of realisations: bit-identical
    c = gen.generate(3, 13, batch=1)
    ref = synth.philox_sky_visibilities(32, 8, 3, 13)
    assert np.abs(c[0].cpu().numpy() - ref).max() < TOL * np.abs(ref).max()
    with pytest.raises(bs.BsError):
        gen.generate(3, 0, batch=7)
    gen.close()


def test_rejects_unsupported_sizes():
    _torch()
    import paper_2506_10526_gb300 as bs
    with pytest.raises(bs.BsError):
        bs.SkyGenerator(14, 8)   # 14 = 2 * 7
    with pytest.raises(bs.BsError):
        bs.SkyGenerator(32, 7)
    with pytest.raises(bs.BsError):
        bs.SkyGenerator(33, 8)   # odd nt


def test_ensemble_on_generated_sky_matches_host_sky():
    """Monte Carlo statistics with the sky drawn on the GPU equal those with
    the same realisations drawn on the host (FP64) and copied in."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, b = 32, 8, 4
    edges = list(synth.edges_linear(5, 16))
    spec = dict(nt=nt, nchan=nc, edges=edges, batch=b)
    ens = bs.Ensemble([spec, spec])
    gen = bs.SkyGenerator(nt, nc, max_batch=b)
    buf_gpu = torch.empty((b, nc, nt, nt), dtype=torch.complex64, device="cuda")
    buf_host = torch.empty_like(buf_gpu)
    ens.set_input(0, buf_gpu)
    ens.set_input(1, buf_host)
    for step in range(3):
        gen.generate(21, step * b, out=buf_gpu)
        v = np.stack([synth.philox_sky_visibilities(nt, nc, 21, step * b + k) for k in range(b)])
        buf_host.copy_(torch.from_numpy(v.astype(np.complex64)))
        ens.run(use_graph=False)
    m0, v0, n0 = ens.stats(0, 1)
    m1, v1, n1 = ens.stats(1, 1)
    assert n0 == n1 == 12
    ok = np.isfinite(m1)
    assert np.array_equal(np.isfinite(m0), ok)
    assert np.abs(m0[ok] - m1[ok]).max() <= 1e-3 * np.abs(m1[ok]).max()
    assert np.abs(v0[ok] - v1[ok]).max() <= 2e-3 * np.abs(v1[ok]).max()
    gen.close()
    ens.close()


def test_generator_full_box_timing():
    """A 256^2 x 768-channel box (the MWA-like workload): Hermitian output,
    variance of the sky plane sums, and the time per realisation."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, b = 256, 768, 2
    gen = bs.SkyGenerator(nt, nc, max_batch=b)
    out = torch.empty((b, nc, nt, nt), dtype=torch.complex64, device="cuda")
    for _ in range(2):
        gen.generate(5, 0, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 5
    for r in range(reps):
        gen.generate(5, 2 * r, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (reps * b)
    print(f"sky generator: {ms:.3f} ms per 256^2 x 768 realisation")
    inner = out[:, :, 1:, 1:]
    herm = (inner - torch.conj(torch.flip(inner, dims=(2, 3)))).abs().max().item()
    assert herm <= 1e-5 * inner.abs().max().item()
    assert torch.isfinite(out).all()
    gen.close()
