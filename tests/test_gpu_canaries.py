"""Canary-guarded output buffers: every output-writing entry point writes
inside its buffer and nowhere else.  Each output tensor is a view into a
larger buffer whose margins hold a sentinel; after the call (and a device
synchronise) the margins must be unchanged.  Covers the full cube, the folded
planes and Eq. (dft) in both layouts, the error bound and the per-bin
relative bound, the exported collapse sums, the monopole and cylindrical
binnings, the gridding outputs, the general and per-channel sampling plans,
and the allocation-free counts."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GUARD = 4096  # elements of sentinel on each side


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class Guarded:
    def __init__(self, shape, dtype, sentinel=-12345.0):
        torch = _torch()
        self.n = int(np.prod(shape))
        self.buf = torch.full((self.n + 2 * GUARD,), sentinel, dtype=dtype, device="cuda")
        self.sentinel = self.buf[:1].clone()
        self.t = self.buf[GUARD:GUARD + self.n].view(shape)

    def intact(self):
        torch = _torch()
        torch.cuda.synchronize()
        lo, hi = self.buf[:GUARD], self.buf[GUARD + self.n:]
        return bool(torch.equal(lo, self.sentinel.expand_as(lo)) and
                    torch.equal(hi, self.sentinel.expand_as(hi)))


@pytest.mark.parametrize("precision,multires", [(0, False), (1, True)])
def test_plan_outputs_stay_inside_their_buffers(precision, multires):
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    from oracle import monopole as mo
    nt, nc = 40, 10
    edges = synth.edges_log(5, 1.5, 19.0)
    plan = bs.Plan(nt, nc, edges, precision=precision, multires=multires, batch=2)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (1, 2)])
    plan.grid_load(torch.from_numpy(v).cuda())
    n2 = 2 * nc - 1
    f64 = torch.float64
    full = Guarded((2, plan.ntrip, nc, nc, nc), f64)
    plan.mabs(block=(1, 7, 2, 9, 0, 10), out_full=full.t, accumulate=True)
    dd = Guarded((2, plan.ntrip, n2, n2), f64)
    plan.mabs_delta(dd.t)
    dc = Guarded((2, plan.n_closable, n2, n2), f64)
    plan.mabs_delta_closable(dc.t)
    b3 = Guarded((2, plan.ntrip, nc, nc), f64)
    plan.bs3d(b3.t)
    b3c = Guarded((2, plan.n_closable, nc, nc), f64)
    plan.bs3d_closable(b3c.t)
    checks = [full, dd, dc, b3, b3c]
    bound = Guarded((2, plan.ntrip), f64)
    rel = Guarded((2, plan.n_closable, n2, n2), f64)
    plan._check(plan._L.bs_mabs_error_bound(plan._h, bs._dptr(bound.t), bs._dptr(dc.t), 1,
                                            bs._dptr(rel.t), None))
    checks += [bound, rel]
    sums = Guarded((2, plan.ntrip, n2, n2), f64)
    nnu = np.zeros((n2, n2), np.int64)
    plan._check(plan._L.bs_delta_export(plan._h, bs._dptr(sums.t),
                                        nnu.ctypes.data_as(bs.ctypes.c_void_p), None))
    checks.append(sums)
    kperp = 2 * np.pi * plan.ring_umean()
    kpar = mo.kpar_axis(nc)
    k1e = np.geomspace(0.5 * kperp.min(), 2.0 * np.sqrt(kperp.max() ** 2 + 4 * kpar.max() ** 2), 7)
    ms = Guarded((2, 6, 5, 5), f64)
    mc = Guarded((6, 5, 5), torch.int64, sentinel=-7)
    e = np.ascontiguousarray(k1e, dtype=np.float64)
    kp = np.ascontiguousarray(kperp, dtype=np.float64)
    kz = np.ascontiguousarray(kpar, dtype=np.float64)
    P = bs.ctypes.c_void_p
    plan._check(plan._L.bs_bs_monopole(plan._h, bs._dptr(b3c.t), kp.ctypes.data_as(P),
                                       kz.ctypes.data_as(P), e.ctypes.data_as(P), 6, 5, 5,
                                       bs.ctypes.c_double(0), bs.ctypes.c_double(0),
                                       bs.ctypes.c_double(0), bs._dptr(ms.t), bs._dptr(mc.t), None))
    checks += [ms, mc]
    ke = np.ascontiguousarray(np.linspace(-0.8 * kpar.max(), 0.8 * kpar.max(), 9))
    cs = Guarded((2, plan.n_closable, 8, 8), f64)
    cc = Guarded((8, 8), torch.int64, sentinel=-7)
    plan._check(plan._L.bs_bs_cylindrical(plan._h, bs._dptr(b3c.t), kz.ctypes.data_as(P),
                                          ke.ctypes.data_as(P), 8, bs._dptr(cs.t), bs._dptr(cc.t),
                                          None))
    checks += [cs, cc]
    for k, g in enumerate(checks):
        assert g.intact(), k
    plan.close()


def test_gridding_general_chans_and_noalloc_outputs_stay_inside():
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc = 32, 6
    edges = synth.edges_linear(4, 14)
    plan = bs.Plan(nt, nc, edges)
    nbl = 500
    r = np.random.default_rng(3)
    uv = torch.from_numpy(r.uniform(-15, 15, size=(nbl, 2))).cuda()
    vis = torch.from_numpy((r.normal(size=(nbl, nc)) + 1j * r.normal(size=(nbl, nc))).astype(
        np.complex64)).cuda()
    vg = Guarded((nc, nt, nt), torch.complex64, sentinel=-12345.0)
    ng = Guarded((nc, nt, nt), torch.float32)
    plan._check(plan._L.bs_grid_visibilities(plan._h, bs._dptr(uv), bs._dptr(vis), None,
                                             bs.ctypes.c_int64(nbl), nc, 1, 0, bs._dptr(vg.t),
                                             bs._dptr(ng.t), None))
    assert vg.intact() and ng.intact()
    plan.close()
    g = bs.Plan(nt, nc, edges, general=True)
    gv = r.normal(size=(1, nc, nt, nt)) + 1j * r.normal(size=(1, nc, nt, nt))
    g.grid_load(torch.from_numpy(gv.astype(np.complex64)).cuda())
    full = Guarded((1, g.ntrip, nc, nc, nc), torch.complex128)
    g.mabs(out_full=full.t, accumulate=True)
    dd = Guarded((1, g.ntrip, 2 * nc - 1, 2 * nc - 1), torch.complex128)
    g.mabs_delta(dd.t)
    b3 = Guarded((1, g.n_closable, nc, nc), torch.complex128)
    g.bs3d_closable(b3.t)
    assert full.intact() and dd.intact() and b3.intact()
    g.close()
    c = bs.Plan(nt, nc, edges, chan_sampling=True)
    occ = np.ones((nc, nt, nt), np.float32)
    c.grid_load(torch.from_numpy(synth.sky_visibilities(nt, nc, seed=5)[None]).cuda(),
                ngrid=torch.from_numpy(occ).cuda())
    full = Guarded((1, c.ntrip, nc, nc, nc), torch.float64)
    c.mabs(out_full=full.t, accumulate=True)
    b3 = Guarded((1, c.ntrip, nc, nc), torch.float64)
    c.bs3d(b3.t)
    assert full.intact() and b3.intact()
    c.close()
    tri = Guarded((20,), torch.int64, sentinel=-7)
    bs.counts_noalloc(nt, edges, tri.t)
    assert tri.intact()
