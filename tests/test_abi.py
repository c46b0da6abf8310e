"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol that include/bs.h declares, and refuses cleanly (no CPU fallback)
when no sm_103a device is present.  No compute call runs here."""
import contextlib
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2506_10526_gb300 as bs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_10526_gb300 import build
    build.build()
    return bs.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "bs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bs_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_exported(lib):
    names = _declared()
    assert set(names) == set(bs.EXPORTS), names
    for n in names:
        assert hasattr(lib, n), n


def test_abi_version(lib):
    assert lib.bs_abi_version() == bs.ABI_VERSION == 13


def test_binding_constants_match_header():
    src = open(os.path.join(ROOT, "include", "bs.h")).read()
    assert int(re.search(r"#define BS_ABI_VERSION (\d+)", src).group(1)) == bs.ABI_VERSION
    assert int(re.search(r"#define BS_MLP_FEATURES (\d+)", src).group(1)) == bs.MLP_FEATURES


def test_desc_validation_and_no_device(lib):
    import torch
    edges = (ctypes.c_double * 3)(0.0, 2.0, 4.0)
    h = ctypes.c_void_p()
    bad = bs.PlanDesc(7, 4, 2, edges, 0, 0, 1, 1, 1, 1, 1, 0)  # odd nt
    assert lib.bs_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    assert b"nt" in lib.bs_last_error(None)
    desc_edges = (ctypes.c_double * 3)(0.0, 4.0, 2.0)  # not ascending
    bad = bs.PlanDesc(16, 4, 2, desc_edges, 0, 0, 1, 1, 1, 1, 1, 0)
    assert lib.bs_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = bs.PlanDesc(16, 4, 2, edges, 0, 3, 1, 1, 1, 1, 1, 0)  # no precision 3
    assert lib.bs_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    assert b"precision" in lib.bs_last_error(None)
    assert (bs.PREC_FP32, bs.PREC_SPLIT_BF16, bs.PREC_SPLIT_FP16) == (0, 1, 2)
    good = bs.PlanDesc(16, 4, 2, edges, 0, 0, 1, 1, 1, 1, 1, 0)
    st = lib.bs_plan_create(ctypes.byref(good), ctypes.byref(h))
    if not torch.cuda.is_available():
        assert st == 2  # BS_ERR_NO_DEVICE: no CPU fallback
        with pytest.raises(bs.BsError):
            bs.Plan(16, 4, [0.0, 2.0, 4.0])
    else:
        assert st == 0
        lib.bs_plan_destroy(h)


def test_null_handles(lib):
    assert lib.bs_plan_destroy(None) == 0
    assert lib.bs_grid_load(None, None, None, None, None) == 1
    assert lib.bs_mabs(None, None, None, 0, None) == 1


def test_null_handles_of_the_output_and_analysis_entry_points(lib):
    """Every entry point added for the closable layouts, the binning and the
    gridding refuses a NULL plan with BS_ERR_ARG before touching a device."""
    d = ctypes.c_double(0.0)
    assert lib.bs_mabs_delta_closable(None, None, None) == 1
    assert lib.bs_bs3d_closable(None, None, None) == 1
    assert lib.bs_plan_ring_umean(None, None) == 1
    assert lib.bs_bs_monopole(None, None, None, None, None, 12, 5, 5, d, d, d, None, None,
                              None) == 1
    assert lib.bs_bs_cylindrical(None, None, None, None, 20, None, None, None) == 1
    assert lib.bs_grid_visibilities(None, None, None, None, ctypes.c_int64(0), 4, 4, 0, None,
                                    None, None) == 1


def test_every_declaration_is_documented():
    """Each entry point of include/bs.h follows a comment block (its arguments,
    layout, ownership, errors and the passage it implements); declarations
    that share one block (create / destroy / last_error) may follow each other
    or a typedef."""
    lines = open(os.path.join(ROOT, "include", "bs.h")).read().split("\n")
    decl = re.compile(r"^(bs_status|int|const char \*)\s*\*?\s*bs_\w+\s*\(")
    for i, line in enumerate(lines):
        if not decl.match(line):
            continue
        j = i - 1
        while j >= 0 and lines[j].strip() and not lines[j].rstrip().endswith("*/"):
            assert (decl.match(lines[j]) or lines[j].startswith((" ", "typedef"))), (line, lines[j])
            j -= 1
        assert j >= 0 and lines[j].rstrip().endswith("*/"), line


def test_counts_noalloc_binding_refuses_wrong_tensors():
    """The allocation-free counts write nb(nb+1)(nb+2)/6 int64 entries and read
    an nt x nt float grid: the binding refuses other dtypes and sizes before
    any pointer reaches the library."""
    import torch
    edges = [1.0, 3.0, 5.0, 7.0, 9.0]  # 4 rings: 20 ring triples
    with pytest.raises(ValueError):
        bs.counts_noalloc(32, edges, torch.zeros(20, dtype=torch.int32))
    with pytest.raises(ValueError):
        bs.counts_noalloc(32, edges, torch.zeros(21, dtype=torch.int64))
    with pytest.raises(ValueError):
        bs.counts_noalloc(32, edges, torch.zeros(20, dtype=torch.int64),
                          ngrid=torch.ones((32, 16), dtype=torch.float32))
    with pytest.raises(ValueError):
        bs.counts_noalloc(32, edges, torch.zeros(20, dtype=torch.int64),
                          ngrid=torch.ones((32, 32), dtype=torch.float64))


class _NoLibrary:
    """Stands in for the loaded library: any entry point that is called fails
    the test, so a refusal must come before the call."""

    def __getattr__(self, name):
        def reached(*args):
            raise AssertionError(f"{name} was called with unchecked arguments")
        return reached


def _bare(cls, props=None, **attrs):
    """An instance of a binding class with the given attributes (props: class
    attributes in place of properties that ask the library) and no library
    handle: the argument checks run before any call into the library."""
    if props:
        cls = type("Bare" + cls.__name__, (cls,), dict(props))
    obj = object.__new__(cls)
    obj.__dict__.update(attrs)
    obj._h = None
    obj._L = _NoLibrary()
    return obj


@contextlib.contextmanager
def _refused():
    """The call raises ValueError from a dtype or size check (the tensors here
    live on the CPU, so the later 'expected a CUDA tensor' check must not be
    what refuses them)."""
    with pytest.raises(ValueError) as e:
        yield
    assert "CUDA tensor" not in str(e.value), str(e.value)


def test_bindings_refuse_wrong_tensors_before_the_library():
    """Entry points that read or write caller tensors through bare pointers:
    the binding refuses a dtype or extent other than the one the kernels
    touch, so no undersized buffer reaches the device."""
    import torch
    plan = _bare(bs.Plan, {"n_closable": 4}, nt=16, nchan=4, batch=2, nbins=3, ntrip=10,
                 general=False, chan_sampling=False)
    with _refused():  # half the cells
        plan.check_hermitian(torch.zeros((1, 4, 16, 16), dtype=torch.complex64))
    with _refused():  # the right count of the wrong type
        plan.check_hermitian(torch.zeros((2, 4, 16, 16), dtype=torch.complex128))
    with _refused():
        plan.grid_load(torch.zeros((2, 4, 16, 8), dtype=torch.complex64))
    with _refused():
        plan.grid_load(torch.zeros((2, 4, 16, 16), dtype=torch.complex64),
                       ngrid=torch.ones((4, 16, 16), dtype=torch.float32))
    with _refused():
        plan.mabs(block=(0, 4, 0, 4))
    with _refused():
        plan.mabs_delta(torch.zeros((2, 10, 7, 7), dtype=torch.float32))
    with _refused():
        plan.bs3d(torch.zeros((2, 10, 4, 3), dtype=torch.float64))
    with _refused():
        plan.mlp_features(np.zeros(3, np.uint8))
    with _refused():
        plan.delta_import(torch.zeros((2, 10, 7, 6), dtype=torch.float64), np.zeros(49, np.int64))
    with _refused():  # a plane of the wrong type for a real plan
        plan.error_bound(torch.zeros((2, 10, 7, 7), dtype=torch.complex128))
    kp, kz, ke = np.ones(3), np.linspace(-1, 1, 4), np.linspace(0.1, 2, 5)
    with _refused():
        plan.bs_monopole(torch.zeros((2, 4, 4, 3), dtype=torch.float64), kp, kz, ke)
    with _refused():
        plan.bs_multipoles(torch.zeros((2, 4, 4, 4), dtype=torch.float32), kp, kz, ke)
    with _refused():
        plan.bs_cylindrical(torch.zeros((1, 4, 4, 4), dtype=torch.float64), kz, ke)
    gplan = _bare(bs.Plan, {"n_closable": 4}, nt=16, nchan=4, batch=2, nbins=3, ntrip=10,
                  general=True, chan_sampling=False)
    with _refused():  # a general plan's values are complex
        gplan.bs_monopole(torch.zeros((2, 4, 4, 4), dtype=torch.float64), kp, kz, ke)
    with _refused():
        gplan.bs_cylindrical(torch.zeros((2, 4, 4, 4), dtype=torch.float64), kz, ke)
    with _refused():
        gplan.error_bound(torch.zeros((2, 10, 7, 7), dtype=torch.float64))

    net = _bare(bs.Surrogate, d=45, w=128, n_weights=100, n_total=192)
    x = torch.zeros((8, 45), dtype=torch.float32)
    t = torch.zeros(8, dtype=torch.float32)
    for bad_x, bad_t in ((torch.zeros((8, 44), dtype=torch.float32), t),   # too few features
                         (x.double(), t),                                  # FP64 rows
                         (x, torch.zeros(7, dtype=torch.float32)),         # fewer targets
                         (x, t.double())):
        with _refused():
            net.fit_norm(bad_x, bad_t)
        with _refused():
            net.grad(bad_x, bad_t)
        with _refused():
            net.train(bad_x, bad_t, steps=1)
    with _refused():
        net.forward(torch.zeros((8, 44), dtype=torch.float32))
    with _refused():
        net.set_params(np.zeros(191, np.float32))

    ens = _bare(bs.Ensemble, groups=[dict(nt=16, nchan=4, batch=2)], _torch=torch)
    with _refused():  # the right shape of the wrong type
        ens.set_input(0, torch.zeros((2, 4, 16, 16), dtype=torch.float32))
    with _refused():
        ens.set_input(-1, torch.zeros((2, 4, 16, 16), dtype=torch.complex64))
    with _refused():
        ens.set_flags(1, np.zeros(4, np.uint8))
    with _refused():
        ens.set_flags(0, np.zeros(5, np.uint8))
    with _refused():
        ens.set_block(0, (0, 4, 0, 4, 0))


def test_null_handles_of_the_ensemble_surrogate_and_sky_entry_points(lib):
    """Every entry point of the Monte Carlo ensemble, the surrogate network and
    the sky generator refuses a NULL handle with BS_ERR_ARG (destroy accepts
    it) on the host, without a device and without dereferencing it."""
    c = ctypes.c_int()
    u = ctypes.c_uint64()
    blk = (ctypes.c_int32 * 6)(0, 1, 0, 1, 0, 1)
    arr = (ctypes.c_int64 * 7)()
    assert lib.bs_mc_destroy(None) == 0
    assert lib.bs_mlp_destroy(None) == 0
    assert lib.bs_sky_destroy(None) == 0
    calls = [
        lambda: lib.bs_mc_info(None, 0, arr, 7),
        lambda: lib.bs_mc_set_input(None, 0, None),
        lambda: lib.bs_mc_set_flags(None, 0, None),
        lambda: lib.bs_mc_set_tuning(None, 1),
        lambda: lib.bs_mc_autotune(None, None, ctypes.byref(c), None),
        lambda: lib.bs_mc_tuning(None, None, None),
        lambda: lib.bs_mc_set_block(None, 0, blk),
        lambda: lib.bs_mc_run(None, 1, None),
        lambda: lib.bs_mc_reset(None, None),
        lambda: lib.bs_mc_stats(None, 0, 0, None, None, None, None),
        lambda: lib.bs_mc_checkpoint(None, b"x", ctypes.c_uint64(0), None),
        lambda: lib.bs_mc_restore(None, b"x", ctypes.byref(u), None),
        lambda: lib.bs_mlp_params(None, None, ctypes.c_int64(0), 0),
        lambda: lib.bs_mlp_fit_norm(None, None, None, 2, None),
        lambda: lib.bs_mlp_forward(None, None, 1, None, None),
        lambda: lib.bs_mlp_set_kernels(None, 0),
        lambda: lib.bs_mlp_grad(None, None, None, 1, None, None, None),
        lambda: lib.bs_mlp_train(None, None, None, 1, 1, 1, ctypes.c_float(1e-3),
                                 ctypes.c_uint64(0), None, None),
        lambda: lib.bs_mlp_features(None, None, None, None),
        lambda: lib.bs_sky_generate(None, ctypes.c_uint64(0), ctypes.c_uint64(0), 1, None, None),
    ]
    for k, call in enumerate(calls):
        assert call() == 1, k
