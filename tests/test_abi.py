"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol that include/bs.h declares, and refuses cleanly (no CPU fallback)
when no sm_103a device is present.  No compute call runs here."""
import ctypes
import os
import re

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
