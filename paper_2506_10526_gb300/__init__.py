"""GB300 (sm_103a) visibility bispectrum estimator: Python binding of libbs.

Thin ctypes layer over the C ABI in ``include/bs.h`` (arXiv:2506.10526,
Section 3.2).  It only marshals arguments: every step of the estimator runs
in libbs's own CUDA kernels.  PyTorch provides device memory (tensors whose
``data_ptr()`` is passed down) and streams.  There is no CPU fallback: if
libbs.so is missing or no sm_103a device is present, calls raise.

Names follow the C entry points: ``bs_plan_create`` -> :class:`Plan`,
``bs_grid_load`` -> :meth:`Plan.grid_load`, ``bs_counts`` ->
:meth:`Plan.counts`, ``bs_mabs`` -> :meth:`Plan.mabs`, ``bs_mabs_delta`` ->
:meth:`Plan.mabs_delta`, ``bs_bs3d`` -> :meth:`Plan.bs3d`.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbs.so")
# BS_LIBRARY=checked loads the -DBS_CHECKED build (device bounds checks that
# record a violation instead of faulting; build.build(checked=True) makes it)
LIB_CHECKED_PATH = os.path.join(HERE, "_build_checked", "libbs_checked.so")


def _lib_path() -> str:
    return LIB_CHECKED_PATH if os.environ.get("BS_LIBRARY") == "checked" else LIB_PATH

BS_OK = 0
STATUS = {0: "BS_OK", 1: "BS_ERR_ARG", 2: "BS_ERR_NO_DEVICE", 3: "BS_ERR_CUDA", 4: "BS_ERR_OOM",
          5: "BS_ERR_NOT_HERMITIAN", 6: "BS_ERR_TIMEOUT", 7: "BS_ERR_STATE",
          8: "BS_ERR_UNSUPPORTED"}
PREC_FP32 = 0
PREC_SPLIT_BF16 = 1
PREC_SPLIT_FP16 = 2
ABI_VERSION = 13     # BS_ABI_VERSION of include/bs.h
MLP_FEATURES = 45    # BS_MLP_FEATURES of include/bs.h

# every symbol declared in include/bs.h
EXPORTS = ("bs_abi_version", "bs_plan_create", "bs_plan_destroy", "bs_last_error",
           "bs_plan_info", "bs_plan_trip_sides", "bs_plan_set_workspace", "bs_grid_load", "bs_counts", "bs_mabs",
           "bs_delta_reset", "bs_mabs_delta", "bs_bs3d", "bs_mabs_delta_closable",
           "bs_bs3d_closable", "bs_mabs_error_bound", "bs_delta_export", "bs_delta_import", "bs_grid_visibilities", "bs_plan_ring_umean", "bs_bs_monopole",
           "bs_bs_cylindrical", "bs_bs_multipoles", "bs_check_hermitian",
           "bs_mc_create", "bs_mc_destroy", "bs_mc_last_error", "bs_mc_info", "bs_mc_set_input",
           "bs_mc_set_flags", "bs_mc_set_tuning", "bs_mc_autotune", "bs_mc_run", "bs_mc_reset",
           "bs_mc_stats", "bs_mc_tuning", "bs_mc_set_block", "bs_mc_checkpoint",
           "bs_mc_restore",
           "bs_mlp_features", "bs_mlp_create", "bs_mlp_destroy", "bs_mlp_last_error",
           "bs_mlp_params", "bs_mlp_fit_norm", "bs_mlp_forward", "bs_mlp_set_kernels", "bs_mlp_grad", "bs_mlp_train",
           "bs_sky_create", "bs_sky_destroy", "bs_sky_last_error", "bs_sky_generate",
           "bs_counts_noalloc", "bs_measure_peak", "bs_checked_build", "bs_checked_status",
           "bs_checked_selftest")

_lib = None
_lock = threading.Lock()


class BsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [("nt", ctypes.c_int), ("nchan", ctypes.c_int), ("nbins", ctypes.c_int),
                ("bin_edges", ctypes.POINTER(ctypes.c_double)), ("fft_m", ctypes.c_int),
                ("precision", ctypes.c_int), ("batch", ctypes.c_int),
                ("norm_A", ctypes.c_double), ("r", ctypes.c_double),
                ("rprime", ctypes.c_double), ("dnu_c", ctypes.c_double),
                ("multires", ctypes.c_int), ("general", ctypes.c_int),
                ("chan_sampling", ctypes.c_int)]


def lib() -> ctypes.CDLL:
    """Load libbs.so (built in-tree by ``build.py``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            path = _lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{os.path.basename(path)} not built ({path}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(path)
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            L.bs_abi_version.restype = I
            L.bs_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(P)]
            L.bs_plan_destroy.argtypes = [P]
            L.bs_last_error.argtypes = [P]
            L.bs_last_error.restype = ctypes.c_char_p
            L.bs_plan_info.argtypes = [P, P, I]
            L.bs_plan_trip_sides.argtypes = [P, P]
            L.bs_plan_set_workspace.argtypes = [P, P, ctypes.c_size_t]
            L.bs_grid_load.argtypes = [P, P, P, P, P]
            L.bs_counts.argtypes = [P, P, P]
            L.bs_mabs.argtypes = [P, P, P, I, P]
            L.bs_delta_reset.argtypes = [P, P]
            L.bs_mabs_delta.argtypes = [P, P, P]
            L.bs_bs3d.argtypes = [P, P, P]
            L.bs_check_hermitian.argtypes = [P, P, D, P]
            L.bs_mabs_error_bound.argtypes = [P, P, P, I, P, P]
            L.bs_delta_export.argtypes = [P, P, P, P]
            L.bs_delta_import.argtypes = [P, P, P, I, P]
            L.bs_counts_noalloc.argtypes = [I, I, P, P, P, P]
            L.bs_measure_peak.argtypes = [I, I, P, P]
            L.bs_checked_build.restype = I
            L.bs_checked_build.argtypes = []
            L.bs_checked_status.argtypes = [I, P]
            L.bs_checked_selftest.argtypes = [ctypes.c_int64, ctypes.c_int64, P]
            L.bs_plan_ring_umean.argtypes = [P, P]
            L.bs_bs_monopole.argtypes = [P, P, P, P, P, I, I, I, D, D, D, P, P, P]
            L.bs_bs_multipoles.argtypes = [P, P, P, P, P, I, I, I, I, P, P, P]
            L.bs_bs_cylindrical.argtypes = [P, P, P, P, I, P, P, P]
            L.bs_sky_create.argtypes = [I, I, D, D, D, I, ctypes.POINTER(P)]
            L.bs_sky_destroy.argtypes = [P]
            L.bs_sky_last_error.argtypes = [P]
            L.bs_sky_last_error.restype = ctypes.c_char_p
            L.bs_sky_generate.argtypes = [P, ctypes.c_uint64, ctypes.c_uint64, I, P, P]
            L.bs_mc_create.argtypes = [P, I, ctypes.POINTER(P)]
            L.bs_mc_destroy.argtypes = [P]
            L.bs_mc_last_error.argtypes = [P]
            L.bs_mc_last_error.restype = ctypes.c_char_p
            L.bs_mc_info.argtypes = [P, I, P, I]
            L.bs_mc_set_input.argtypes = [P, I, P]
            L.bs_mc_set_tuning.argtypes = [P, I]
            L.bs_mc_set_flags.argtypes = [P, I, P]
            L.bs_mc_run.argtypes = [P, I, P]
            L.bs_mc_autotune.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(I), P]
            L.bs_mc_reset.argtypes = [P, P]
            L.bs_mc_tuning.argtypes = [P, P, P]
            L.bs_mc_set_block.argtypes = [P, I, P]
            L.bs_mc_checkpoint.argtypes = [P, ctypes.c_char_p, ctypes.c_uint64, P]
            L.bs_mc_restore.argtypes = [P, ctypes.c_char_p, P, P]
            L.bs_mc_stats.argtypes = [P, I, I, P, P, P, P]
            L.bs_mlp_features.argtypes = [P, P, P, P]
            L.bs_mlp_create.argtypes = [I, I, ctypes.c_uint64, ctypes.POINTER(P)]
            L.bs_mlp_destroy.argtypes = [P]
            L.bs_mlp_last_error.argtypes = [P]
            L.bs_mlp_last_error.restype = ctypes.c_char_p
            L.bs_mlp_params.argtypes = [P, P, ctypes.c_int64, I]
            L.bs_mlp_fit_norm.argtypes = [P, P, P, I, P]
            L.bs_mlp_forward.argtypes = [P, P, I, P, P]
            L.bs_mlp_set_kernels.argtypes = [P, I]
            L.bs_mlp_grad.argtypes = [P, P, P, I, P, P, P]
            L.bs_mlp_train.argtypes = [P, P, P, I, I, I, ctypes.c_float, ctypes.c_uint64, P, P]
            for name in EXPORTS:
                if name not in ("bs_abi_version", "bs_last_error", "bs_mc_last_error", "bs_checked_build",
                                "bs_mlp_last_error", "bs_sky_last_error"):
                    getattr(L, name).restype = I
            _lib = L
    return _lib


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _dptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _require(t, dtype, numel, what):
    """Refuse a caller tensor whose dtype or element count differs from what the
    entry point reads or writes, before its pointer reaches the library (the C
    side receives bare pointers and cannot check their extent)."""
    if t.dtype != dtype or t.numel() != numel:
        raise ValueError(f"{what} must be {dtype} with {numel} elements "
                         f"(got {t.dtype} with {t.numel()})")


class Plan:
    """bs_plan_create / bs_plan_destroy.  Workspace comes from torch."""

    def __init__(self, nt: int, nchan: int, edges, precision: int = PREC_FP32, batch: int = 1,
                 fft_m: int = 0, norm_A: float = 1.0, r: float = 1.0, rprime: float = 1.0,
                 dnu_c: float = 1.0, torch_workspace: bool = True, multires: bool = False,
                 general: bool = False, chan_sampling: bool = False):
        import torch
        L = lib()
        self._L = L
        e = [float(x) for x in edges]
        self._edges = (ctypes.c_double * len(e))(*e)
        d = PlanDesc(nt, nchan, len(e) - 1, self._edges, fft_m, precision, batch, norm_A, r,
                     rprime, dnu_c, 1 if multires else 0, 1 if general else 0,
                     1 if chan_sampling else 0)
        self.general = bool(general)
        self.chan_sampling = bool(chan_sampling)
        h = ctypes.c_void_p()
        st = L.bs_plan_create(ctypes.byref(d), ctypes.byref(h))
        if st != BS_OK:
            raise BsError(st, L.bs_last_error(None).decode())
        self._h = h
        self.nt, self.nchan, self.nbins, self.batch = nt, nchan, len(e) - 1, batch
        self.precision = precision
        info = self.info()
        self.M, self.ntrip, self.nfields, self.ws_bytes, self.ucols = info[:5]
        self._ws = None
        if torch_workspace:
            self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            off = (-base) % 256
            self._check(L.bs_plan_set_workspace(self._h, ctypes.c_void_p(base + off),
                                                ctypes.c_size_t(self.ws_bytes)))

    def _check(self, st):
        if st != BS_OK:
            raise BsError(st, self._L.bs_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.bs_plan_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        arr = (ctypes.c_int64 * 7)()
        self._check(self._L.bs_plan_info(self._h, arr, 7))
        return list(arr)

    def trip_sides(self):
        """bs_plan_trip_sides: image side M of every ring triple (numpy int64)."""
        import numpy as np
        out = np.zeros(self.ntrip, np.int64)
        self._check(self._L.bs_plan_trip_sides(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def grid_load(self, vis, ngrid=None, chan_flags=None, stream=None):
        """bs_grid_load: vis complex64 CUDA tensor [batch, nchan, nt, nt]; ngrid float32
        [nt, nt] (or [nchan, nt, nt] in a per-channel sampling plan) or None."""
        import numpy as np
        import torch
        if vis.dtype != torch.complex64 or vis.numel() != self.batch * self.nchan * self.nt ** 2:
            raise ValueError("vis must be complex64 [batch, nchan, nt, nt]")
        if ngrid is not None:
            want = (self.nchan if self.chan_sampling else 1) * self.nt ** 2
            if ngrid.dtype != torch.float32 or ngrid.numel() != want:
                raise ValueError(f"ngrid must be float32 with {want} elements")
        flags = None
        if chan_flags is not None:
            f = np.ascontiguousarray(np.asarray(chan_flags, dtype=np.uint8))
            if f.size != self.nchan:
                raise ValueError("chan_flags must have nchan entries")
            self._flags = f
            flags = f.ctypes.data_as(ctypes.c_void_p)
        self._check(self._L.bs_grid_load(self._h, _dptr(vis), _dptr(ngrid), flags,
                                         _stream_ptr(stream)))

    def counts(self):
        """bs_counts: (T [ntrip] int64, folded N_nu [(2nc-1)^2] int64) as numpy."""
        import numpy as np
        tri = np.zeros(self.ntrip, np.int64)
        nnu = np.zeros((2 * self.nchan - 1) ** 2, np.int64)
        self._check(self._L.bs_counts(self._h, tri.ctypes.data_as(ctypes.c_void_p),
                                      nnu.ctypes.data_as(ctypes.c_void_p)))
        return tri, nnu.reshape(2 * self.nchan - 1, 2 * self.nchan - 1)

    def _out(self, t, planes, side):
        """Pointer of an output tensor of [batch, planes, side, side] float64 values
        (complex128 for general plans), refused when the type or size differs."""
        import torch
        want = torch.complex128 if self.general else torch.float64
        if t.dtype != want or t.numel() != self.batch * planes * side * side:
            raise ValueError(f"output must be {want} with {self.batch * planes * side * side} "
                             "elements")
        return _dptr(t)

    def mabs(self, block=None, out_full=None, accumulate=True, stream=None, symmetric=False):
        """bs_mabs over channel block (nu1_lo, nu1_hi, nu2_lo, nu2_hi, nu3_lo, nu3_hi).
        symmetric=True accumulates a cube block S x S x S with the channel symmetry
        of repeated rings (accumulate = 2)."""
        full = None
        if out_full is not None:
            full = self._out(out_full, self.ntrip * self.nchan, self.nchan)
        blk = None
        if block is not None:
            if len(block) != 6:
                raise ValueError("block is (nu1_lo, nu1_hi, nu2_lo, nu2_hi, nu3_lo, nu3_hi)")
            self._blk = (ctypes.c_int32 * 6)(*[int(x) for x in block])
            blk = self._blk
        acc = 2 if symmetric else (1 if accumulate else 0)
        self._check(self._L.bs_mabs(self._h, blk, full, acc, _stream_ptr(stream)))

    def delta_reset(self, stream=None):
        self._check(self._L.bs_delta_reset(self._h, _stream_ptr(stream)))

    def mabs_delta(self, out, stream=None):
        """bs_mabs_delta: out float64 CUDA [batch, ntrip, 2nc-1, 2nc-1]."""
        self._check(self._L.bs_mabs_delta(self._h, self._out(out, self.ntrip, 2 * self.nchan - 1),
                                          _stream_ptr(stream)))

    def bs3d(self, out, stream=None):
        """bs_bs3d: out float64 CUDA [batch, ntrip, nc, nc]."""
        self._check(self._L.bs_bs3d(self._h, self._out(out, self.ntrip, self.nchan),
                                    _stream_ptr(stream)))

    @property
    def n_closable(self):
        """Ring triples with at least one closed triangle (bs_plan_info [5]; -1 before
        the first grid load or count)."""
        return self.info()[5]

    def mabs_delta_closable(self, out, stream=None):
        """bs_mabs_delta_closable: out float64 CUDA [batch, n_closable, 2nc-1, 2nc-1], the
        closable ring triples in ascending index."""
        self._check(self._L.bs_mabs_delta_closable(
            self._h, self._out(out, self.n_closable, 2 * self.nchan - 1), _stream_ptr(stream)))

    def grid_visibilities(self, uv, vis, flags=None, avg=1, mode=0, stream=None):
        """bs_grid_visibilities (Eq. vg): uv float64 CUDA [nbl, 2] in grid units, vis
        complex64 CUDA [nbl, avg * nchan], flags uint8 CUDA or None.  Returns
        (vis_g complex64 [nchan, nt, nt], n_g float32 [nchan, nt, nt]); mode 1 gives the
        per-channel mean and a 0/1 occupancy for grid_load."""
        import torch
        nbl = int(vis.shape[0])
        if (uv.dtype != torch.float64 or tuple(uv.shape) != (nbl, 2) or vis.dtype != torch.complex64
                or vis.dim() != 2 or (flags is not None and (flags.dtype != torch.uint8
                                                             or flags.shape != vis.shape))):
            raise ValueError("uv float64 [nbl, 2], vis complex64 [nbl, nchan_in], flags uint8")
        out = torch.empty((self.nchan, self.nt, self.nt), dtype=torch.complex64, device="cuda")
        ng = torch.empty((self.nchan, self.nt, self.nt), dtype=torch.float32, device="cuda")
        self._check(self._L.bs_grid_visibilities(
            self._h, _dptr(uv), _dptr(vis), _dptr(flags), ctypes.c_int64(nbl), int(vis.shape[1]),
            int(avg), int(mode), _dptr(out), _dptr(ng), _stream_ptr(stream)))
        return out, ng

    def ring_umean(self):
        """bs_plan_ring_umean: mean |U| of each ring's cells (numpy float64 [nbins])."""
        import numpy as np
        out = np.zeros(self.nbins, np.float64)
        self._check(self._L.bs_plan_ring_umean(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def bs_monopole(self, b3d, kperp, kpar, k1_edges, n_mu=5, n_t=5, model=None, stream=None):
        """bs_bs_monopole: binned 3D-bispectrum monopole.  b3d: float64 CUDA tensor as
        bs3d_closable writes it, or None with model = (f_ng, p_amp, p_index) for the binned
        Eq. (bsana).  Returns (sums [batch, n_k1, n_mu, n_t] float64 CUDA (complex128
        for a general plan's complex b3d), counts [n_k1, n_mu, n_t] int64 CUDA)."""
        import numpy as np
        import torch
        kp = np.ascontiguousarray(np.asarray(kperp, np.float64))
        kz = np.ascontiguousarray(np.asarray(kpar, np.float64))
        ed = np.ascontiguousarray(np.asarray(k1_edges, np.float64))
        if kp.size != self.nbins or kz.size != self.nchan:
            raise ValueError("kperp needs nbins entries and kpar nchan entries")
        n_k1 = ed.size - 1
        batch = 1 if b3d is None else self.batch
        vt = torch.complex128 if self.general else torch.float64  # a general plan's values
        if b3d is not None:
            _require(b3d, vt, batch * self.n_closable * self.nchan ** 2,
                     "b3d [batch, n_closable, nchan, nchan]")
        sdt = torch.float64 if b3d is None else vt
        sums = torch.empty((batch, n_k1, n_mu, n_t), dtype=sdt, device="cuda")
        cnt = torch.empty((n_k1, n_mu, n_t), dtype=torch.int64, device="cuda")
        f, a, pi = model if model is not None else (0.0, 0.0, 0.0)
        self._check(self._L.bs_bs_monopole(
            self._h, _dptr(b3d), kp.ctypes.data_as(ctypes.c_void_p),
            kz.ctypes.data_as(ctypes.c_void_p), ed.ctypes.data_as(ctypes.c_void_p), n_k1, n_mu, n_t,
            ctypes.c_double(f), ctypes.c_double(a), ctypes.c_double(pi), _dptr(sums), _dptr(cnt),
            _stream_ptr(stream)))
        return sums, cnt

    def bs_multipoles(self, b3d, kperp, kpar, k1_edges, n_mu=5, n_t=5, lmax=4, stream=None):
        """bs_bs_multipoles: m = 0 multipoles binned like bs_monopole.  Returns
        (sums [batch, lmax + 1, n_k1, n_mu, n_t] float64 CUDA (complex128 for a general
        plan), counts [n_k1, n_mu, n_t] int64 CUDA); B_l^0 = sums / counts."""
        import numpy as np
        import torch
        kp = np.ascontiguousarray(np.asarray(kperp, np.float64))
        kz = np.ascontiguousarray(np.asarray(kpar, np.float64))
        ed = np.ascontiguousarray(np.asarray(k1_edges, np.float64))
        if kp.size != self.nbins or kz.size != self.nchan:
            raise ValueError("kperp needs nbins entries and kpar nchan entries")
        vt = torch.complex128 if self.general else torch.float64  # a general plan's values
        _require(b3d, vt, self.batch * self.n_closable * self.nchan ** 2,
                 "b3d [batch, n_closable, nchan, nchan]")
        n_k1 = ed.size - 1
        sums = torch.empty((self.batch, lmax + 1, n_k1, n_mu, n_t), dtype=vt, device="cuda")
        cnt = torch.empty((n_k1, n_mu, n_t), dtype=torch.int64, device="cuda")
        P = ctypes.c_void_p
        self._check(self._L.bs_bs_multipoles(
            self._h, _dptr(b3d), kp.ctypes.data_as(P), kz.ctypes.data_as(P), ed.ctypes.data_as(P),
            int(n_k1), int(n_mu), int(n_t), int(lmax), _dptr(sums), _dptr(cnt),
            _stream_ptr(stream)))
        return sums, cnt

    def bs_cylindrical(self, b3d, kpar, edges, stream=None):
        """bs_bs_cylindrical: the closable 3D bispectrum binned on the (k_par1, k_par2)
        grid of the given edges.  Returns (sums [batch, n_closable, n, n] float64 CUDA
        (complex128 for a general plan), counts [n, n] int64 CUDA)."""
        import numpy as np
        import torch
        kz = np.ascontiguousarray(np.asarray(kpar, np.float64))
        ed = np.ascontiguousarray(np.asarray(edges, np.float64))
        n = ed.size - 1
        if kz.size != self.nchan:
            raise ValueError("kpar needs nchan entries")
        vt = torch.complex128 if self.general else torch.float64  # a general plan's values
        _require(b3d, vt, self.batch * self.n_closable * self.nchan ** 2,
                 "b3d [batch, n_closable, nchan, nchan]")
        sums = torch.empty((self.batch, self.n_closable, n, n), dtype=vt, device="cuda")
        cnt = torch.empty((n, n), dtype=torch.int64, device="cuda")
        self._check(self._L.bs_bs_cylindrical(
            self._h, _dptr(b3d), kz.ctypes.data_as(ctypes.c_void_p),
            ed.ctypes.data_as(ctypes.c_void_p), n, _dptr(sums), _dptr(cnt), _stream_ptr(stream)))
        return sums, cnt

    def bs3d_closable(self, out, stream=None):
        """bs_bs3d_closable: out float64 CUDA [batch, n_closable, nc, nc], the closable ring
        triples in ascending index."""
        self._check(self._L.bs_bs3d_closable(self._h, self._out(out, self.n_closable, self.nchan),
                                             _stream_ptr(stream)))

    def delta_export(self, stream=None):
        """bs_delta_export: (sums float64 CUDA [batch, ntrip, 2nc-1, 2nc-1], nnu int64 numpy
        [2nc-1, 2nc-1]): the raw collapse sums and unfolded sampling."""
        import numpy as np
        import torch
        n2 = 2 * self.nchan - 1
        sums = torch.empty((self.batch, self.ntrip, n2, n2), dtype=torch.float64, device="cuda")
        nnu = np.zeros((n2, n2), np.int64)
        self._check(self._L.bs_delta_export(self._h, _dptr(sums),
                                            nnu.ctypes.data_as(ctypes.c_void_p),
                                            _stream_ptr(stream)))
        return sums, nnu

    def delta_import(self, sums, nnu, add=False, stream=None):
        """bs_delta_import: replace (or add to) the collapse accumulators."""
        import numpy as np
        import torch
        n2 = 2 * self.nchan - 1
        if sums.dtype != torch.float64 or sums.numel() != self.batch * self.ntrip * n2 * n2:
            raise ValueError("sums must be float64 [batch, ntrip, 2nc-1, 2nc-1]")
        nn = np.ascontiguousarray(np.asarray(nnu, dtype=np.int64))
        if nn.size != n2 * n2:
            raise ValueError("nnu must hold (2nc-1)^2 entries")
        self._check(self._L.bs_delta_import(self._h, _dptr(sums), nn.ctypes.data_as(ctypes.c_void_p),
                                            int(bool(add)), _stream_ptr(stream)))

    def error_bound(self, delta=None, closable=False, stream=None):
        """bs_mabs_error_bound: float64 CUDA [batch, ntrip] bounds on |B_A error| per ring
        triple (the modulus of the complex error in a general plan); with ``delta`` (a
        folded plane from mabs_delta, or from mabs_delta_closable with closable=True) also
        the per-bin relative bound, float64 of the same shape.  A per-channel sampling plan
        needs ``delta``: its bound is per bin, and ``bound`` is the largest over each ring
        triple's bins.  Returns (bound, relerr or None)."""
        import torch
        rel = None
        if delta is not None:
            npl = self.n_closable if closable else self.ntrip
            want = torch.complex128 if self.general else torch.float64
            _require(delta, want, self.batch * npl * (2 * self.nchan - 1) ** 2,
                     "delta [batch, planes, 2nc-1, 2nc-1]")
            rel = torch.empty(delta.shape, dtype=torch.float64, device="cuda")
        bound = torch.empty((self.batch, self.ntrip), dtype=torch.float64, device="cuda")
        self._check(self._L.bs_mabs_error_bound(self._h, _dptr(bound), _dptr(delta),
                                                int(bool(closable)), _dptr(rel),
                                                _stream_ptr(stream)))
        return bound, rel

    def mlp_features(self, chan_flags=None, stream=None):
        """bs_mlp_features: float32 CUDA tensor [ntrip*nc*nc, MLP_FEATURES] (NaN rows: no
        triangle)."""
        import numpy as np
        import torch
        fl = None
        if chan_flags is not None:
            self._mflags = np.ascontiguousarray(np.asarray(chan_flags, dtype=np.uint8))
            if self._mflags.size != self.nchan:
                raise ValueError("chan_flags must have nchan entries")
            fl = self._mflags.ctypes.data_as(ctypes.c_void_p)
        out = torch.empty((self.ntrip * self.nchan * self.nchan, MLP_FEATURES), dtype=torch.float32,
                          device="cuda")
        self._check(self._L.bs_mlp_features(self._h, fl, _dptr(out), _stream_ptr(stream)))
        return out

    def check_hermitian(self, vis, tol=1e-6, stream=None):
        """bs_check_hermitian; returns True when Hermitian within tol."""
        import torch
        _require(vis, torch.complex64, self.batch * self.nchan * self.nt ** 2,
                 "vis [batch, nchan, nt, nt]")
        st = self._L.bs_check_hermitian(self._h, _dptr(vis), ctypes.c_double(tol),
                                        _stream_ptr(stream))
        if st == 5:
            return False
        self._check(st)
        return True


def counts_noalloc(nt: int, edges, tri_out, ngrid=None, stream=None):
    """bs_counts_noalloc: closed-triangle counts into a caller-owned int64 CUDA
    tensor of nbins(nbins+1)(nbins+2)/6 entries; allocates no device memory."""
    import numpy as np
    import torch
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.float64))
    nb = e.size - 1
    # the kernels write nb(nb+1)(nb+2)/6 int64 counts and read nt x nt floats:
    # refuse anything else before it reaches the device
    if tri_out.dtype != torch.int64 or tri_out.numel() != nb * (nb + 1) * (nb + 2) // 6:
        raise ValueError(f"tri_out must be int64 with {nb * (nb + 1) * (nb + 2) // 6} elements")
    if ngrid is not None and (ngrid.dtype != torch.float32 or tuple(ngrid.shape) != (nt, nt)):
        raise ValueError(f"ngrid must be float32 of shape ({nt}, {nt})")
    st = lib().bs_counts_noalloc(int(nt), int(e.size - 1), e.ctypes.data_as(ctypes.c_void_p),
                                 _dptr(ngrid), _dptr(tri_out), _stream_ptr(stream))
    if st != BS_OK:
        raise BsError(st, "bs_counts_noalloc failed (sizes beyond nt <= 1024, nbins <= 32 are "
                          "rejected)")



def measure_peak(kind: str = "fp32", iters: int = 1 << 16, stream=None) -> float:
    """bs_measure_peak: measured FMA rate of the current device in FLOP/s
    (kind "fp32" or "fp64")."""
    out = ctypes.c_double(0.0)
    st = lib().bs_measure_peak({"fp32": 0, "fp64": 1}[kind], int(iters), ctypes.byref(out),
                               _stream_ptr(stream))
    if st != BS_OK:
        raise BsError(st, "bs_measure_peak failed")
    return out.value


class SkyGenerator:
    """bs_sky_*: realisations of the non-Gaussian validation sky (Eq. mb1)
    drawn on the GPU, written as centred visibilities [batch][nchan][nt][nt]."""

    def __init__(self, nt, nchan, slope=-2.0, sigma=0.5, f_ng=0.5, max_batch=1):
        L = lib()
        self._L = L
        h = ctypes.c_void_p()
        st = L.bs_sky_create(int(nt), int(nchan), float(slope), float(sigma), float(f_ng),
                             int(max_batch), ctypes.byref(h))
        if st != BS_OK:
            raise BsError(st, L.bs_sky_last_error(None).decode())
        self._h = h
        self.nt, self.nchan, self.max_batch = int(nt), int(nchan), int(max_batch)

    def generate(self, seed, realisation0, out=None, batch=None, stream=None):
        """Realisations realisation0 .. + batch - 1 into `out` (a complex64 CUDA
        tensor of shape (batch, nchan, nt, nt); allocated when None)."""
        import torch
        if out is None:
            b = self.max_batch if batch is None else int(batch)
            out = torch.empty((b, self.nchan, self.nt, self.nt), dtype=torch.complex64,
                              device="cuda")
        if out.dtype != torch.complex64 or not out.is_cuda or not out.is_contiguous() or \
                tuple(out.shape[1:]) != (self.nchan, self.nt, self.nt):
            raise ValueError("out must be a contiguous complex64 CUDA tensor (batch, nchan, nt, nt)")
        st = self._L.bs_sky_generate(self._h, ctypes.c_uint64(int(seed)),
                                     ctypes.c_uint64(int(realisation0)), int(out.shape[0]),
                                     _dptr(out), _stream_ptr(stream))
        if st != BS_OK:
            raise BsError(st, self._L.bs_sky_last_error(self._h).decode())
        return out

    def close(self):
        if self._h:
            self._L.bs_sky_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

class Ensemble:
    """bs_mc_*: batched Monte Carlo over shape groups.

    groups: list of dicts with keys nt, nchan, edges, batch (and optionally
    fft_m, norm_A, r, rprime, dnu_c, precision).  All groups use one tensor-core
    precision: PREC_SPLIT_BF16 (default) or PREC_SPLIT_FP16."""

    def __init__(self, groups, tiles_per_sm=None):
        import torch
        L = lib()
        self._L = L
        n = len(groups)
        descs = (PlanDesc * n)()
        self._edges = []
        for g, spec in enumerate(groups):
            e = [float(x) for x in spec["edges"]]
            arr = (ctypes.c_double * len(e))(*e)
            self._edges.append(arr)
            descs[g] = PlanDesc(spec["nt"], spec["nchan"], len(e) - 1, arr, spec.get("fft_m", 0),
                                spec.get("precision", PREC_SPLIT_BF16), spec["batch"],
                                spec.get("norm_A", 1.0),
                                spec.get("r", 1.0), spec.get("rprime", 1.0), spec.get("dnu_c", 1.0),
                                1 if spec.get("multires", False) else 0)
        h = ctypes.c_void_p()
        st = L.bs_mc_create(descs, n, ctypes.byref(h))
        if st != BS_OK:
            raise BsError(st, L.bs_last_error(None).decode())
        self._h = h
        self.groups = [dict(g) for g in groups]
        for g, spec in enumerate(self.groups):
            info = (ctypes.c_int64 * 7)()
            self._check(L.bs_mc_info(h, g, info, 7))
            spec["M"], spec["ntrip"] = info[0], info[1]
        if tiles_per_sm is not None:
            self._check(L.bs_mc_set_tuning(h, int(tiles_per_sm)))
        self._torch = torch

    def _check(self, st):
        if st != BS_OK:
            raise BsError(st, self._L.bs_mc_last_error(self._h).decode())

    def set_input(self, g, vis):
        """bs_mc_set_input: vis is a complex64 CUDA tensor [batch, nchan, nt, nt]
        that the caller keeps alive and refills before each run."""
        if not 0 <= g < len(self.groups):
            raise ValueError(f"group {g} out of range")
        spec = self.groups[g]
        want = (spec["batch"], spec["nchan"], spec["nt"], spec["nt"])
        if tuple(vis.shape) != want or vis.dtype != self._torch.complex64:
            raise ValueError(f"group {g} expects complex64 {want}, got {vis.dtype} "
                             f"{tuple(vis.shape)}")
        self._inputs = getattr(self, "_inputs", {})
        self._inputs[g] = vis
        self._check(self._L.bs_mc_set_input(self._h, g, _dptr(vis)))

    def set_flags(self, g, flags):
        """bs_mc_set_flags: uint8 [nchan] (1 = flagged) or None."""
        import numpy as np
        if not 0 <= g < len(self.groups):
            raise ValueError(f"group {g} out of range")
        if flags is None:
            self._check(self._L.bs_mc_set_flags(self._h, g, None))
            return
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
        if f.size != self.groups[g]["nchan"]:
            raise ValueError("flags must have nchan entries")
        self._check(self._L.bs_mc_set_flags(self._h, g, f.ctypes.data_as(ctypes.c_void_p)))

    def autotune(self, cache_path=None, stream=None):
        """bs_mc_autotune: returns the chosen tiles-per-SM target."""
        c = ctypes.c_int()
        path = None if cache_path is None else str(cache_path).encode()
        self._check(self._L.bs_mc_autotune(self._h, path, ctypes.byref(c), _stream_ptr(stream)))
        return c.value

    def tuning(self):
        """bs_mc_tuning: (tiles_per_sm, tile_order) in effect."""
        t, o = ctypes.c_int(), ctypes.c_int()
        self._check(self._L.bs_mc_tuning(self._h, ctypes.byref(t), ctypes.byref(o)))
        return t.value, o.value

    def set_block(self, g, block):
        """bs_mc_set_block: channel block (nu1_lo, nu1_hi, nu2_lo, nu2_hi, nu3_lo, nu3_hi)
        that every run of group g contracts."""
        if len(block) != 6:
            raise ValueError("block is (nu1_lo, nu1_hi, nu2_lo, nu2_hi, nu3_lo, nu3_hi)")
        self._blk = (ctypes.c_int32 * 6)(*[int(x) for x in block])
        self._check(self._L.bs_mc_set_block(self._h, int(g), self._blk))

    def checkpoint(self, path, counter=0, stream=None):
        """bs_mc_checkpoint: statistics, runs, tuning and the caller's counter to `path`."""
        self._check(self._L.bs_mc_checkpoint(self._h, str(path).encode(),
                                             ctypes.c_uint64(int(counter)), _stream_ptr(stream)))

    def restore(self, path, stream=None):
        """bs_mc_restore: load a checkpoint of the same shapes; returns the counter."""
        c = ctypes.c_uint64(0)
        self._check(self._L.bs_mc_restore(self._h, str(path).encode(), ctypes.byref(c),
                                          _stream_ptr(stream)))
        return c.value

    def run(self, use_graph=True, stream=None):
        self._check(self._L.bs_mc_run(self._h, 1 if use_graph else 0, _stream_ptr(stream)))

    def reset(self, stream=None):
        self._check(self._L.bs_mc_reset(self._h, _stream_ptr(stream)))

    def stats(self, g, which=0, stream=None):
        """(mean, var, realisations) of group g: which=0 collapsed plane, 1 = 3D BS."""
        torch = self._torch
        spec = self.groups[g]
        nc, nt_ = spec["nchan"], spec["ntrip"]
        shape = (nt_, 2 * nc - 1, 2 * nc - 1) if which == 0 else (nt_, nc, nc)
        mean = torch.empty(shape, dtype=torch.float64, device="cuda")
        var = torch.empty(shape, dtype=torch.float64, device="cuda")
        n = ctypes.c_int64()
        self._check(self._L.bs_mc_stats(self._h, g, which, _dptr(mean), _dptr(var),
                                        ctypes.byref(n), _stream_ptr(stream)))
        torch.cuda.synchronize()
        return mean.cpu().numpy(), var.cpu().numpy(), n.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.bs_mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """bs_mlp_*: the error-bar network (d_in inputs, width hidden units)."""

    def __init__(self, d_in=None, width=128, seed=1):
        d_in = MLP_FEATURES if d_in is None else d_in
        L = lib()
        self._L = L
        h = ctypes.c_void_p()
        st = L.bs_mlp_create(int(d_in), int(width), ctypes.c_uint64(seed), ctypes.byref(h))
        if st != BS_OK:
            raise BsError(st, "bs_mlp_create failed")
        self._h = h
        self.d, self.w = int(d_in), int(width)
        self.n_weights = self.w * self.d + self.w + self.w * self.w + self.w + self.w + 1
        self.n_total = self.n_weights + 2 * self.d + 2

    def _check(self, st):
        if st != BS_OK:
            raise BsError(st, self._L.bs_mlp_last_error(self._h).decode())

    def params(self):
        import numpy as np
        p = np.empty(self.n_total, np.float32)
        self._check(self._L.bs_mlp_params(self._h, p.ctypes.data_as(ctypes.c_void_p),
                                          self.n_total, 0))
        return p

    def _rows(self, x, t=None):
        """Row count of a feature matrix x float32 [n, d_in] (and targets t float32
        [n]), refused when the kernels would read past either."""
        import torch
        if x.dim() != 2 or x.shape[1] != self.d:
            raise ValueError(f"x must be [n, {self.d}]")
        n = int(x.shape[0])
        _require(x, torch.float32, n * self.d, f"x [n, {self.d}]")
        if t is not None:
            _require(t, torch.float32, n, "t [n]")
        return n

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        if p.size != self.n_total:
            raise ValueError(f"params must hold {self.n_total} values")
        self._check(self._L.bs_mlp_params(self._h, p.ctypes.data_as(ctypes.c_void_p),
                                          self.n_total, 1))

    def fit_norm(self, x, t, stream=None):
        self._rows(x, t)
        self._check(self._L.bs_mlp_fit_norm(self._h, _dptr(x), _dptr(t), int(x.shape[0]),
                                            _stream_ptr(stream)))

    def forward(self, x, stream=None):
        import torch
        self._rows(x)
        y = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
        self._check(self._L.bs_mlp_forward(self._h, _dptr(x), int(x.shape[0]), _dptr(y),
                                           _stream_ptr(stream)))
        return y

    def set_kernels(self, kind):
        """bs_mlp_set_kernels: "tensor" (BF16 mma.sync, width 128) or "simt" (FP32)."""
        k = {"tensor": 0, "simt": 1}[kind]
        self._check(self._L.bs_mlp_set_kernels(self._h, k))

    def grad(self, x, t, stream=None):
        import numpy as np
        self._rows(x, t)
        g = np.empty(self.n_weights, np.float32)
        loss = np.zeros(1, np.float32)
        self._check(self._L.bs_mlp_grad(self._h, _dptr(x), _dptr(t), int(x.shape[0]),
                                        g.ctypes.data_as(ctypes.c_void_p),
                                        loss.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
        return float(loss[0]), g

    def train(self, x, t, steps, batch=8192, lr=2e-3, seed=7, stream=None):
        import numpy as np
        self._rows(x, t)
        loss = np.zeros(1, np.float32)
        self._check(self._L.bs_mlp_train(self._h, _dptr(x), _dptr(t), int(x.shape[0]), int(steps),
                                         int(batch), ctypes.c_float(lr), ctypes.c_uint64(seed),
                                         loss.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
        return float(loss[0])

    def close(self):
        if getattr(self, "_h", None):
            self._L.bs_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def checked_build() -> bool:
    """bs_checked_build: whether the loaded library is the -DBS_CHECKED build."""
    return bool(lib().bs_checked_build())


def checked_status(reset: bool = True):
    """bs_checked_status: {"violations", "site", "index", "extent"} since the
    last reset (checked build only)."""
    import numpy as np
    out = np.zeros(4, np.uint64)
    st = lib().bs_checked_status(int(bool(reset)), out.ctypes.data_as(ctypes.c_void_p))
    if st != BS_OK:
        raise BsError(st, "bs_checked_status failed")
    return {"violations": int(out[0]), "site": int(out[1]),
            "index": int(out[2].astype(np.int64)), "extent": int(out[3])}


def checked_selftest(n: int, idx: int, stream=None):
    """bs_checked_selftest: one guarded access to element idx of an n-element buffer."""
    st = lib().bs_checked_selftest(int(n), int(idx), _stream_ptr(stream))
    if st != BS_OK:
        raise BsError(st, "bs_checked_selftest failed")
