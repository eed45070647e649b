"""ctypes binding of libs2dw.so: the C ABI of include/s2dw.h under the same
names, plus a thin ``Plan`` class.  Argument marshalling only -- every step
of the transform runs in the library's CUDA kernels.  Device memory and
streams come from PyTorch.  There is no CPU fallback: if the library is
missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libs2dw.so")

S2DW_OK, S2DW_EINVAL, S2DW_ENOMEM, S2DW_ECUDA, S2DW_ETIMEOUT, S2DW_EBUSY, S2DW_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
S2DW_FP64, S2DW_MIXED, S2DW_REAL_SIGNAL, S2DW_MULTIRES, S2DW_MW = 1, 2, 4, 8, 16

_lib = None

_c_p = ctypes.c_void_p
_c_i = ctypes.c_int
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_ip = ctypes.POINTER(ctypes.c_int)
_c_dp = ctypes.POINTER(ctypes.c_double)

_SIGNATURES = {
    "s2dw_plan": (_c_i, [ctypes.POINTER(_c_p), _c_i, _c_i, ctypes.c_double, _c_i, ctypes.c_uint]),
    "s2dw_plan_destroy": (_c_i, [_c_p]),
    "s2dw_query": (_c_i, [_c_p, _c_ip, _c_i64p, _c_i64p, _c_i64p, _c_i64p]),
    "s2dw_launch_counts": (_c_i, [_c_p, _c_ip, _c_ip]),
    "s2dw_scale_grid": (_c_i, [_c_p, _c_i, _c_ip, _c_i64p, _c_i64p]),
    "s2dw_alpha_method": (_c_i, [_c_p, _c_i, _c_i, _c_ip, _c_ip, _c_ip, _c_ip]),
    "s2dw_steer": (_c_i, [_c_p, _c_p, _c_dp, _c_i, _c_p, _c_p]),
    "s2dw_sht_inverse": (_c_i, [_c_p, _c_p, _c_p, _c_p]),
    "s2dw_sht_forward": (_c_i, [_c_p, _c_p, _c_p, _c_p]),
    "s2dw_kernels": (_c_i, [_c_p, _c_dp, _c_dp]),
    "s2dw_analysis": (_c_i, [_c_p, _c_p, _c_p, _c_p, _c_p]),
    "s2dw_synthesis": (_c_i, [_c_p, _c_p, _c_p, _c_p, _c_p]),
    "s2dw_analysis_batch": (_c_i, [ctypes.POINTER(_c_p), ctypes.POINTER(_c_p), ctypes.POINTER(_c_p),
                                   ctypes.POINTER(_c_p), _c_i, _c_p]),
    "s2dw_synthesis_batch": (_c_i, [ctypes.POINTER(_c_p), ctypes.POINTER(_c_p), ctypes.POINTER(_c_p),
                                    ctypes.POINTER(_c_p), _c_i, _c_p]),
    "s2dw_strerror": (ctypes.c_char_p, [_c_i]),
    "s2dw_scale_support": (_c_i, [_c_p, _c_i, _c_ip, _c_ip]),
    "s2dw_delta_slab": (_c_i, [_c_p, _c_i, _c_dp]),
    "s2dw_stage": (_c_i, [_c_p, _c_i, _c_i, _c_p, _c_i64p]),
    "s2dw_profile": (_c_i, [_c_p, _c_i]),
    "s2dw_profile_read": (_c_i, [_c_p, _c_dp, _c_ip]),
    "s2dw_delta_table_noalloc": (_c_i, [_c_i, _c_p, _c_p, _c_i64p, _c_p]),
    "s2dw_wait_timeouts": (_c_i, [_c_ip]),
    "s2dw_plan_choices": (_c_i, [_c_p, _c_ip, _c_ip]),
    "s2dw_plan_set_choices": (_c_i, [_c_p, _c_ip, _c_i]),
    "s2dw_plan_tune": (_c_i, [_c_p, _c_i, _c_ip, _c_ip]),
    "s2dw_wait_probe": (_c_i, [ctypes.c_longlong, _c_p]),
}

STAGES = ["ana_contract", "ana_contract_phi", "ana_beta", "ana_alpha_czt", "ana_alpha_seg", "ana_alpha_direct",
          "syn_alpha_direct", "syn_alpha_czt", "syn_alpha_seg", "syn_beta", "syn_contract", "syn_contract_phi",
          "syn_reduce"]


class S2dwError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {s2dw_strerror(status)} ({status})")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libs2dw.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(rc: int, where: str):
    if rc != S2DW_OK:
        raise S2dwError(rc, where)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- C ABI, same names ------------------------------------------------------

def s2dw_strerror(status: int) -> str:
    return lib().s2dw_strerror(status).decode()


def s2dw_plan(L: int, N: int, lam: float, J0: int, flags: int) -> int:
    h = _c_p()
    _check(lib().s2dw_plan(ctypes.byref(h), L, N, float(lam), J0, flags), "s2dw_plan")
    return h.value


def s2dw_plan_destroy(plan: int) -> None:
    _check(lib().s2dw_plan_destroy(plan), "s2dw_plan_destroy")


def s2dw_query(plan: int) -> dict:
    J = ctypes.c_int()
    w, wp, ws, tot = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().s2dw_query(plan, ctypes.byref(J), ctypes.byref(w), ctypes.byref(wp), ctypes.byref(ws),
                            ctypes.byref(tot)), "s2dw_query")
    return {"J": J.value, "w_elems_per_scale": w.value, "wphi_elems": wp.value,
            "workspace_bytes": ws.value, "total_device_bytes": tot.value}


def s2dw_steer(plan: int, W, gammas, out, stream=None) -> None:
    """out[j][t] = W steered to orientation gammas[t] (Eq. (10))."""
    g = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64).ravel())
    _check(lib().s2dw_steer(plan, _ptr(W), g.ctypes.data_as(_c_dp), int(g.size), _ptr(out), _stream(stream)),
           "s2dw_steer")


def s2dw_sht_inverse(plan: int, flm, fpix, stream=None) -> None:
    """Pixel values on the DH sphere grid from f_lm (inverse SHT)."""
    _check(lib().s2dw_sht_inverse(plan, _ptr(flm), _ptr(fpix), _stream(stream)), "s2dw_sht_inverse")


def s2dw_sht_forward(plan: int, fpix, flm, stream=None) -> None:
    """f_lm from pixel values on the DH sphere grid (forward SHT, exact quadrature)."""
    _check(lib().s2dw_sht_forward(plan, _ptr(fpix), _ptr(flm), _stream(stream)), "s2dw_sht_forward")


def s2dw_scale_grid(plan: int, j: int):
    """(band-limit Lg, element offset in W, element count) of scale j's grid."""
    Lg, off, n = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().s2dw_scale_grid(plan, j, ctypes.byref(Lg), ctypes.byref(off), ctypes.byref(n)), "s2dw_scale_grid")
    return Lg.value, off.value, n.value


def s2dw_alpha_method(plan: int, j: int, direction: int):
    """(method, fft_len, segments, seg_len) of the alpha sums of scale j;
    direction 0 analysis, 1 synthesis; method 0 direct, 1 chirp-z,
    2 segmented chirp-z."""
    vals = [ctypes.c_int() for _ in range(4)]
    _check(lib().s2dw_alpha_method(plan, j, direction, *[ctypes.byref(v) for v in vals]), "s2dw_alpha_method")
    return tuple(v.value for v in vals)


def s2dw_launch_counts(plan: int):
    """(analysis, synthesis) kernel launches issued by one call of the plan."""
    a, s = ctypes.c_int(), ctypes.c_int()
    _check(lib().s2dw_launch_counts(plan, ctypes.byref(a), ctypes.byref(s)), "s2dw_launch_counts")
    return a.value, s.value


def s2dw_wait_timeouts() -> int:
    """Bounded waits in the library's kernels that gave up since the last
    call (0 in normal operation); synchronises the device.  The status
    S2DW_ETIMEOUT that accompanies a nonzero count is not raised: the count
    is the result."""
    c = ctypes.c_int()
    st = lib().s2dw_wait_timeouts(ctypes.byref(c))
    if st not in (0, -4):
        _check(st, "s2dw_wait_timeouts")
    return c.value


def s2dw_wait_probe(limit_cycles: int, stream=None) -> None:
    """One warp waits, at most limit_cycles SM cycles, on an mbarrier nothing
    arrives on and counts the give-up (the failure path of the bounded waits)."""
    _check(lib().s2dw_wait_probe(int(limit_cycles), _stream(stream)), "s2dw_wait_probe")


def s2dw_kernels(plan: int, J: int, L: int, N: int):
    psi = np.zeros((J + 1, L, N, 2), dtype=np.float64)
    phi = np.zeros(L, dtype=np.float64)
    _check(lib().s2dw_kernels(plan, psi.ctypes.data_as(_c_dp), phi.ctypes.data_as(_c_dp)), "s2dw_kernels")
    return psi[..., 0] + 1j * psi[..., 1], phi


def s2dw_analysis(plan: int, flm, W, Wphi, stream=None) -> None:
    _check(lib().s2dw_analysis(plan, _ptr(flm), _ptr(W), _ptr(Wphi), _stream(stream)), "s2dw_analysis")


def s2dw_synthesis(plan: int, W, Wphi, flm, stream=None) -> None:
    _check(lib().s2dw_synthesis(plan, _ptr(W), _ptr(Wphi), _ptr(flm), _stream(stream)), "s2dw_synthesis")


def _arr(vals):
    a = (_c_p * len(vals))()
    for i, v in enumerate(vals):
        a[i] = _ptr(v)
    return a


def s2dw_analysis_batch(plans: Sequence[int], flm, W, Wphi, stream=None) -> None:
    n = len(plans)
    _check(lib().s2dw_analysis_batch(_arr(plans), _arr(flm), _arr(W), _arr(Wphi), n, _stream(stream)),
           "s2dw_analysis_batch")


def s2dw_synthesis_batch(plans: Sequence[int], W, Wphi, flm, stream=None) -> None:
    n = len(plans)
    _check(lib().s2dw_synthesis_batch(_arr(plans), _arr(W), _arr(Wphi), _arr(flm), n, _stream(stream)),
           "s2dw_synthesis_batch")


def s2dw_scale_support(plan: int, j: int):
    lo, hi = ctypes.c_int(), ctypes.c_int()
    _check(lib().s2dw_scale_support(plan, j, ctypes.byref(lo), ctypes.byref(hi)), "s2dw_scale_support")
    return lo.value, hi.value


def s2dw_delta_slab(plan: int, l: int) -> np.ndarray:
    out = np.zeros((l + 1, l + 1), dtype=np.float64)
    _check(lib().s2dw_delta_slab(plan, l, out.ctypes.data_as(_c_dp)), "s2dw_delta_slab")
    return out


def s2dw_stage(plan: int, stage: int, j: int, complex_dtype) -> np.ndarray:
    nb = ctypes.c_int64()
    _check(lib().s2dw_stage(plan, stage, j, None, ctypes.byref(nb)), "s2dw_stage")
    out = np.zeros(nb.value // np.dtype(complex_dtype).itemsize, dtype=complex_dtype)
    _check(lib().s2dw_stage(plan, stage, j, out.ctypes.data, ctypes.byref(nb)), "s2dw_stage")
    return out


def s2dw_profile(plan: int, enable: bool) -> None:
    _check(lib().s2dw_profile(plan, 1 if enable else 0), "s2dw_profile")


def s2dw_profile_read(plan: int):
    """(per-stage summed ms, number of analysis calls, number of synthesis calls)."""
    ms = np.zeros(len(STAGES), dtype=np.float64)
    nc = (ctypes.c_int * 2)()
    _check(lib().s2dw_profile_read(plan, ms.ctypes.data_as(_c_dp), nc), "s2dw_profile_read")
    return dict(zip(STAGES, ms.tolist())), nc[0], nc[1]


def s2dw_delta_table_noalloc(Lmax: int, table64=None, table32=None, stream=None) -> int:
    """Number of table entries; with table64 given, builds the table into the
    caller's device buffers (no allocation by the library).

    The buffers are checked here before the C call (the library cannot see
    their sizes or types): table64 a contiguous float64 CUDA tensor of at
    least that many entries on the current device, table32 None or the same
    in float32.  ValueError otherwise."""
    n = ctypes.c_int64()
    if table64 is None:
        _check(lib().s2dw_delta_table_noalloc(Lmax, None, None, ctypes.byref(n), None), "s2dw_delta_table_noalloc")
        return n.value
    _check(lib().s2dw_delta_table_noalloc(Lmax, None, None, ctypes.byref(n), None), "s2dw_delta_table_noalloc")
    import torch
    dev = torch.cuda.current_device()
    for name, t, dt in (("table64", table64, torch.float64), ("table32", table32, torch.float32)):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < n.value:
            raise ValueError(f"{name} holds {t.numel()} entries, the table needs {n.value}")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    _check(lib().s2dw_delta_table_noalloc(Lmax, _ptr(table64), _ptr(table32), ctypes.byref(n), _stream(stream)),
           "s2dw_delta_table_noalloc")
    return n.value


def s2dw_plan_choices(plan: int):
    """The plan's launch methods (layout in include/s2dw.h)."""
    n = ctypes.c_int(0)
    _check(lib().s2dw_plan_choices(plan, None, ctypes.byref(n)), "s2dw_plan_choices")
    arr = (ctypes.c_int * n.value)()
    _check(lib().s2dw_plan_choices(plan, arr, ctypes.byref(n)), "s2dw_plan_choices")
    return list(arr)


def s2dw_plan_set_choices(plan: int, choices):
    arr = (ctypes.c_int * len(choices))(*[int(c) for c in choices])
    _check(lib().s2dw_plan_set_choices(plan, arr, len(choices)), "s2dw_plan_set_choices")


def s2dw_plan_tune(plan: int, reps: int = 5):
    """Times the candidate launch methods and applies the fastest; returns them."""
    n = ctypes.c_int(0)
    _check(lib().s2dw_plan_choices(plan, None, ctypes.byref(n)), "s2dw_plan_choices")
    arr = (ctypes.c_int * n.value)()
    _check(lib().s2dw_plan_tune(plan, reps, arr, ctypes.byref(n)), "s2dw_plan_tune")
    return list(arr)


_lib_fp = None


def lib_fingerprint() -> str:
    """Short hash of the loaded library file: tuned choices are cached per
    build, so that a rebuilt library is tuned again."""
    global _lib_fp
    if _lib_fp is None:
        import hashlib
        with open(LIB_PATH, "rb") as fh:
            _lib_fp = hashlib.sha1(fh.read()).hexdigest()[:12]
    return _lib_fp


def autotune_cache_path() -> str:
    """JSON file of tuned launch methods: $S2DW_AUTOTUNE_CACHE, else a file in
    the temporary directory."""
    import tempfile
    return os.environ.get("S2DW_AUTOTUNE_CACHE") or os.path.join(tempfile.gettempdir(), "s2dw_autotune.json")


# ---- thin object wrapper ----------------------------------------------------

class Plan:
    """A transform plan (owns the C plan handle).

    precision: "fp64" (complex128 f, float64 W) or "mixed" (complex64 f,
    float32 W).  Buffers are torch CUDA tensors; see ``alloc_*``.
    """

    def __init__(self, L: int, N: int, lam: float = 2.0, J0: int = 0, precision: str = "mixed",
                 multires: bool = False, mw: bool = False, autotune: bool = False):
        flags = (S2DW_FP64 if precision == "fp64" else S2DW_MIXED) | S2DW_REAL_SIGNAL
        if multires:
            flags |= S2DW_MULTIRES
        if mw:
            flags |= S2DW_MW
        if precision not in ("fp64", "mixed"):
            raise ValueError(precision)
        self.L, self.N, self.lam, self.J0, self.precision = L, N, float(lam), J0, precision
        self.multires = bool(multires)
        self.mw = bool(mw)
        self.nb = L if mw else 2 * L  # beta samples
        self.handle = s2dw_plan(L, N, lam, J0, flags)
        q = s2dw_query(self.handle)
        self.J = q["J"]
        self.nscale = self.J + 1
        self.info = q
        # (band-limit, offset, elements) of every scale's grid; last: scaling part
        self.grids = [s2dw_scale_grid(self.handle, j) for j in range(self.nscale + 1)]
        self.tuned = None
        if autotune:
            self.tuned = self.autotune()

    def tune_key(self) -> str:
        import torch
        return (f"{torch.cuda.get_device_name()}|L={self.L}|N={self.N}|lam={self.lam!r}|J0={self.J0}|"
                f"{self.precision}|multires={int(self.multires)}|mw={int(self.mw)}|lib={lib_fingerprint()}")

    def autotune(self, reps: int = 5):
        """Launch methods from the tuning cache, or tuned now (and cached);
        returns (choices, "cache" | "tuned")."""
        import json
        path = autotune_cache_path()
        key = self.tune_key()
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            try:
                s2dw_plan_set_choices(self.handle, cache[key])
                return cache[key], "cache"
            except S2dwError:
                pass  # stale entry (another build): tune again
        ch = s2dw_plan_tune(self.handle, reps)
        cache[key] = ch
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=0)
        os.replace(tmp, path)
        return ch, "tuned"

    def choices(self):
        return s2dw_plan_choices(self.handle)

    def set_choices(self, choices):
        s2dw_plan_set_choices(self.handle, choices)

    def close(self):
        if getattr(self, "handle", None):
            s2dw_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shapes and dtypes
    @property
    def w_shape(self):
        if self.multires:  # the scales one after the other, each [N][2Lg][2Lg-1]
            Lg, off, n = self.grids[self.nscale - 1]
            return (off + n,)
        return (self.nscale, self.N, self.nb, 2 * self.L - 1)

    @property
    def wphi_shape(self):
        Lg = self.grids[self.nscale][0]
        return (Lg if self.mw else 2 * Lg, 2 * Lg - 1)

    def w_scale(self, W, j):
        """View of scale j of W as [N][2Lg][2Lg-1]."""
        if not self.multires:
            return W[j]
        Lg, off, n = self.grids[j]
        return W[off:off + n].view(self.N, 2 * Lg, 2 * Lg - 1)

    def torch_dtypes(self):
        import torch
        return (torch.complex128, torch.float64) if self.precision == "fp64" else (torch.complex64, torch.float32)

    def alloc_flm(self, device="cuda"):
        import torch
        return torch.zeros(self.L * self.L, dtype=self.torch_dtypes()[0], device=device)

    def alloc_w(self, device="cuda"):
        import torch
        rd = self.torch_dtypes()[1]
        return torch.empty(self.w_shape, dtype=rd, device=device), torch.empty(self.wphi_shape, dtype=rd, device=device)

    def kernels(self):
        return s2dw_kernels(self.handle, self.J, self.L, self.N)

    def launch_counts(self):
        return s2dw_launch_counts(self.handle)

    def alloc_pix(self, device="cuda"):
        import torch
        return torch.empty((2 * self.L, 2 * self.L - 1), dtype=self.torch_dtypes()[1], device=device)

    def sht_inverse(self, flm, fpix, stream=None):
        s2dw_sht_inverse(self.handle, flm, fpix, stream)

    def sht_forward(self, fpix, flm, stream=None):
        s2dw_sht_forward(self.handle, fpix, flm, stream)

    def steer(self, W, gammas, out=None, stream=None):
        """W steered to the orientations `gammas` (Eq. (10)); allocates out if None."""
        import torch
        ng = len(np.atleast_1d(gammas))
        if out is None:
            shape = ((self.w_shape[0] // self.N) * ng,) if self.multires else \
                (self.J + 1, ng, self.nb, 2 * self.L - 1)
            out = torch.empty(shape, dtype=W.dtype, device=W.device)
        s2dw_steer(self.handle, W, gammas, out, stream)
        return out

    def analysis(self, flm, W, Wphi, stream=None):
        s2dw_analysis(self.handle, flm, W, Wphi, stream)

    def synthesis(self, W, Wphi, flm, stream=None):
        s2dw_synthesis(self.handle, W, Wphi, flm, stream)

    def alpha_method(self, j: int, direction: int):
        """(method, fft_len, segments, seg_len) of scale j's alpha sums (see s2dw_alpha_method)."""
        return s2dw_alpha_method(self.handle, j, direction)

    def support(self, j):
        return s2dw_scale_support(self.handle, j)

    def delta_slab(self, l):
        return s2dw_delta_slab(self.handle, l)

    def profile(self, enable=True):
        s2dw_profile(self.handle, enable)

    def profile_read(self):
        return s2dw_profile_read(self.handle)

    def stage(self, stage, j):
        cd = np.complex128 if self.precision == "fp64" else np.complex64
        return s2dw_stage(self.handle, stage, j, cd)
