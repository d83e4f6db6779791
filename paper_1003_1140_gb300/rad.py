"""ctypes binding of the C ABI in include/rad.h (argument marshalling only).

Every step of the diagnostic runs in the CUDA library ``librad.so``; this
module only converts arguments.  It raises if the library cannot be loaded:
there is no CPU fallback.  Arrays may be NumPy arrays (host), or torch
tensors on the CPU (pageable or pinned) or on the GPU.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

RAD_OK = 0
RAD_EINVAL = -1
RAD_ENOMEM = -2
RAD_ECUDA = -3
RAD_ESTEP = -4
RAD_EINCOMPLETE = -5
RAD_ETIMEOUT = -6
RAD_ENAN = -7
RAD_ESTATE = -8
RAD_ENOSPACE = -9

RAD_INCOHERENT = 0
RAD_COHERENT = 1
RAD_FP64 = 0
RAD_FP32_SPLIT = 1
RAD_VARIANT_AUTO = 0
RAD_VARIANT_SFU = 1
RAD_VARIANT_MIX = 2
RAD_VARIANT_PRECISE = 3

_ERRNAMES = {RAD_EINVAL: "RAD_EINVAL", RAD_ENOMEM: "RAD_ENOMEM", RAD_ECUDA: "RAD_ECUDA",
             RAD_ESTEP: "RAD_ESTEP", RAD_EINCOMPLETE: "RAD_EINCOMPLETE",
             RAD_ETIMEOUT: "RAD_ETIMEOUT", RAD_ENAN: "RAD_ENAN", RAD_ESTATE: "RAD_ESTATE"}

#: every symbol include/rad.h declares
EXPORTED = ("rad_init", "rad_set_options", "rad_get_options", "rad_accumulate",
            "rad_accumulate_steps", "rad_finalize", "rad_reset", "rad_spectrum_size",
            "rad_updates", "rad_timing", "rad_last_error", "rad_destroy",
            "rad_spectrum_noalloc", "rad_partial_sums", "rad_set_selectors", "rad_next_shard",
            "rad_spectrum_from_sums")


class RadError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class rad_species(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("charge", ctypes.c_double), ("mass", ctypes.c_double)]


class rad_window(ctypes.Structure):
    _fields_ = [("s0", ctypes.c_int64), ("s1", ctypes.c_int64), ("species_mask", ctypes.c_uint32),
                ("freq_grid", ctypes.c_int32), ("dir_set", ctypes.POINTER(ctypes.c_int32)),
                ("n_dir_set", ctypes.c_int32), ("reserved", ctypes.c_int32)]


RAD_SEL_BOX = 1
RAD_SEL_CONE = 2


class rad_selector(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("axis", ctypes.c_double * 3), ("theta_c", ctypes.c_double),
                ("dtheta", ctypes.c_double)]


class rad_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("anchor_K", ctypes.c_int32),
                ("freq_per_lane", ctypes.c_int32), ("defer", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("check_inputs", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("subcycle", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 8)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librad.so (building it first if needed); raise if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run build() first")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        lib.rad_init.restype = ctypes.c_int
        lib.rad_init.argtypes = [ctypes.POINTER(vp), dp, ctypes.c_int32, dp,
                                 ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.c_double,
                                 ctypes.POINTER(rad_species), ctypes.c_int32,
                                 ctypes.POINTER(rad_window), ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_double, vp]
        lib.rad_set_options.restype = ctypes.c_int
        lib.rad_set_options.argtypes = [vp, ctypes.POINTER(rad_options)]
        lib.rad_get_options.restype = ctypes.c_int
        lib.rad_get_options.argtypes = [vp, ctypes.POINTER(rad_options)]
        lib.rad_accumulate.restype = ctypes.c_int
        lib.rad_accumulate.argtypes = [vp, ctypes.c_int64, vp, vp]
        lib.rad_accumulate_steps.restype = ctypes.c_int
        lib.rad_accumulate_steps.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, vp, vp]
        lib.rad_finalize.restype = ctypes.c_int
        lib.rad_finalize.argtypes = [vp, vp]
        lib.rad_set_selectors.restype = ctypes.c_int
        lib.rad_set_selectors.argtypes = [vp, ctypes.POINTER(rad_selector), ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32)]
        lib.rad_partial_sums.restype = ctypes.c_int
        lib.rad_partial_sums.argtypes = [vp, vp]
        lib.rad_reset.restype = ctypes.c_int
        lib.rad_reset.argtypes = [vp]
        lib.rad_next_shard.restype = ctypes.c_int
        lib.rad_next_shard.argtypes = [vp]
        lib.rad_spectrum_from_sums.restype = ctypes.c_int
        lib.rad_spectrum_from_sums.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
        lib.rad_spectrum_size.restype = ctypes.c_int64
        lib.rad_spectrum_size.argtypes = [vp]
        lib.rad_updates.restype = ctypes.c_int64
        lib.rad_updates.argtypes = [vp]
        lib.rad_timing.restype = ctypes.c_int
        lib.rad_timing.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)]
        lib.rad_last_error.restype = ctypes.c_char_p
        lib.rad_last_error.argtypes = [vp]
        lib.rad_destroy.restype = None
        lib.rad_destroy.argtypes = [vp]
        _lib = lib
        return lib


def _ptr(a):
    """Raw pointer of a NumPy array or torch tensor (must be contiguous FP64)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous float64")
        return a.ctypes.data
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def spectrum_from_sums(sums, mode, out, stream=None):
    """rad_spectrum_from_sums on device tensors: the spectrum of the union of particle
    shards from the sum of their partial sums (sums [n] or [n, 4], out [n])."""
    lib = load()
    n = out.numel()
    if sums.numel() != n * (4 if mode == RAD_COHERENT else 1):
        raise ValueError("sums and out sizes do not match the summation mode")
    if stream is None:
        import torch
        st = torch.cuda.current_stream().cuda_stream
    else:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    rc = lib.rad_spectrum_from_sums(_ptr(sums), n, int(mode), _ptr(out), st)
    if rc != RAD_OK:
        raise RadError(rc, "rad_spectrum_from_sums failed")
    return out


class Radiation:
    """One radiation-diagnostic context (rad_init ... rad_destroy)."""

    def __init__(self, dirs, grids, dt, species, windows, mode=RAD_INCOHERENT,
                 precision=RAD_FP32_SPLIT, box_L=0.0, stream=None, options=None):
        """windows: (s0, s1, species_mask, grid) or (s0, s1, species_mask, grid,
        direction indices) -- the optional fifth element is the window's subset of
        `dirs`, whose spectra it returns in that order."""
        self._lib = load()
        self._h = ctypes.c_void_p()
        dirs = np.ascontiguousarray(np.reshape(dirs, (-1, 3)), dtype=np.float64)
        grids = [np.ascontiguousarray(np.atleast_1d(g), dtype=np.float64) for g in grids]
        freqs = np.ascontiguousarray(np.concatenate(grids))
        glen = (ctypes.c_int32 * len(grids))(*[len(g) for g in grids])
        sp = (rad_species * len(species))()
        for i, s in enumerate(species):
            count, charge = s[0], s[1]
            mass = s[2] if len(s) > 2 else 1.0
            sp[i] = rad_species(int(count), float(charge), float(mass))
        wn = (rad_window * len(windows))()
        keep = []              # direction-set arrays stay alive until rad_init has copied them
        self.window_dirs = []
        for i, wdef in enumerate(windows):
            s0, s1, mask, g = wdef[:4]
            dset = wdef[4] if len(wdef) > 4 else None
            wn[i] = rad_window(int(s0), int(s1), int(mask), int(g))
            if dset is not None:
                arr = (ctypes.c_int32 * len(dset))(*[int(d) for d in dset])
                keep.append(arr)
                wn[i].dir_set = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32))
                wn[i].n_dir_set = len(dset)
                self.window_dirs.append(len(dset))
            else:
                self.window_dirs.append(dirs.shape[0])
        if stream is None:
            st = None
        elif isinstance(stream, int):
            st = stream
        else:
            st = stream.cuda_stream
        dp = ctypes.POINTER(ctypes.c_double)
        rc = self._lib.rad_init(ctypes.byref(self._h), dirs.ctypes.data_as(dp), dirs.shape[0],
                                freqs.ctypes.data_as(dp), glen, len(grids), float(dt), sp,
                                len(species), wn, len(windows), int(mode), int(precision),
                                float(box_L), st)
        if rc != RAD_OK:
            self._h = None
            raise RadError(rc, "rad_init failed")
        self.n_windows = len(windows)
        self.mode = int(mode)
        self.D = dirs.shape[0]
        self.grid_lens = [len(grids[w[3]]) for w in windows]
        del keep
        if options:
            self.set_options(**options)

    # -- helpers
    def _check(self, rc):
        if rc != RAD_OK:
            msg = self._lib.rad_last_error(self._h).decode()
            raise RadError(rc, msg)

    def set_options(self, **kw):
        o = rad_options()
        for k, v in kw.items():
            if k == "time_ingest":
                o.reserved[0] = int(v)
            elif k == "poly_per_lane":
                o.reserved[1] = int(v)
            elif k == "host_stage_mib":
                o.reserved[2] = int(v)
            elif k == "phase_budget":
                # radians per update, passed as whole nanoradians
                o.reserved[3] = int(round(float(v) * 1e9))
            else:
                setattr(o, k, int(v))
        self._check(self._lib.rad_set_options(self._h, ctypes.byref(o)))

    def set_selectors(self, selectors, window_selector):
        """selectors: list of dicts {"kind": "box", "lo": [...], "hi": [...]} or
        {"kind": "cone", "axis": [...], "theta_c": a, "dtheta": d};
        window_selector: per window, a selector index or -1."""
        arr = (rad_selector * max(1, len(selectors)))()
        for i, sdef in enumerate(selectors):
            r = rad_selector()
            if sdef["kind"] == "box":
                r.kind = RAD_SEL_BOX
                r.lo[:] = [float(v) for v in sdef["lo"]]
                r.hi[:] = [float(v) for v in sdef["hi"]]
            else:
                r.kind = RAD_SEL_CONE
                r.axis[:] = [float(v) for v in sdef["axis"]]
                r.theta_c = float(sdef["theta_c"])
                r.dtheta = float(sdef["dtheta"])
            arr[i] = r
        ws = (ctypes.c_int32 * len(window_selector))(*[int(v) for v in window_selector])
        self._check(self._lib.rad_set_selectors(self._h, arr, len(selectors), ws))

    def options(self) -> dict:
        o = rad_options()
        self._check(self._lib.rad_get_options(self._h, ctypes.byref(o)))
        out = {f: getattr(o, f) for f, _ in rad_options._fields_ if f != "reserved"}
        out["poly_per_lane"] = int(o.reserved[1])
        out["phase_budget"] = o.reserved[3] * 1e-9
        return out

    def accumulate(self, step, x, u):
        self._check(self._lib.rad_accumulate(self._h, int(step), _ptr(x), _ptr(u)))

    def accumulate_steps(self, step0, x, u):
        n = x.shape[0]
        self._check(self._lib.rad_accumulate_steps(self._h, int(step0), int(n), _ptr(x), _ptr(u)))

    def spectrum_size(self) -> int:
        return int(self._lib.rad_spectrum_size(self._h))

    def updates(self) -> int:
        return int(self._lib.rad_updates(self._h))

    def finalize(self, out=None):
        """Return the spectra: list of [D, len(grid)] arrays (or fill `out`)."""
        n = self.spectrum_size()
        host = out is None
        if host:
            out = np.empty(n, dtype=np.float64)
        self._check(self._lib.rad_finalize(self._h, _ptr(out)))
        if not host:
            return out
        res, off = [], 0
        for nd, L in zip(self.window_dirs, self.grid_lens):
            res.append(out[off:off + nd * L].reshape(nd, L))
            off += nd * L
        return res

    def partial_sums(self, out=None):
        """Unscaled FP64 particle sums (see rad_partial_sums): [n_bins] or [n_bins, 4]."""
        n = self.spectrum_size() * (4 if self.mode == RAD_COHERENT else 1)
        host = out is None
        if host:
            out = np.empty(n, dtype=np.float64)
        self._check(self._lib.rad_partial_sums(self._h, _ptr(out)))
        return out.reshape(-1, 4) if (host and self.mode == RAD_COHERENT) else out

    def reset(self):
        self._check(self._lib.rad_reset(self._h))

    def next_shard(self):
        """Start a further particle shard: steps restart at 0, sums are kept."""
        self._check(self._lib.rad_next_shard(self._h))

    def timing(self):
        a = ctypes.c_double()
        g = ctypes.c_double()
        na = ctypes.c_int64()
        ng = ctypes.c_int64()
        self._check(self._lib.rad_timing(self._h, ctypes.byref(a), ctypes.byref(g),
                                         ctypes.byref(na), ctypes.byref(ng)))
        return {"accum_ms": a.value, "ingest_ms": g.value, "accum_launches": na.value,
                "ingest_launches": ng.value}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rad_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
