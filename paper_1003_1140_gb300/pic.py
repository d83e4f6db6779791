"""ctypes binding of include/rad_pic.h (argument marshalling only): the small
live 2D3V PIC of the two-stream setup that drives the diagnostic in situ."""
from __future__ import annotations

import ctypes

import numpy as np

from . import rad as _rad

RAD_PIC_OK = 0
EXPORTED = ("rad_pic_init", "rad_pic_set_fields", "rad_pic_get_fields", "rad_pic_get_particles",
            "rad_pic_step", "rad_pic_steps_done", "rad_pic_tracked", "rad_pic_run_coupled",
            "rad_pic_energy", "rad_pic_last_error", "rad_pic_destroy")


class rad_pic_species(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("charge", ctypes.c_double),
                ("mass", ctypes.c_double), ("weight", ctypes.c_double)]


def _lib():
    lib = _rad.load()
    if not getattr(lib, "_pic_bound", False):
        vp = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.rad_pic_init.restype = ctypes.c_int
        lib.rad_pic_init.argtypes = [ctypes.POINTER(vp), i32, f64, f64,
                                     ctypes.POINTER(rad_pic_species), i32, vp, vp, vp]
        for name in ("rad_pic_set_fields", "rad_pic_get_fields", "rad_pic_get_particles"):
            getattr(lib, name).restype = ctypes.c_int
            getattr(lib, name).argtypes = [vp, vp, vp]
        lib.rad_pic_step.restype = ctypes.c_int
        lib.rad_pic_step.argtypes = [vp, i32]
        lib.rad_pic_steps_done.restype = i64
        lib.rad_pic_steps_done.argtypes = [vp]
        lib.rad_pic_tracked.restype = ctypes.c_int
        lib.rad_pic_tracked.argtypes = [vp, i64, i64, vp, vp]
        lib.rad_pic_run_coupled.restype = ctypes.c_int
        lib.rad_pic_run_coupled.argtypes = [vp, vp, i64, i64, i32]
        lib.rad_pic_energy.restype = ctypes.c_int
        lib.rad_pic_energy.argtypes = [vp, ctypes.POINTER(f64), ctypes.POINTER(f64)]
        lib.rad_pic_last_error.restype = ctypes.c_char_p
        lib.rad_pic_last_error.argtypes = [vp]
        lib.rad_pic_destroy.restype = None
        lib.rad_pic_destroy.argtypes = [vp]
        lib._pic_bound = True
    return lib


class Pic:
    """species: [(count, charge, mass, weight)] in particle order; x, u [3][N]
    FP64 (host or device) initial state x_0, u_{-1/2}."""

    def __init__(self, n, d, dt, species, x, u, stream=None):
        self._lib = _lib()
        self.n, self.d, self.dt = int(n), float(d), float(dt)
        self.N = int(sum(int(s[0]) for s in species))
        sp = (rad_pic_species * max(1, len(species)))()
        for i, (c, q, m, w) in enumerate(species):
            sp[i] = rad_pic_species(int(c), float(q), float(m), float(w))
        st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        self.h = ctypes.c_void_p()
        rc = self._lib.rad_pic_init(ctypes.byref(self.h), self.n, self.d, self.dt, sp,
                                    len(species), _rad._ptr(x), _rad._ptr(u), st)
        if rc != RAD_PIC_OK:
            raise RuntimeError(f"rad_pic_init failed ({rc})")

    @classmethod
    def two_stream(cls, ts, stream=None):
        """From a trajgen.TwoStream setup (electrons first, then partners)."""
        X, U, q, m, w = ts.particles()
        ne = X.shape[1] // 2
        species = [(ne, -1.0, 1.0, float(w[0])), (ne, 1.0, float(ts.mass_ratio), float(w[0]))]
        return cls(ts.n, ts.d, ts.dt, species, np.ascontiguousarray(X), np.ascontiguousarray(U),
                   stream)

    def _chk(self, rc, what):
        if rc != RAD_PIC_OK:
            raise RuntimeError(f"{what} failed ({rc}): "
                               f"{self._lib.rad_pic_last_error(self.h).decode(errors='replace')}")

    def set_fields(self, E=None, B=None):
        self._chk(self._lib.rad_pic_set_fields(self.h, _rad._ptr(E), _rad._ptr(B)),
                  "rad_pic_set_fields")

    def fields(self):
        E = np.empty((3, self.n, self.n))
        B = np.empty((3, self.n, self.n))
        self._chk(self._lib.rad_pic_get_fields(self.h, _rad._ptr(E), _rad._ptr(B)),
                  "rad_pic_get_fields")
        return E, B

    def particles(self):
        x = np.empty((3, self.N))
        u = np.empty((3, self.N))
        self._chk(self._lib.rad_pic_get_particles(self.h, _rad._ptr(x), _rad._ptr(u)),
                  "rad_pic_get_particles")
        return x, u

    def step(self, n_steps=1):
        self._chk(self._lib.rad_pic_step(self.h, int(n_steps)), "rad_pic_step")

    @property
    def steps_done(self) -> int:
        return int(self._lib.rad_pic_steps_done(self.h))

    def tracked(self, first, count, x_out, u_out):
        self._chk(self._lib.rad_pic_tracked(self.h, int(first), int(count), _rad._ptr(x_out),
                                            _rad._ptr(u_out)), "rad_pic_tracked")

    def run_coupled(self, radiation, first, count, n_steps):
        self._chk(self._lib.rad_pic_run_coupled(self.h, radiation._h, int(first), int(count),
                                                int(n_steps)), "rad_pic_run_coupled")

    def energy(self):
        f, k = ctypes.c_double(), ctypes.c_double()
        self._chk(self._lib.rad_pic_energy(self.h, ctypes.byref(f), ctypes.byref(k)),
                  "rad_pic_energy")
        return f.value, k.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.rad_pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
