"""GB300 (sm_103a) energies, forces and MD for the Allegro potential of Allegro-FM
(arXiv 2502.06073).

A thin ctypes binding of the C ABI in include/ff.h: every step of the path (neighbour
lists, edge features, MLPs, tensor products, adjoint, force gather, velocity Verlet) runs
in the library's CUDA kernels.  PyTorch only supplies device memory and streams, and
`FFEnergy` exposes the hand-written adjoint as a torch.autograd.Function.

There is no CPU fallback: importing works without a GPU (for building and introspection),
but every compute call raises if the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LIB_PATH = _build.LIB

FF_OK = 0
ERRORS = {-1: "FF_ERR_ARG", -2: "FF_ERR_SPECIES", -3: "FF_ERR_OOM", -4: "FF_ERR_CUDA",
          -5: "FF_ERR_CAPACITY", -6: "FF_ERR_NONFINITE", -7: "FF_ERR_STATE", -8: "FF_ERR_BOX",
          -9: "FF_ERR_TIMEOUT"}

# Every function the C ABI exports (include/ff.h).
ABI = ("ff_create", "ff_destroy", "ff_neighbors", "ff_energy_forces", "ff_forces",
       "ff_md_step", "ff_export_params", "ff_get_edges", "ff_kernel_launches", "ff_last_error",
       "ff_profile_enable", "ff_profile_read", "ff_profile_class", "ff_neighbors_noalloc",
       "ff_energy_forces_graph", "ff_set_graph", "ff_autotune", "ff_virial", "ff_md_nvt",
       "ff_set_tiles")


class HParams(ctypes.Structure):
    _fields_ = [("rc", ctypes.c_float), ("skin", ctypes.c_float),
                ("n_basis", ctypes.c_int), ("poly_p", ctypes.c_int), ("lmax", ctypes.c_int),
                ("parity", ctypes.c_int), ("n_layers", ctypes.c_int), ("channels", ctypes.c_int),
                ("two_body", ctypes.c_int * 4), ("n_two_body", ctypes.c_int),
                ("latent", ctypes.c_int * 4), ("n_latent", ctypes.c_int),
                ("edge_eng", ctypes.c_int * 2), ("n_edge_eng", ctypes.c_int),
                ("avg_num_neighbors", ctypes.c_float), ("precision", ctypes.c_int)]


class FFError(RuntimeError):
    pass


_lib = None


def load_library(path: str | None = None):
    """Load libff.so (building it first if it is missing); raises if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.ff_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(HParams), ctypes.c_uint64]
    lib.ff_destroy.argtypes = [vp]
    lib.ff_destroy.restype = None
    lib.ff_neighbors.argtypes = [vp, vp, vp, i32, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int), vp, i32, vp]
    lib.ff_energy_forces.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ff_energy_forces_graph.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ff_set_graph.argtypes = [vp, i32]
    lib.ff_set_tiles.argtypes = [vp, i32, i32]
    lib.ff_virial.argtypes = [vp, vp, vp]
    lib.ff_md_nvt.argtypes = [vp, vp, vp, vp, i32, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, vp, vp, vp, vp, vp]
    lib.ff_autotune.argtypes = [vp, vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(ctypes.c_double), vp]
    lib.ff_forces.argtypes = [vp, vp, vp, vp]
    lib.ff_md_step.argtypes = [vp, vp, vp, vp, i32, ctypes.c_double, vp, vp, vp]
    lib.ff_export_params.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.ff_get_edges.argtypes = [vp, ctypes.POINTER(i64), vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.ff_kernel_launches.argtypes = [vp]
    lib.ff_kernel_launches.restype = i64
    lib.ff_last_error.argtypes = [vp]
    lib.ff_last_error.restype = ctypes.c_char_p
    lib.ff_profile_enable.argtypes = [i32]
    lib.ff_profile_read.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
    lib.ff_profile_class.argtypes = [i32]
    lib.ff_profile_class.restype = ctypes.c_char_p
    lib.ff_neighbors_noalloc.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_float, vp, vp,
                                         vp, i64, ctypes.POINTER(i64), ctypes.c_char_p,
                                         ctypes.c_size_t, vp]
    for name in ABI:
        getattr(lib, name)
    _lib = lib
    return lib


def hparams_struct(hp: dict, precision: int = 0) -> HParams:
    h = HParams()
    h.rc = float(hp["rc"])
    h.skin = float(hp.get("skin", 0.0))
    h.n_basis = int(hp["n_basis"])
    h.poly_p = int(hp["poly_p"])
    h.lmax = int(hp["lmax"])
    h.parity = int(hp.get("parity", 1))
    h.n_layers = int(hp["n_layers"])
    h.channels = int(hp["channels"])
    for name in ("two_body", "latent", "edge_eng"):
        arr = list(hp[name])
        cap = 2 if name == "edge_eng" else 4
        if len(arr) > cap:
            raise ValueError(f"{name} has more than {cap} entries")
        fld = getattr(h, name)
        for k, w in enumerate(arr):
            fld[k] = int(w)
        setattr(h, "n_" + name, len(arr))
    h.avg_num_neighbors = float(hp["avg_num_neighbors"])
    h.precision = int(precision)
    return h


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise FFError("a CUDA device is required (this library has no CPU path)")
    return torch


def _stream(torch):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class FFModel:
    """One potential (weights drawn from `seed`) bound to at most one system at a time."""

    def __init__(self, hp: dict, seed: int = 42, precision: int = 0):
        self.lib = load_library()
        self.hp = dict(hp)
        self.seed = seed
        self.precision = precision
        self._h = ctypes.c_void_p()
        st = hparams_struct(hp, precision)
        rc = self.lib.ff_create(ctypes.byref(self._h), ctypes.byref(st), ctypes.c_uint64(seed))
        self._check(rc, create=True)
        self.n = 0
        self.n_sys = 0

    def _check(self, rc, create=False):
        if rc != FF_OK:
            msg = self.lib.ff_last_error(None if create else self._h)
            raise FFError(f"{ERRORS.get(rc, rc)}: {msg.decode() if msg else ''}")

    def close(self):
        if self._h:
            self.lib.ff_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- system
    def bind(self, pos, Z, box, pbc, sys_ptr=None):
        """Bind a system: pos (cuda float64 [n,3]), Z (cuda int32 [n]), box [3], pbc [3]."""
        torch = _torch()
        pos = pos.contiguous()
        Z = Z.to(torch.int32).contiguous()
        n = pos.shape[0]
        b = (ctypes.c_double * 3)(*[float(x) for x in box])
        p = (ctypes.c_int * 3)(*[int(bool(x)) for x in pbc])
        if sys_ptr is None:
            sp, ns = None, 1
        else:
            arr = np.ascontiguousarray(np.asarray(sys_ptr, dtype=np.int32))
            self._sys_ptr_keep = arr
            sp, ns = ctypes.c_void_p(arr.ctypes.data), arr.shape[0] - 1
        rc = self.lib.ff_neighbors(self._h, _ptr(pos), _ptr(Z), n, b, p, sp, ns, _stream(torch))
        self._check(rc)
        self.n, self.n_sys = n, ns
        self._Z = Z
        return self

    def energy_forces(self, pos, forces=True, E_atom=True):
        torch = _torch()
        pos = pos.contiguous()
        dev = pos.device
        Es = torch.empty(self.n_sys, dtype=torch.float64, device=dev)
        Ea = torch.empty(self.n, dtype=torch.float32, device=dev) if E_atom else None
        F = torch.empty(self.n, 3, dtype=torch.float32, device=dev) if forces else None
        rc = self.lib.ff_energy_forces(self._h, _ptr(pos), _ptr(Es), _ptr(Ea), _ptr(F),
                                       _stream(torch))
        self._check(rc)
        return Es, Ea, F

    def energy_forces_graph(self, pos, Es=None, Ea=None, F=None):
        """E (+F) on the frozen Verlet list through a captured CUDA graph.  Pass the same
        output tensors on every call to replay the graph (new tensors recapture)."""
        torch = _torch()
        dev = pos.device
        Es = Es if Es is not None else torch.empty(self.n_sys, dtype=torch.float64, device=dev)
        rc = self.lib.ff_energy_forces_graph(self._h, _ptr(pos), _ptr(Es), _ptr(Ea), _ptr(F),
                                             _stream(torch))
        self._check(rc)
        return Es, Ea, F

    def autotune(self, pos) -> dict:
        """Pick the fastest tensor-core GEMM tile configuration for the bound system."""
        torch = _torch()
        sl, st, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.ff_autotune(self._h, _ptr(pos), ctypes.byref(sl), ctypes.byref(st),
                                         ctypes.byref(ms), _stream(torch)))
        return {"slice": sl.value, "stages": st.value, "ms_per_evaluation": ms.value}

    def virial(self):
        """Per-system virial W = -sum_e r_e (x) dE/dr_e, shape [n_sys, 3, 3] (eV)."""
        torch = _torch()
        W = torch.empty(self.n_sys, 3, 3, dtype=torch.float64, device="cuda")
        self._check(self.lib.ff_virial(self._h, _ptr(W), _stream(torch)))
        return W

    def set_tiles(self, slice: int, stages: int):
        """Select the tensor-core GEMM tile configuration (see ff_set_tiles)."""
        self._check(self.lib.ff_set_tiles(self._h, int(slice), int(stages)))

    def set_graph(self, enable: bool = True):
        """Make md() replay a captured CUDA graph on a frozen Verlet list."""
        self._check(self.lib.ff_set_graph(self._h, 1 if enable else 0))

    def forces_adjoint(self, grad_E=None):
        torch = _torch()
        F = torch.empty(self.n, 3, dtype=torch.float32, device="cuda")
        g = None if grad_E is None else grad_E.to(torch.float64).contiguous()
        rc = self.lib.ff_forces(self._h, _ptr(g), _ptr(F), _stream(torch))
        self._check(rc)
        return F

    def energy(self, pos):
        """Per-system energies with autograd: d(E)/d(pos) runs the CUDA adjoint."""
        return FFEnergy.apply(pos, self)

    def md(self, x, v, mass, n_steps, dt_fs, energies=True):
        torch = _torch()
        Ep = Ek = None
        if energies:
            Ep = torch.empty(n_steps * self.n_sys, dtype=torch.float64, device=x.device)
            Ek = torch.empty(n_steps * self.n_sys, dtype=torch.float64, device=x.device)
        rc = self.lib.ff_md_step(self._h, _ptr(x), _ptr(v), _ptr(mass), int(n_steps),
                                 float(dt_fs), _ptr(Ep), _ptr(Ek), _stream(torch))
        self._check(rc)
        return Ep, Ek

    def md_nvt(self, x, v, mass, n_steps, dt_fs, T, tau_fs, thermo=None):
        """Nose-Hoover NVT steps; thermo (cuda float64 [n_sys, 2]) carries (xi, eta)."""
        torch = _torch()
        if thermo is None:
            thermo = torch.zeros(self.n_sys, 2, dtype=torch.float64, device=x.device)
        out = [torch.empty(n_steps * self.n_sys, dtype=torch.float64, device=x.device)
               for _ in range(3)]
        rc = self.lib.ff_md_nvt(self._h, _ptr(x), _ptr(v), _ptr(mass), int(n_steps),
                                float(dt_fs), float(T), float(tau_fs), _ptr(thermo),
                                _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _stream(torch))
        self._check(rc)
        return out[0], out[1], out[2], thermo

    # ---------------------------------------------------------------- introspection
    def export_params(self) -> np.ndarray:
        need = ctypes.c_size_t()
        self._check(self.lib.ff_export_params(self._h, None, 0, ctypes.byref(need)))
        buf = np.empty(need.value, dtype=np.float64)
        self._check(self.lib.ff_export_params(self._h, ctypes.c_void_p(buf.ctypes.data),
                                              need.value, ctypes.byref(need)))
        return buf

    def edges(self):
        torch = _torch()
        ne = ctypes.c_int64()
        self._check(self.lib.ff_get_edges(self._h, ctypes.byref(ne), None, None, None, None, 0,
                                          _stream(torch)))
        E = ne.value
        rp = np.empty(self.n + 1, np.int32)
        col = np.empty(max(E, 1), np.int32)
        sh = np.empty((max(E, 1), 3), np.int32)
        rev = np.empty(max(E, 1), np.int32)
        self._check(self.lib.ff_get_edges(
            self._h, ctypes.byref(ne), ctypes.c_void_p(rp.ctypes.data),
            ctypes.c_void_p(col.ctypes.data), ctypes.c_void_p(sh.ctypes.data),
            ctypes.c_void_p(rev.ctypes.data), max(E, 1), _stream(torch)))
        return rp, col[:E], sh[:E], rev[:E]

    def launches(self) -> int:
        return int(self.lib.ff_kernel_launches(self._h))


def profile_enable(on: bool = True) -> None:
    """Bracket every kernel launch with CUDA events (see ff_profile_enable)."""
    lib = load_library()
    if lib.ff_profile_enable(1 if on else 0) != FF_OK:
        raise FFError("ff_profile_enable failed")


def profile_read() -> dict:
    """{kernel class: (launches, device ms)} since the last read (synchronises)."""
    lib = load_library()
    cap = 64
    la = np.zeros(cap, np.int64)
    ms = np.zeros(cap, np.float64)
    n = ctypes.c_int()
    rc = lib.ff_profile_read(ctypes.c_void_p(la.ctypes.data), ctypes.c_void_p(ms.ctypes.data),
                             cap, ctypes.byref(n))
    if rc != FF_OK:
        raise FFError(f"ff_profile_read failed ({ERRORS.get(rc, rc)})")
    return {lib.ff_profile_class(k).decode(): (int(la[k]), float(ms[k])) for k in range(n.value)}


def _make_energy_fn():
    import torch

    class FFEnergy(torch.autograd.Function):
        """E_sys(pos) whose backward is the library's hand-written adjoint (ff_forces)."""

        @staticmethod
        def forward(ctx, pos, model):
            Es, _, _ = model.energy_forces(pos, forces=False, E_atom=False)
            ctx.model = model
            return Es

        @staticmethod
        def backward(ctx, gE):
            F = ctx.model.forces_adjoint(gE)
            return (-F).to(torch.float64), None

    return FFEnergy


class _LazyFn:
    _fn = None

    def apply(self, *a):
        if _LazyFn._fn is None:
            _LazyFn._fn = _make_energy_fn()
        return _LazyFn._fn.apply(*a)


FFEnergy = _LazyFn()
