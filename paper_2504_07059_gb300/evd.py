"""Python binding of libevd's C ABI (``include/evd.h``).

Argument marshalling only: every function below has the name of the C entry
point it calls, converts numpy arrays / torch tensors / integers into the
plain pointers the ABI takes, and raises :class:`EVDError` on a non-OK status.
All computation happens in the CUDA kernels of libevd.  PyTorch is used only
for device memory and streams; there is no CPU fallback, and a missing
library is an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

EVD_OK, EVD_ERR_ARG, EVD_ERR_CUDA, EVD_ERR_UNSTABLE, EVD_ERR_TIMEOUT, EVD_ERR_STATE = range(6)
EVD_D2Q9, EVD_D3Q19 = 0, 1
EVD_FP64, EVD_FP32, EVD_FP16_STORE = 0, 1, 2
EVD_WALL_XM, EVD_WALL_XP, EVD_WALL_YM, EVD_WALL_YP, EVD_WALL_ZM, EVD_WALL_ZP = (1, 2, 4, 8, 16, 32)
EVD_MAX_SPECIES = 6
EVD_MAX_SPECIES_D3Q19 = 3
EVD_KERNEL_AUTO, EVD_KERNEL_GENERAL, EVD_KERNEL_TMA = 0, 1, 2
EVD_ADJOINT_REVERSE, EVD_ADJOINT_DUAL = 0, 1
EVD_FORCE_S_DIFF, EVD_FORCE_S_P, EVD_FORCE_S_RHO = 1, 2, 4
EVD_REF_AUTO, EVD_REF_SPECIES, EVD_REF_NODE = 0, 1, 2

STATUS_NAMES = {0: "EVD_OK", 1: "EVD_ERR_ARG", 2: "EVD_ERR_CUDA", 3: "EVD_ERR_UNSTABLE",
                4: "EVD_ERR_TIMEOUT", 5: "EVD_ERR_STATE"}
PRECISIONS = {"fp64": EVD_FP64, "fp32": EVD_FP32, "fp16": EVD_FP16_STORE}


class EVDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class evd_grid(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("precision", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("wall_mask", ctypes.c_uint)]


class evd_species(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int),
                ("molar_mass", ctypes.POINTER(ctypes.c_double)),
                ("diffusivity", ctypes.POINTER(ctypes.c_double)),
                ("tau1", ctypes.c_double),
                ("g", ctypes.c_double * 3),
                ("flags", ctypes.c_uint)]


class evd_member(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("wall_mask", ctypes.c_uint), ("species", evd_species)]


_lock = threading.Lock()
_lib = None
_vp, _dp, _st = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int

_SIGNATURES = {
    "evd_version": (ctypes.c_int, []),
    "evd_required_bytes": (ctypes.c_size_t, [ctypes.POINTER(evd_grid), ctypes.POINTER(evd_species)]),
    "evd_create": (_st, [ctypes.POINTER(evd_grid), ctypes.POINTER(evd_species), _vp, ctypes.POINTER(_vp)]),
    "evd_create_with_buffers": (_st, [ctypes.POINTER(evd_grid), ctypes.POINTER(evd_species), _vp, _vp, _vp,
                                      ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "evd_set_stream": (_st, [_vp, _vp]),
    "evd_set_fields": (_st, [_vp, _vp, _vp]),
    "evd_set_fields_device": (_st, [_vp, _vp, _vp]),
    "evd_set_populations": (_st, [_vp, _vp]),
    "evd_step": (_st, [_vp, ctypes.c_longlong]),
    "evd_readout_device": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "evd_get_mole_fractions": (_st, [_vp, _vp]),
    "evd_get_densities": (_st, [_vp, _vp]),
    "evd_get_velocities": (_st, [_vp, _vp, _vp]),
    "evd_get_species_mass": (_st, [_vp, _vp]),
    "evd_species_mass_device": (_st, [_vp, _vp]),
    "evd_get_populations": (_st, [_vp, _vp]),
    "evd_time": (ctypes.c_longlong, [_vp]),
    "evd_check": (_st, [_vp]),
    "evd_launch_count": (ctypes.c_longlong, [_vp]),
    "evd_set_kernel": (_st, [_vp, ctypes.c_int]),
    "evd_get_kernel": (ctypes.c_int, [_vp]),
    "evd_set_tile_rows": (_st, [_vp, ctypes.c_int]),
    "evd_set_adjoint_mode": (_st, [_vp, ctypes.c_int]),
    "evd_set_adjoint_forward": (_st, [_vp, ctypes.c_int]),
    "evd_set_force_field": (_st, [_vp, _vp]),
    "evd_loss_gradient": (_st, [_vp, _vp, _vp, ctypes.c_longlong, _vp, ctypes.c_int, _vp, _vp, _vp]),
    "evd_set_mass_correction": (_st, [_vp, ctypes.c_int]),
    "evd_set_wait_limit": (_st, [_vp, ctypes.c_int]),
    "evd_set_reference_mode": (_st, [_vp, ctypes.c_int]),
    "evd_get_reference_mode": (ctypes.c_int, [_vp]),
    "evd_get_target_mass": (_st, [_vp, _vp]),
    "evd_population_mass_noalloc": (_st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, _vp, _vp]),
    "evd_fma_rate": (_st, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           _vp]),
    "evd_destroy": (_st, [_vp]),
    "evd_last_error": (ctypes.c_char_p, [_vp]),
    # include/evd_batch.h
    "evd_batch_create": (_st, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(evd_member), ctypes.c_int, _vp,
                               ctypes.POINTER(_vp)]),
    "evd_batch_sizes": (_st, [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "evd_batch_set_fields": (_st, [_vp, _vp, _vp]),
    "evd_batch_step": (_st, [_vp, ctypes.c_longlong]),
    "evd_batch_readout_device": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "evd_batch_get_mole_fractions": (_st, [_vp, _vp]),
    "evd_batch_get_densities": (_st, [_vp, _vp]),
    "evd_batch_get_velocities": (_st, [_vp, _vp, _vp]),
    "evd_batch_get_species_mass": (_st, [_vp, _vp]),
    "evd_batch_set_schedule": (_st, [_vp, ctypes.c_int, ctypes.c_int]),
    "evd_batch_get_schedule": (_st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "evd_batch_autotune": (_st, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "evd_batch_set_graph": (_st, [_vp, ctypes.c_int]),
    "evd_batch_set_mass_correction": (_st, [_vp, ctypes.c_int]),
    "evd_batch_time": (ctypes.c_longlong, [_vp]),
    "evd_batch_launch_count": (ctypes.c_longlong, [_vp]),
    "evd_batch_check": (_st, [_vp]),
    "evd_batch_destroy": (_st, [_vp]),
    "evd_batch_last_error": (ctypes.c_char_p, [_vp]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libevd.  Raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libevd is not built ({path} missing); run "
                                   "paper_2504_07059_gb300.build.build() first")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != EVD_OK:
        msg = lib().evd_last_error(ctx)
        raise EVDError(status, msg.decode() if msg else "")


def _bcheck(status: int, batch=None):
    if status != EVD_OK:
        msg = lib().evd_batch_last_error(batch)
        raise EVDError(status, msg.decode() if msg else "")


def _ptr(a, nelem: int | None = None, writable: bool = False):
    """Pointer of a float64 buffer: numpy array, torch tensor or raw int."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous float64")
        if writable and not a.flags.writeable:
            raise TypeError("output array is read-only")
        if nelem is not None and a.size < nelem:
            raise ValueError(f"array has {a.size} elements, needs {nelem}")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):  # torch tensor (host or device)
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        if nelem is not None and a.numel() < nelem:
            raise ValueError(f"tensor has {a.numel()} elements, needs {nelem}")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def make_grid(lattice: int, precision: int, shape, wall_mask: int) -> evd_grid:
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    return evd_grid(int(lattice), int(precision), int(nx), int(ny), int(nz), int(wall_mask))


class SpeciesTable:
    """An evd_species with the arrays it points to kept alive."""

    def __init__(self, molar_mass, diffusivity, tau1: float, g=(0.0, 0.0, 0.0), flags: int = 0):
        self.M = np.ascontiguousarray(molar_mass, dtype=np.float64)
        ns = len(self.M)
        self.D = np.ascontiguousarray(np.asarray(diffusivity, dtype=np.float64).reshape(ns, ns))
        gg = (tuple(g) + (0.0, 0.0, 0.0))[:3]
        self.struct = evd_species(ns, self.M.ctypes.data_as(_dp), self.D.ctypes.data_as(_dp),
                                  float(tau1), (ctypes.c_double * 3)(*gg), int(flags))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


# --------------------------------------------------------------- the ABI
def evd_version() -> int:
    return lib().evd_version()


def evd_required_bytes(grid: evd_grid, species: SpeciesTable) -> int:
    return lib().evd_required_bytes(ctypes.byref(grid), ctypes.byref(species.struct))


def evd_create(grid: evd_grid, species: SpeciesTable, stream=None):
    out = _vp()
    _check(lib().evd_create(ctypes.byref(grid), ctypes.byref(species.struct), _stream(stream),
                            ctypes.byref(out)))
    return out


def evd_create_with_buffers(grid: evd_grid, species: SpeciesTable, stream, pop_a, pop_b, bytes_each: int):
    out = _vp()
    pa = pop_a if isinstance(pop_a, int) else pop_a.data_ptr()
    pb = pop_b if isinstance(pop_b, int) else pop_b.data_ptr()
    _check(lib().evd_create_with_buffers(ctypes.byref(grid), ctypes.byref(species.struct), _stream(stream),
                                         pa, pb, int(bytes_each), ctypes.byref(out)))
    return out


def evd_set_stream(ctx, stream):
    _check(lib().evd_set_stream(ctx, _stream(stream)), ctx)


def evd_set_fields(ctx, x, n=None):
    _check(lib().evd_set_fields(ctx, _ptr(x), _ptr(n)), ctx)


def evd_set_fields_device(ctx, x_dev, n_dev=None):
    _check(lib().evd_set_fields_device(ctx, _ptr(x_dev), _ptr(n_dev)), ctx)


def evd_set_populations(ctx, f):
    _check(lib().evd_set_populations(ctx, _ptr(f)), ctx)


def evd_step(ctx, nsteps: int):
    _check(lib().evd_step(ctx, int(nsteps)), ctx)


def evd_readout_device(ctx, x=None, rho=None, u=None, ui=None):
    _check(lib().evd_readout_device(ctx, _ptr(x), _ptr(rho), _ptr(u), _ptr(ui)), ctx)


def evd_get_mole_fractions(ctx, out):
    _check(lib().evd_get_mole_fractions(ctx, _ptr(out, writable=True)), ctx)


def evd_get_densities(ctx, out):
    _check(lib().evd_get_densities(ctx, _ptr(out, writable=True)), ctx)


def evd_get_velocities(ctx, u_out=None, ui_out=None):
    _check(lib().evd_get_velocities(ctx, _ptr(u_out, writable=True), _ptr(ui_out, writable=True)), ctx)


def evd_get_species_mass(ctx, out):
    _check(lib().evd_get_species_mass(ctx, _ptr(out, writable=True)), ctx)


def evd_species_mass_device(ctx, m_dev):
    _check(lib().evd_species_mass_device(ctx, _ptr(m_dev)), ctx)


def evd_get_populations(ctx, out):
    _check(lib().evd_get_populations(ctx, _ptr(out, writable=True)), ctx)


def evd_time(ctx) -> int:
    return lib().evd_time(ctx)


def evd_check(ctx):
    _check(lib().evd_check(ctx), ctx)


def evd_launch_count(ctx) -> int:
    return lib().evd_launch_count(ctx)


def evd_set_kernel(ctx, kernel: int):
    _check(lib().evd_set_kernel(ctx, int(kernel)), ctx)


def evd_get_kernel(ctx) -> int:
    return lib().evd_get_kernel(ctx)


def evd_set_force_field(ctx, k=None):
    """k: [D][sites] float64 (host), or None to remove the field."""
    _check(lib().evd_set_force_field(ctx, _ptr(k)), ctx)


def evd_loss_gradient(ctx, x0, target, nsteps: int, n0=None, checkpoint_every: int = 0):
    """(loss, dL/dD [ns][ns], dL/dg [3]) of the mole-fraction misfit after
    nsteps steps from x0 (evd_loss_gradient)."""
    ns = target.shape[0]
    loss = np.zeros(1)
    dD = np.zeros(ns * ns)
    dg = np.zeros(3)
    _check(lib().evd_loss_gradient(ctx, _ptr(x0), _ptr(n0), int(nsteps), _ptr(target), int(checkpoint_every),
                                   loss.ctypes.data, dD.ctypes.data, dg.ctypes.data), ctx)
    return float(loss[0]), dD.reshape(ns, ns), dg


def evd_set_adjoint_mode(ctx, mode: int):
    _check(lib().evd_set_adjoint_mode(ctx, int(mode)), ctx)


def evd_set_adjoint_forward(ctx, precision):
    """precision: "fp64" / "fp32" or EVD_FP64 / EVD_FP32."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib().evd_set_adjoint_forward(ctx, p), ctx)


def evd_set_tile_rows(ctx, rows: int):
    _check(lib().evd_set_tile_rows(ctx, int(rows)), ctx)


def evd_set_mass_correction(ctx, every: int):
    _check(lib().evd_set_mass_correction(ctx, int(every)), ctx)


def evd_set_wait_limit(ctx, polls: int):
    _check(lib().evd_set_wait_limit(ctx, int(polls)), ctx)


def evd_set_reference_mode(ctx, mode: int):
    _check(lib().evd_set_reference_mode(ctx, int(mode)), ctx)


def evd_get_reference_mode(ctx) -> int:
    return lib().evd_get_reference_mode(ctx)


def evd_get_target_mass(ctx, out):
    _check(lib().evd_get_target_mass(ctx, _ptr(out, writable=True)), ctx)


def evd_population_mass_noalloc(f_dev, n_species: int, q: int, nsites: int, m_dev, stream=None):
    """Species masses of a device population array; allocates nothing."""
    _check(lib().evd_population_mass_noalloc(_ptr(f_dev), int(n_species), int(q), int(nsites),
                                             _ptr(m_dev), _stream(stream)))


def evd_destroy(ctx):
    _check(lib().evd_destroy(ctx))


def evd_last_error(ctx=None) -> str:
    return lib().evd_last_error(ctx).decode()


# ------------------------------------------------ the batch (evd_batch.h)
def evd_batch_create(lattice: int, precision: int, members, stream=None):
    """members: a ctypes array of evd_member (keep the species arrays alive)."""
    out = _vp()
    _bcheck(lib().evd_batch_create(int(lattice), int(precision), members, len(members), _stream(stream),
                                   ctypes.byref(out)))
    return out


def evd_batch_sizes(b) -> tuple[int, int]:
    s, ss = ctypes.c_longlong(), ctypes.c_longlong()
    _bcheck(lib().evd_batch_sizes(b, ctypes.byref(s), ctypes.byref(ss)), b)
    return s.value, ss.value


def evd_batch_set_fields(b, x, n=None):
    _bcheck(lib().evd_batch_set_fields(b, _ptr(x), _ptr(n)), b)


def evd_batch_step(b, nsteps: int):
    _bcheck(lib().evd_batch_step(b, int(nsteps)), b)


def evd_batch_readout_device(b, x=None, rho=None, u=None, ui=None):
    _bcheck(lib().evd_batch_readout_device(b, _ptr(x), _ptr(rho), _ptr(u), _ptr(ui)), b)


def evd_batch_get_mole_fractions(b, out):
    _bcheck(lib().evd_batch_get_mole_fractions(b, _ptr(out, writable=True)), b)


def evd_batch_get_densities(b, out):
    _bcheck(lib().evd_batch_get_densities(b, _ptr(out, writable=True)), b)


def evd_batch_get_velocities(b, u_out=None, ui_out=None):
    _bcheck(lib().evd_batch_get_velocities(b, _ptr(u_out, writable=True), _ptr(ui_out, writable=True)), b)


def evd_batch_get_species_mass(b, out):
    _bcheck(lib().evd_batch_get_species_mass(b, _ptr(out, writable=True)), b)


def evd_batch_set_schedule(b, item_sites: int, ctas_per_sm: int):
    _bcheck(lib().evd_batch_set_schedule(b, int(item_sites), int(ctas_per_sm)), b)


def evd_batch_get_schedule(b) -> tuple[int, int]:
    i, c = ctypes.c_int(), ctypes.c_int()
    _bcheck(lib().evd_batch_get_schedule(b, ctypes.byref(i), ctypes.byref(c)), b)
    return i.value, c.value


def evd_batch_autotune(b, steps_per_trial: int = 8) -> tuple[int, int]:
    i, c = ctypes.c_int(), ctypes.c_int()
    _bcheck(lib().evd_batch_autotune(b, int(steps_per_trial), ctypes.byref(i), ctypes.byref(c)), b)
    return i.value, c.value


def evd_batch_set_graph(b, steps_per_graph: int):
    _bcheck(lib().evd_batch_set_graph(b, int(steps_per_graph)), b)


def evd_batch_set_mass_correction(b, every: int):
    _bcheck(lib().evd_batch_set_mass_correction(b, int(every)), b)


def evd_batch_time(b) -> int:
    return lib().evd_batch_time(b)


def evd_batch_launch_count(b) -> int:
    return lib().evd_batch_launch_count(b)


def evd_batch_check(b):
    _bcheck(lib().evd_batch_check(b), b)


def evd_batch_destroy(b):
    _bcheck(lib().evd_batch_destroy(b))


def evd_batch_last_error(b=None) -> str:
    return lib().evd_batch_last_error(b).decode()


# ------------------------------------------------------- convenience layer
class Simulation:
    """One EVD lattice on the current CUDA device (owns an evd_ctx).

    ``shape`` is (nx, ny[, nz]); arrays returned are numpy float64 with the
    site axes in (nz, ny, nx) order, matching the seeded workloads."""

    def __init__(self, lattice, shape, wall_mask, molar_mass, diffusivity, tau1, g=(0.0, 0.0, 0.0),
                 precision="fp64", stream=None, flags=0):
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.grid = make_grid(lattice, self.precision, shape, wall_mask)
        self.species = SpeciesTable(molar_mass, diffusivity, tau1, g, flags)
        self.lattice = int(lattice)
        self.ns = len(self.species.M)
        self.Q = 9 if self.lattice == EVD_D2Q9 else 19
        self.D = 2 if self.lattice == EVD_D2Q9 else 3
        self.sites = (self.grid.nz, self.grid.ny, self.grid.nx)
        self.nsites = self.grid.nx * self.grid.ny * self.grid.nz
        self.ctx = evd_create(self.grid, self.species, stream)

    @classmethod
    def from_workload(cls, wl, precision="fp64", stream=None):
        sim = cls(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, precision, stream,
                  getattr(wl, "flags", 0))
        if getattr(wl, "force", None) is not None:
            sim.set_force_field(wl.force)
        sim.set_fields(wl.x, wl.n)
        return sim

    def close(self):
        if getattr(self, "ctx", None) is not None:
            evd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, x, n=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = None if n is None else np.ascontiguousarray(n, dtype=np.float64)
        evd_set_fields(self.ctx, x, n)

    def set_force_field(self, k):
        """Per-node specific force (3 or D, nz, ny, nx) added to g; None removes it."""
        if k is None:
            evd_set_force_field(self.ctx, None)
            return
        k = np.ascontiguousarray(np.asarray(k, dtype=np.float64)[:self.D]).reshape(self.D, -1)
        evd_set_force_field(self.ctx, np.ascontiguousarray(k))

    def set_populations(self, f):
        evd_set_populations(self.ctx, np.ascontiguousarray(f, dtype=np.float64))

    def step(self, nsteps=1):
        evd_step(self.ctx, nsteps)

    @property
    def t(self):
        return evd_time(self.ctx)

    def mole_fractions(self):
        out = np.empty((self.ns,) + self.sites)
        evd_get_mole_fractions(self.ctx, out)
        return out

    def densities(self):
        out = np.empty((self.ns,) + self.sites)
        evd_get_densities(self.ctx, out)
        return out

    def velocities(self):
        u = np.empty((self.D,) + self.sites)
        ui = np.empty((self.ns, self.D) + self.sites)
        evd_get_velocities(self.ctx, u, ui)
        return u, ui

    def species_mass(self):
        out = np.empty(self.ns)
        evd_get_species_mass(self.ctx, out)
        return out

    def populations(self):
        out = np.empty((self.ns, self.Q) + self.sites)
        evd_get_populations(self.ctx, out)
        return out

    def check(self):
        evd_check(self.ctx)


class Batch:
    """Many independent lattices of one lattice type and precision advanced
    together (owns an evd_batch).  Members are given as seeded workloads (or
    anything with lattice, shape, wall_mask, M, D, tau1, g); per-member
    arrays are returned as lists in member order, site axes (nz, ny, nx)."""

    def __init__(self, members, precision="fp32", stream=None):
        members = list(members)
        if not members:
            raise ValueError("a batch needs at least one member")
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.lattice = int(members[0].lattice)
        self.Q = 9 if self.lattice == EVD_D2Q9 else 19
        self.D = 2 if self.lattice == EVD_D2Q9 else 3
        self._tables = [SpeciesTable(m.M, m.D, m.tau1, m.g) for m in members]
        arr = (evd_member * len(members))()
        self.shapes, self.ns = [], []
        for k, m in enumerate(members):
            nx, ny, nz = (tuple(m.shape) + (1, 1))[:3]
            arr[k] = evd_member(int(nx), int(ny), int(nz), int(m.wall_mask), self._tables[k].struct)
            self.shapes.append((nz, ny, nx))
            self.ns.append(len(self._tables[k].M))
        self._members = arr
        self.b = evd_batch_create(self.lattice, self.precision, arr, stream)
        self.nsites, self.nspecies_sites = evd_batch_sizes(self.b)

    @classmethod
    def from_workloads(cls, workloads, precision="fp32", stream=None):
        bt = cls(workloads, precision, stream)
        bt.set_fields([w.x for w in workloads], [w.n for w in workloads])
        return bt

    def close(self):
        if getattr(self, "b", None) is not None:
            evd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, xs, ns=None):
        x = np.concatenate([np.ascontiguousarray(a, dtype=np.float64).ravel() for a in xs])
        n = None
        if ns is not None and any(a is not None for a in ns):
            n = np.concatenate([np.ones(int(np.prod(s))) if a is None else
                                np.ascontiguousarray(a, dtype=np.float64).ravel()
                                for a, s in zip(ns, self.shapes)])
        evd_batch_set_fields(self.b, x, n)

    def step(self, nsteps=1):
        evd_batch_step(self.b, nsteps)

    @property
    def t(self):
        return evd_batch_time(self.b)

    def _split(self, flat, per_site):
        out, k = [], 0
        for s, c in zip(self.shapes, per_site):
            n = int(np.prod(s)) * c
            out.append(flat[k:k + n].reshape((c,) + s))
            k += n
        return out

    def mole_fractions(self):
        out = np.empty(self.nspecies_sites)
        evd_batch_get_mole_fractions(self.b, out)
        return self._split(out, self.ns)

    def densities(self):
        out = np.empty(self.nspecies_sites)
        evd_batch_get_densities(self.b, out)
        return self._split(out, self.ns)

    def velocities(self):
        u = np.empty(self.D * self.nsites)
        ui = np.empty(self.D * self.nspecies_sites)
        evd_batch_get_velocities(self.b, u, ui)
        us = self._split(u, [self.D] * len(self.ns))
        uis = [a.reshape((n, self.D) + a.shape[1:]) for a, n in
               zip(self._split(ui, [self.D * n for n in self.ns]), self.ns)]
        return us, uis

    def species_mass(self):
        out = np.empty(len(self.ns) * EVD_MAX_SPECIES)
        evd_batch_get_species_mass(self.b, out)
        return [out[k * EVD_MAX_SPECIES:k * EVD_MAX_SPECIES + n] for k, n in enumerate(self.ns)]

    def check(self):
        evd_batch_check(self.b)


def evd_fma_rate(kind: int, iters: int = 1 << 16, stream=None):
    """(flops, milliseconds) of the FMA-chain throughput kernel: kind 0
    double, 1 float, 2 float pairs."""
    f, m = ctypes.c_double(), ctypes.c_double()
    _check(lib().evd_fma_rate(int(kind), int(iters), ctypes.byref(f), ctypes.byref(m), _stream(stream)))
    return f.value, m.value
