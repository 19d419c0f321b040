"""Python access to the FP64 CPU oracle in ``evd_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference for the
forced EVD lattice Boltzmann step (Lourenco, Constantino & Tavares 2025).  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares nothing with the CUDA library.

Array layouts (all float64, C order):
  populations  [ns][Q][nz][ny][nx]   (post-stream state f_t)
  x, rho       [ns][nz][ny][nx]
  u            [3][nz][ny][nx]
  ui, ueq      [ns][3][nz][ny][nx]
"""
from __future__ import annotations

import atexit
import contextlib
import ctypes
import os
import shutil
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None
_variants = 0

MAXS = 6
MAXQ = 19


_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_FLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc"] + _FLAGS + ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def build_omp(force: bool = False) -> str | None:
    """The same source compiled with OpenMP (the streaming tasks and the node
    collisions on all host cores; bitwise the serial results).  Returns None
    where the compiler has no OpenMP."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO_OMP)
            and os.path.getmtime(_SO_OMP) >= os.path.getmtime(_SRC)):
        return _SO_OMP
    tmp = _SO_OMP + f".tmp{os.getpid()}"
    cmd = ["gcc", "-fopenmp"] + _FLAGS + ["-o", tmp, _SRC, "-lm"]
    if subprocess.run(cmd, capture_output=True).returncode != 0:
        return None
    os.replace(tmp, _SO_OMP)
    return _SO_OMP


class Config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_mask", ctypes.c_uint),
        ("ns", ctypes.c_int),
        ("M", ctypes.c_double * MAXS),
        ("D", ctypes.c_double * (MAXS * MAXS)),
        ("tau1", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("tau_mode", ctypes.c_int),
        ("flags", ctypes.c_uint),
    ]


# corrective forcing terms of Eq. (improved_forcing_scheme), Config.flags bits
S_DIFF, S_P, S_RHO = 1, 2, 4


class Diag(ctypes.Structure):
    _fields_ = [
        ("rho", ctypes.c_double * MAXS),
        ("ueq", (ctypes.c_double * 3) * MAXS),
        ("u", ctypes.c_double * 3),
        ("rho_mix", ctypes.c_double), ("n", ctypes.c_double), ("p", ctypes.c_double),
        ("tau", ctypes.c_double * MAXS),
        ("tau_x", ctypes.c_double * (MAXS * MAXS)),
        ("feq", (ctypes.c_double * MAXQ) * MAXS),
        ("f0", (ctypes.c_double * MAXQ) * MAXS),
        ("om_self", (ctypes.c_double * MAXQ) * MAXS),
        ("om_pair", ((ctypes.c_double * MAXQ) * MAXS) * MAXS),
        ("S", (ctypes.c_double * MAXQ) * MAXS),
        ("theta", (ctypes.c_double * 3) * MAXS),
    ]


def _bind(path: str):
    """Load an oracle library and declare its entry points."""
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    L.or_create.restype = ctypes.c_void_p
    L.or_create.argtypes = [P(Config)]
    L.or_destroy.argtypes = [ctypes.c_void_p]
    L.or_init.restype = ctypes.c_int
    L.or_init.argtypes = [ctypes.c_void_p, dp, dp]
    L.or_set_force_field.restype = ctypes.c_int
    L.or_set_force_field.argtypes = [ctypes.c_void_p, dp]
    L.or_step.restype = ctypes.c_long
    L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    L.or_stream_only.argtypes = [ctypes.c_void_p]
    L.or_collide_only.restype = ctypes.c_int
    L.or_collide_only.argtypes = [ctypes.c_void_p]
    L.or_set_f.argtypes = [ctypes.c_void_p, dp]
    L.or_get_f.argtypes = [ctypes.c_void_p, dp]
    L.or_time.restype = ctypes.c_long
    L.or_time.argtypes = [ctypes.c_void_p]
    L.or_threads.restype = ctypes.c_int
    L.or_threads.argtypes = []
    L.or_observables.restype = ctypes.c_int
    L.or_observables.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
    L.or_mass.argtypes = [ctypes.c_void_p, dp]
    L.or_collide_node.restype = ctypes.c_int
    L.or_collide_node.argtypes = [ctypes.c_void_p, dp, dp, P(Diag)]
    L.or_diag_size.restype = ctypes.c_int
    L.or_tau_cross.restype = ctypes.c_int
    L.or_tau_cross.argtypes = [P(Config), dp, dp]
    L.or_tau_cross_dense.restype = ctypes.c_int
    L.or_tau_cross_dense.argtypes = [P(Config), dp, dp]
    L.or_lattice_info.restype = ctypes.c_int
    L.or_lattice_info.argtypes = [ctypes.c_int, P(ctypes.c_int), dp, P(ctypes.c_int)]
    L.or_species_info.argtypes = [ctypes.c_void_p, dp, dp, dp]
    assert L.or_diag_size() == ctypes.sizeof(Diag), "oracle diag layout mismatch"
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


_variant_dir = None


def _variants_dir() -> str:
    """A private temporary directory for compiled variants, removed when the
    process exits (a loaded library stays mapped after its file is gone)."""
    global _variant_dir
    if _variant_dir is None:
        _variant_dir = tempfile.mkdtemp(prefix="evd_oracle_variants_")
        atexit.register(shutil.rmtree, _variant_dir, True)
    return _variant_dir


def compile_variant(source: str, tag: str) -> str:
    """Compile C source text (a modified copy of the oracle, for the tests that
    check that the pins catch planted mistakes) with the oracle's flags, in a
    temporary directory removed at exit; returns the library path."""
    global _variants
    _variants += 1
    # a fresh file name each time: the dynamic loader keeps a library it has
    # already loaded under the same path
    base = os.path.join(_variants_dir(), f"variant_{tag}_{_variants}")
    src, so = base + ".c", base + ".so"
    with open(src, "w") as fh:
        fh.write(source)
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", so, src, "-lm"]
    subprocess.run(cmd, check=True)
    return so


@contextlib.contextmanager
def swapped_library(path: str):
    """Every oracle call inside the block goes to the library at path."""
    global _lib
    L = _bind(path)
    with _lock:
        old = _lib
        _lib = L
    try:
        yield
    finally:
        with _lock:
            _lib = old


def threads() -> int:
    """Threads a step of the library in use runs on (1 for the serial build)."""
    return int(lib().or_threads())


def source() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice_info(lattice: int):
    """(e [Q,3] int, w [Q], opp [Q]) of the oracle's lattice table."""
    e = (ctypes.c_int * (MAXQ * 3))()
    w = np.zeros(MAXQ)
    opp = (ctypes.c_int * MAXQ)()
    Q = lib().or_lattice_info(lattice, e, _dp(w), opp)
    return (np.array(e[:Q * 3], dtype=np.int64).reshape(Q, 3), w[:Q].copy(),
            np.array(opp[:Q], dtype=np.int64))


def make_config(lattice, shape, wall_mask, M, D, tau1, g, tau_mode=0, flags=0) -> Config:
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    ns = len(M)
    c = Config()
    c.lattice = int(lattice)
    c.nx, c.ny, c.nz = int(nx), int(ny), int(nz)
    c.wall_mask = int(wall_mask)
    c.ns = ns
    for i in range(ns):
        c.M[i] = float(M[i])
    Dm = np.asarray(D, dtype=np.float64).reshape(ns, ns)
    for i in range(ns):
        for j in range(ns):
            c.D[i * ns + j] = float(Dm[i, j])
    c.tau1 = float(tau1)
    gg = list(g) + [0.0] * (3 - len(g))
    for k in range(3):
        c.g[k] = float(gg[k])
    c.tau_mode = int(tau_mode)
    c.flags = int(flags)
    return c


def tau_cross(cfg: Config, rho, dense: bool = False) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.zeros(cfg.ns * cfg.ns)
    fn = lib().or_tau_cross_dense if dense else lib().or_tau_cross
    ok = fn(ctypes.byref(cfg), _dp(rho), _dp(out))
    if not ok:
        raise ValueError("oracle tau_ij solve failed")
    return out.reshape(cfg.ns, cfg.ns)


class Oracle:
    """One lattice in the oracle.  ``shape`` is (nx, ny[, nz])."""

    def __init__(self, lattice, shape, wall_mask, M, D, tau1, g, tau_mode=0, flags=0):
        self.cfg = make_config(lattice, shape, wall_mask, M, D, tau1, g, tau_mode, flags)
        self.lattice = int(lattice)
        self.ns = len(M)
        self.Q = 9 if lattice == 0 else 19
        self.shape_xyz = (self.cfg.nx, self.cfg.ny, self.cfg.nz)
        self.nsites = self.cfg.nx * self.cfg.ny * self.cfg.nz
        self._h = lib().or_create(ctypes.byref(self.cfg))
        if not self._h:
            raise ValueError("oracle rejected the configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    @property
    def grid(self):
        nx, ny, nz = self.shape_xyz
        return (nz, ny, nx)

    def species_info(self):
        c = np.zeros(self.ns); cs2 = np.zeros(self.ns); tau = np.zeros(self.ns)
        lib().or_species_info(self._h, _dp(c), _dp(cs2), _dp(tau))
        return c, cs2, tau

    def init(self, x, n=None):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.ns, self.nsites)
        nn = None if n is None else np.ascontiguousarray(n, dtype=np.float64).reshape(self.nsites)
        if not lib().or_init(self._h, _dp(x), _dp(nn)):
            raise ValueError("oracle init: non-positive density")

    def set_force_field(self, k):
        """Per-node specific force k(x) added to g, shape (3, nz, ny, nx) or
        (3, nsites); None removes it.  Set it before init (Sec. 4.2, Case II)."""
        if k is None:
            lib().or_set_force_field(self._h, None)
            return
        k = np.ascontiguousarray(k, dtype=np.float64).reshape(3, self.nsites)
        if not lib().or_set_force_field(self._h, _dp(k)):
            raise MemoryError("oracle force field")

    def step(self, nsteps=1):
        done = lib().or_step(self._h, int(nsteps))
        if done != nsteps:
            raise FloatingPointError(f"oracle step failed after {done} steps")

    def stream_only(self):
        lib().or_stream_only(self._h)

    def collide_only(self):
        if not lib().or_collide_only(self._h):
            raise FloatingPointError("oracle collision failed")

    @property
    def t(self):
        return lib().or_time(self._h)

    def get_f(self):
        f = np.zeros((self.ns, self.Q) + self.grid)
        lib().or_get_f(self._h, _dp(f))
        return f

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.ns * self.Q * self.nsites
        lib().or_set_f(self._h, _dp(f))

    def observables(self):
        x = np.zeros((self.ns,) + self.grid)
        rho = np.zeros_like(x)
        u = np.zeros((3,) + self.grid)
        ui = np.zeros((self.ns, 3) + self.grid)
        ueq = np.zeros_like(ui)
        if not lib().or_observables(self._h, _dp(x), _dp(rho), _dp(u), _dp(ui), _dp(ueq)):
            raise FloatingPointError("oracle observables failed")
        return {"x": x, "rho": rho, "u": u, "ui": ui, "ueq": ueq}

    def mass(self):
        m = np.zeros(self.ns)
        lib().or_mass(self._h, _dp(m))
        return m

    def collide_node(self, f_node):
        """f_node [ns][Q] -> (fstar [ns][Q], Diag)."""
        f_node = np.ascontiguousarray(f_node, dtype=np.float64).reshape(self.ns * self.Q)
        out = np.zeros_like(f_node)
        dg = Diag()
        if not lib().or_collide_node(self._h, _dp(f_node), _dp(out), ctypes.byref(dg)):
            raise FloatingPointError("oracle node collision failed")
        return out.reshape(self.ns, self.Q), dg


def diag_arrays(dg: Diag, ns: int, Q: int) -> dict:
    """Plain numpy views of a Diag for the first ns species and Q directions."""
    a = lambda v: np.ctypeslib.as_array(v)
    return {
        "rho": a(dg.rho)[:ns].copy(),
        "ueq": a(dg.ueq)[:ns].copy(),
        "u": a(dg.u).copy(),
        "rho_mix": dg.rho_mix, "n": dg.n, "p": dg.p,
        "tau": a(dg.tau)[:ns].copy(),
        "tau_x": a(dg.tau_x)[:ns * ns].reshape(ns, ns).copy(),
        "feq": a(dg.feq)[:ns, :Q].copy(),
        "f0": a(dg.f0)[:ns, :Q].copy(),
        "om_self": a(dg.om_self)[:ns, :Q].copy(),
        "om_pair": a(dg.om_pair)[:ns, :ns, :Q].copy(),
        "S": a(dg.S)[:ns, :Q].copy(),
        "theta": a(dg.theta)[:ns].copy(),
    }
