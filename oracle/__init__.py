"""FP64 CPU oracle of the short-range TreePM tree force -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library (the product path)
never imports, links or calls it; the two share no code.  See ``oracle.c`` for
what each routine computes and which passage of the paper it follows.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  quantize / morton         brute force, closed form on lattices
  tree build (topology)     brute-force node-set definition over all levels
  moments                   exact rational sums rounded once and the rounded
                            exact centre of mass (Python fractions), bitwise
  groups                    partition and size invariants
  lists                     partition invariant (every neighbour covered once),
                            theta = 0 reduces to all particles within the cutoff
  opening decision          hand-placed one-node trees at every threshold of the
                            Barnes-Hut, relative and boundary tests, exact
                            rationals (tests/test_oracle_opening.py)
  cutoff decision           single precision on the exact integer separation,
                            recomputed with exact integers and 24-bit rounding
  force                     two-body closed form from the spline mass profile
                            and the erfc potential (numerical quadrature and
                            differentiation), theta = 0 equals direct summation,
                            uniform sphere interior, lattice zero force,
                            momentum conservation as theta -> 0
  size of the tree error    no value to pin it to: the paper prints no accuracy
  at theta > 0              numbers for its tree; every step that produces it is
                            pinned above, and theta -> 0 reaches the direct sum
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPEN_BH = 0
OPEN_REL = 1

(N, NODES, CHILDREN, GROUPS, LIST_LEN) = range(5)
(F_X, F_Y, F_Z, F_KEY, F_PERM, F_LEVEL, F_BEG, F_END, F_PARENT, F_CBEG, F_CCNT, F_CHILD,
 F_MASS, F_COM, F_MSUM, F_NEXTNODE, F_SIBLING, F_PNEXT, F_GBEG, F_GEND, F_GLO, F_GHI,
 F_EXT_S, F_EXT_L) = range(24)


class Params(C.Structure):
    _fields_ = [("box", C.c_double), ("G", C.c_double), ("eps", C.c_double),
                ("r_s", C.c_double), ("rcut_over_rs", C.c_double), ("theta", C.c_double),
                ("alpha", C.c_double), ("theta_first_pass", C.c_double),
                ("opening", C.c_int32), ("leaf_max", C.c_int32), ("group_max", C.c_int32),
                ("pad", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, FP64, OpenMP,
    no floating-point contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                    os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.c_void_p
            i64 = C.c_int64
            L.ora_quantize1.argtypes = [C.c_double, C.c_double, C.POINTER(C.c_uint32)]
            L.ora_morton.argtypes = [C.c_uint32] * 3
            L.ora_morton.restype = C.c_uint64
            L.ora_soft_g.argtypes = [C.c_double, C.c_double]
            L.ora_soft_g.restype = C.c_double
            L.ora_split_s.argtypes = [C.c_double, C.c_double]
            L.ora_split_s.restype = C.c_double
            L.ora_soft_psi.argtypes = [C.c_double, C.c_double]
            L.ora_soft_psi.restype = C.c_double
            L.ora_split_p.argtypes = [C.c_double, C.c_double]
            L.ora_split_p.restype = C.c_double
            L.ora_tree_force_pot.argtypes = [P, P, C.c_int, C.c_double, C.c_double, P, i64, P, P,
                                             P, P, C.c_int, C.c_int]
            L.ora_direct_pot.argtypes = [P, P, i64, C.POINTER(Params), P, i64, P, P, C.c_int]
            L.ora_tree_build.argtypes = [P, P, i64, C.POINTER(Params), C.POINTER(P)]
            L.ora_tree_free.argtypes = [P]
            L.ora_tree_refit.argtypes = [P, P]
            L.ora_tree_free.restype = None
            L.ora_tree_count.argtypes = [P, C.c_int]
            L.ora_tree_count.restype = i64
            L.ora_tree_get.argtypes = [P, C.c_int, P]
            L.ora_tree_force.argtypes = [P, P, C.c_int, C.c_double, C.c_double, P, i64, P, P,
                                         P, C.c_int, C.c_int]
            L.ora_tree_get_lists.argtypes = [P, i64, P, P]
            L.ora_direct.argtypes = [P, P, i64, C.POINTER(Params), P, i64, P, C.c_int]
            L.ora_cell_exact.argtypes = [P, P, i64, C.POINTER(Params), P, i64, P, C.c_int]
            L.ora_num_threads.restype = C.c_int
            _lib = L
    return _lib


def make_params(p: dict) -> Params:
    return Params(float(p.get("box", 1.0)), float(p.get("G", 1.0)), float(p.get("eps", 0.0)),
                  float(p.get("r_s", 0.0)), float(p.get("rcut_over_rs", 4.5)),
                  float(p.get("theta", 0.5)), float(p.get("alpha", 0.005)),
                  float(p.get("theta_first_pass", 0.5)), int(p.get("opening", OPEN_BH)),
                  int(p.get("leaf_max", 1)), int(p.get("group_max", 32)), 0)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def quantize1(v: float, box: float = 1.0) -> int:
    out = C.c_uint32()
    rc = lib().ora_quantize1(float(v), float(box), C.byref(out))
    if rc:
        raise ValueError("non-finite coordinate")
    return int(out.value)


def morton(x: int, y: int, z: int) -> int:
    return int(lib().ora_morton(x, y, z))


def soft_g(r: float, h: float) -> float:
    return float(lib().ora_soft_g(float(r), float(h)))


def split_s(r: float, rs: float) -> float:
    return float(lib().ora_split_s(float(r), float(rs)))


def soft_psi(r: float, h: float) -> float:
    return float(lib().ora_soft_psi(float(r), float(h)))


def split_p(r: float, rs: float) -> float:
    return float(lib().ora_split_p(float(r), float(rs)))


def num_threads() -> int:
    return int(lib().ora_num_threads())


class Tree:
    """An oracle tree: a1-a6 of the hot path on the CPU in FP64."""

    def __init__(self, pos, mass, params: dict):
        self.params = dict(params)
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.n = pos.shape[0]
        h = C.c_void_p()
        prm = make_params(params)
        rc = lib().ora_tree_build(_ptr(pos), _ptr(mass), self.n, C.byref(prm), C.byref(h))
        if rc:
            raise ValueError(f"oracle tree build failed ({rc})")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.ora_tree_free(h)
            self._h = None

    def count(self, what: int) -> int:
        return int(lib().ora_tree_count(self._h, what))

    @property
    def nnodes(self) -> int:
        return self.count(NODES)

    @property
    def ngroups(self) -> int:
        return self.count(GROUPS)

    def get(self, field: int) -> np.ndarray:
        n, m, g, c = self.n, self.nnodes, self.ngroups, self.count(CHILDREN)
        shape, dt = {
            F_X: (n, np.uint32), F_Y: (n, np.uint32), F_Z: (n, np.uint32),
            F_KEY: (n, np.uint64), F_PERM: (n, np.int64), F_LEVEL: (m, np.int32),
            F_BEG: (m, np.int64), F_END: (m, np.int64), F_PARENT: (m, np.int64),
            F_CBEG: (m, np.int64), F_CCNT: (m, np.int64), F_CHILD: (c, np.int64),
            F_MASS: (m, np.float64), F_COM: ((m, 3), np.uint32), F_MSUM: ((m, 3), np.float64),
            F_NEXTNODE: (m, np.int64), F_SIBLING: (m, np.int64), F_PNEXT: (n, np.int64),
            F_GBEG: (g, np.int64), F_GEND: (g, np.int64), F_GLO: ((g, 3), np.uint32),
            F_GHI: ((g, 3), np.uint32), F_EXT_S: ((m, 3), np.uint32),
            F_EXT_L: ((m, 3), np.uint32)}[field]
        out = np.zeros(shape, dtype=dt)
        rc = lib().ora_tree_get(self._h, field, _ptr(out))
        if rc:
            raise ValueError("bad field")
        return out

    def refit(self, pos):
        """Drifted positions of the same particles (input order): same
        topology and groups, new moments, node extents and group boxes."""
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        if pos.shape[0] != self.n:
            raise ValueError("refit needs the same number of particles")
        rc = lib().ora_tree_refit(self._h, _ptr(pos))
        if rc:
            raise ValueError(f"oracle refit failed ({rc})")

    def force(self, opening=None, theta=None, alpha=None, a_old=None, groups=None,
              keep_lists=False, nthreads=0, want_pot=False):
        """a7-a9.  Returns (acc[N,3] f64, n_pp[N], n_pn[N]) in input order; with
        ``groups`` only the targets of those groups are filled (others NaN).
        ``a_old`` (input order, float32 [N,3]) feeds the relative criterion;
        without it a Barnes-Hut first pass supplies it."""
        p = self.params
        opening = p.get("opening", OPEN_BH) if opening is None else opening
        theta = p.get("theta", 0.5) if theta is None else theta
        alpha = p.get("alpha", 0.005) if alpha is None else alpha
        acc = np.full((self.n, 3), np.nan)
        npp = np.zeros(self.n, dtype=np.uint32)
        npn = np.zeros(self.n, dtype=np.uint32)
        ao = None if a_old is None else np.ascontiguousarray(a_old, dtype=np.float32).reshape(-1, 3)
        sel = None if groups is None else np.ascontiguousarray(groups, dtype=np.int64)
        nsel = 0 if sel is None else sel.shape[0]
        pot = np.full(self.n, np.nan) if want_pot else None
        rc = lib().ora_tree_force_pot(self._h, _ptr(ao), int(opening), float(theta), float(alpha),
                                      _ptr(sel), nsel, _ptr(acc), _ptr(npp), _ptr(npn), _ptr(pot),
                                      int(bool(keep_lists)), int(nthreads))
        if rc:
            raise ValueError(f"oracle force failed ({rc})")
        self._nsel = self.ngroups if sel is None else nsel
        return (acc, npp, npn, pot) if want_pot else (acc, npp, npn)

    def force_pot(self, **kw):
        """force() plus the short-range potential per target (input order):
        returns (acc, n_pp, n_pn, pot)."""
        return self.force(want_pot=True, **kw)

    def lists(self):
        """Per selected group of the last force call: sorted unified refs
        (particle sorted index < N, node preorder id + N)."""
        L = self.count(LIST_LEN)
        off = np.zeros(self._nsel + 1, dtype=np.int64)
        lst = np.zeros(max(L, 1), dtype=np.int64)
        rc = lib().ora_tree_get_lists(self._h, self._nsel, _ptr(off), _ptr(lst))
        if rc:
            raise ValueError("no lists kept")
        return off, lst[:L]


def direct(pos, mass, params: dict, targets=None, nthreads=0) -> np.ndarray:
    """O(N^2) direct summation with the same split, softening, cutoff and
    minimum image (quantized positions)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = pos.shape[0] if t is None else t.shape[0]
    acc = np.zeros((nt, 3))
    prm = make_params(params)
    rc = lib().ora_direct(_ptr(pos), _ptr(mass), pos.shape[0], C.byref(prm), _ptr(t),
                          0 if t is None else nt, _ptr(acc), int(nthreads))
    if rc:
        raise ValueError(f"direct failed ({rc})")
    return acc


def direct_pot(pos, mass, params: dict, targets=None, nthreads=0):
    """direct() plus the short-range potential: returns (acc, pot)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = pos.shape[0] if t is None else t.shape[0]
    acc = np.zeros((nt, 3))
    pot = np.zeros(nt)
    prm = make_params(params)
    rc = lib().ora_direct_pot(_ptr(pos), _ptr(mass), pos.shape[0], C.byref(prm), _ptr(t),
                              0 if t is None else nt, _ptr(acc), _ptr(pot), int(nthreads))
    if rc:
        raise ValueError(f"direct failed ({rc})")
    return acc, pot


def cell_exact(pos, mass, params: dict, targets=None, nthreads=0) -> np.ndarray:
    """Exact short-range sum through a cell list of side >= r_cut."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = pos.shape[0] if t is None else t.shape[0]
    acc = np.zeros((nt, 3))
    prm = make_params(params)
    rc = lib().ora_cell_exact(_ptr(pos), _ptr(mass), pos.shape[0], C.byref(prm), _ptr(t),
                              0 if t is None else nt, _ptr(acc), int(nthreads))
    if rc:
        raise ValueError(f"cell_exact failed ({rc})")
    return acc
