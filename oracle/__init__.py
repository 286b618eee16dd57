"""Plain FP64 CPU oracle of the Barnes-Hut octree Monte Carlo method.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1305_1825_gb300``; the C source
``bhmc_oracle.c`` is compiled with ``gcc -O2 -ffp-contract=off -fno-fast-math``
into ``liboracle.so`` next to it and loaded with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bhmc_oracle.c")
_HDR = os.path.join(_HERE, "bhmc_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, EDOMAIN, EOVERLAP, ENOMEM, ECAPACITY = 0, 1, 2, 3, 4, 9
ACCEPT, REJECT_ENERGY, REJECT_DOMAIN, REJECT_OVERLAP, REJECT_CAPACITY = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile liboracle.so (no FMA contraction, no fast-math)."""
    stale = not os.path.exists(_LIB) or any(
        os.path.getmtime(f) > os.path.getmtime(_LIB) for f in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC",
            "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("lB", C.c_double), ("beta", C.c_double), ("theta", C.c_double),
        ("p", C.c_int32), ("N0", C.c_int32), ("C", C.c_int32), ("Dmax", C.c_int32),
        ("root_lo", C.c_double * 3), ("root_side", C.c_double),
        ("shell", C.c_int32), ("shell_rmin", C.c_double), ("shell_rmax", C.c_double),
        ("images", C.c_int32), ("image_R", C.c_double), ("image_alpha", C.c_double),
        ("hard_core", C.c_double),
        ("fixed_depth", C.c_int32),
        ("fixed_direct", C.c_int32),
    ]


class Eval(C.Structure):
    _fields_ = [("phi", C.c_double), ("abs_sum", C.c_double), ("bound", C.c_double),
                ("visited", C.c_int64), ("accepted", C.c_int64), ("pairs", C.c_int64),
                ("mac_near", C.c_int64)]


class DE(C.Structure):
    _fields_ = [("dE", C.c_double), ("abs_sum", C.c_double), ("bound", C.c_double),
                ("visited", C.c_int64), ("accepted", C.c_int64), ("pairs", C.c_int64),
                ("status", C.c_int32)]


class Record(C.Structure):
    _fields_ = [("i", C.c_int64), ("r_new", C.c_double * 3), ("dE", C.c_double),
                ("abs_sum", C.c_double), ("log_alpha", C.c_double),
                ("outcome", C.c_int32), ("flagged", C.c_int32)]


RECORD_DTYPE = np.dtype([("i", "<i8"), ("r_new", "<f8", (3,)), ("dE", "<f8"),
                         ("abs_sum", "<f8"), ("log_alpha", "<f8"), ("outcome", "<i4"),
                         ("flagged", "<i4")])
assert RECORD_DTYPE.itemsize == C.sizeof(Record)

_lib = None
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                       C.POINTER(C.c_uint32)]
        L.or_nterms.argtypes = [C.c_int]
        L.or_term_index.argtypes = [C.c_int, C.c_int, C.c_int]
        L.or_taylor.argtypes = [C.c_int, _dp, _dp]
        L.or_direct_energy_raw.argtypes = [C.c_int64, _dp, _dp, C.c_double]
        L.or_direct_energy_raw.restype = C.c_double
        L.or_create.argtypes = [C.POINTER(Params), C.c_int64, C.c_int64, _dp, _dp,
                                C.POINTER(C.c_int)]
        L.or_create.restype = C.c_void_p
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_set_bound.argtypes = [C.c_void_p, C.c_int]
        L.or_n_charges.argtypes = [C.c_void_p]
        L.or_n_charges.restype = C.c_int64
        L.or_get_charges.argtypes = [C.c_void_p, _dp, _dp]
        L.or_image_of.argtypes = [C.c_void_p, _dp, C.c_double, _dp, _dp]
        L.or_phi.argtypes = [C.c_void_p, _dp, C.c_int, _i64p, C.POINTER(Eval)]
        L.or_phi_direct.argtypes = [C.c_void_p, _dp, C.c_int, _i64p]
        L.or_phi_direct.restype = C.c_double
        L.or_delta_energy.argtypes = [C.c_void_p, C.c_int64, _dp, C.POINTER(DE)]
        L.or_delta_energy_direct.argtypes = [C.c_void_p, C.c_int64, _dp, _dp]
        L.or_commit_move.argtypes = [C.c_void_p, C.c_int64, _dp]
        L.or_capacity_violation.argtypes = [C.c_void_p, C.c_int64, _dp]
        L.or_mc_run.argtypes = [C.c_void_p, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int64,
                                C.c_double, C.c_void_p, _i64p]
        L.or_energy_direct.argtypes = [C.c_void_p]
        L.or_energy_direct.restype = C.c_double
        L.or_energy_tree.argtypes = [C.c_void_p]
        L.or_energy_tree.restype = C.c_double
        L.or_potentials.argtypes = [C.c_void_p, _dp, _dp]
        L.or_forces.argtypes = [C.c_void_p, _dp, _dp]
        L.or_forces_abs.argtypes = [C.c_void_p, _dp, _dp]
        L.or_radial_counts.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, _i64p, _dp]
        L.or_radial_profiles.argtypes = [C.c_int, C.c_double, C.c_double, _i64p, _dp, C.c_int64, C.c_double,
                                         _dp, _dp, _dp, _dp]
        L.or_ion_energy_grad.argtypes = [C.c_void_p, C.c_int64, _dp, _dp, _dp]
        L.or_phi_grad.argtypes = [C.c_void_p, _dp, C.c_int, _i64p, _dp, _dp]
        L.or_mala_run.argtypes = [C.c_void_p, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int64,
                                  C.c_double, C.c_void_p, _i64p]
        L.or_export_tree.argtypes = [C.c_void_p, _i64p, C.c_int64, _i64p, C.c_int64]
        L.or_export_tree.restype = C.c_int64
        L.or_check.argtypes = [C.c_void_p]
        L.or_node_moments.argtypes = [C.c_void_p, C.c_int, C.c_uint64, _dp]
        L.or_point_key.argtypes = [C.c_void_p, _dp]
        L.or_point_key.restype = C.c_uint64
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def nterms(p: int) -> int:
    return lib().or_nterms(p)


def term_index(n1: int, n2: int, n3: int) -> int:
    return lib().or_term_index(n1, n2, n3)


def taylor(p: int, R) -> np.ndarray:
    R, Rp = _d(R)
    T = np.zeros(nterms(p))
    lib().or_taylor(p, Rp, T.ctypes.data_as(_dp))
    return T


def direct_energy_raw(q, xyz, lB=1.0) -> float:
    q, qp = _d(q)
    x, xp = _d(np.reshape(xyz, (-1, 3)))
    return lib().or_direct_energy_raw(len(q), qp, xp, lB)


def make_params(d: dict) -> Params:
    P = Params()
    P.lB = d.get("lB", 1.0)
    P.beta = d.get("beta", 1.0)
    P.theta = d["theta"]
    P.p = d["p"]
    P.N0 = d.get("N0", 0)
    P.C = d["C"]
    P.Dmax = d["Dmax"]
    for a in range(3):
        P.root_lo[a] = d["root_lo"][a]
    P.root_side = d["root_side"]
    P.shell = 1 if d.get("shell") else 0
    P.shell_rmin, P.shell_rmax = (d["shell"] if d.get("shell") else (0.0, 0.0))
    P.images = 1 if d.get("image") else 0
    P.image_R, P.image_alpha = (d["image"] if d.get("image") else (0.0, 0.0))
    P.hard_core = d.get("hard_core", 0.0) or 0.0
    P.fixed_depth = 1 if d.get("fixed_depth", False) else 0
    P.fixed_direct = 1 if d.get("fixed_direct", False) else 0
    return P


class System:
    """A charged system with its octree (oracle side)."""

    def __init__(self, params: dict, q, xyz, n_mobile: int, n_fixed: int = 0):
        self._P = make_params(params)
        self.params = dict(params)
        q, qp = _d(q)
        x, xp = _d(np.reshape(xyz, (-1, 3)))
        st = C.c_int(0)
        self._h = lib().or_create(C.byref(self._P), n_mobile, n_fixed, qp, xp, C.byref(st))
        self.status = st.value
        if not self._h:
            raise ValueError("oracle create failed with status %d" % st.value)
        self.n_mobile = n_mobile
        self.n_fixed = n_fixed
        self.n_charges = lib().or_n_charges(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def set_bound(self, on=True):
        lib().or_set_bound(self._h, 1 if on else 0)

    def charges(self):
        q = np.zeros(self.n_charges)
        x = np.zeros((self.n_charges, 3))
        lib().or_get_charges(self._h, q.ctypes.data_as(_dp), x.ctypes.data_as(_dp))
        return q, x

    def image_of(self, r, q):
        r, rp = _d(r)
        o = np.zeros(3)
        qi = C.c_double(0)
        st = lib().or_image_of(self._h, rp, q, o.ctypes.data_as(_dp), C.byref(qi))
        return st, o, qi.value

    def phi(self, x, excl=()):
        x, xp = _d(x)
        ex = np.ascontiguousarray(excl, dtype=np.int64)
        e = Eval()
        lib().or_phi(self._h, xp, len(ex), ex.ctypes.data_as(_i64p), C.byref(e))
        return e

    def phi_direct(self, x, excl=()):
        x, xp = _d(x)
        ex = np.ascontiguousarray(excl, dtype=np.int64)
        return lib().or_phi_direct(self._h, xp, len(ex), ex.ctypes.data_as(_i64p))

    def delta_energy(self, i, b) -> DE:
        b, bp = _d(b)
        e = DE()
        lib().or_delta_energy(self._h, int(i), bp, C.byref(e))
        return e

    def delta_energy_direct(self, i, b):
        b, bp = _d(b)
        v = C.c_double(0)
        st = lib().or_delta_energy_direct(self._h, int(i), bp, C.byref(v))
        return st, v.value

    def commit_move(self, i, b) -> int:
        b, bp = _d(b)
        return lib().or_commit_move(self._h, int(i), bp)

    def capacity_violation(self, i, b) -> bool:
        b, bp = _d(b)
        return bool(lib().or_capacity_violation(self._h, int(i), bp))

    def mc_run(self, seed, n_moves, step=1.0, m0=0, replica=0):
        recs = np.zeros(n_moves, dtype=RECORD_DTYPE)
        acc = C.c_int64(0)
        lib().or_mc_run(self._h, seed, replica, m0, n_moves, step,
                        recs.ctypes.data_as(C.c_void_p), C.byref(acc))
        return recs

    def phi_grad(self, x, excl=()):
        x, xp = _d(x)
        ex = np.ascontiguousarray(excl, dtype=np.int64)
        phi = C.c_double(0)
        g = np.zeros(3)
        lib().or_phi_grad(self._h, xp, len(ex), ex.ctypes.data_as(_i64p), C.byref(phi),
                          g.ctypes.data_as(_dp))
        return phi.value, g

    def ion_energy_grad(self, i, x):
        x, xp = _d(x)
        U = C.c_double(0)
        g = np.zeros(3)
        lib().or_ion_energy_grad(self._h, int(i), xp, C.byref(U), g.ctypes.data_as(_dp))
        return U.value, g

    def mala_run(self, seed, n_moves, tau=0.05, m0=0, replica=0):
        recs = np.zeros(n_moves, dtype=RECORD_DTYPE)
        acc = C.c_int64(0)
        lib().or_mala_run(self._h, seed, replica, m0, n_moves, tau,
                          recs.ctypes.data_as(C.c_void_p), C.byref(acc))
        return recs

    def energy_direct(self) -> float:
        return lib().or_energy_direct(self._h)

    def energy_tree(self) -> float:
        return lib().or_energy_tree(self._h)

    def potentials(self):
        vt = np.zeros(self.n_charges)
        vd = np.zeros(self.n_charges)
        lib().or_potentials(self._h, vt.ctypes.data_as(_dp), vd.ctypes.data_as(_dp))
        return vt, vd

    def forces(self):
        """(dE/dr (n x 3), dE/dq (n)) of the treecode energy, MAC decisions fixed."""
        g = np.zeros((self.n_charges, 3))
        dq = np.zeros(self.n_charges)
        rc = lib().or_forces(self._h, g.ctypes.data_as(_dp), dq.ctypes.data_as(_dp))
        if rc:
            raise ValueError("or_forces failed with status %d" % rc)
        return g, dq

    def forces_abs(self):
        """Conditioning sums (A_r (n x 3), A_q (n)): the adjoint with every term
        replaced by its magnitude."""
        g = np.zeros((self.n_charges, 3))
        dq = np.zeros(self.n_charges)
        rc = lib().or_forces_abs(self._h, g.ctypes.data_as(_dp), dq.ctypes.data_as(_dp))
        if rc:
            raise ValueError("or_forces_abs failed with status %d" % rc)
        return g, dq

    def radial_counts(self, nbins, r_lo, r_hi, counts=None, charge=None):
        """Add the mobile ions' radial bins (Sec. 4) to counts / charge (new arrays if None)."""
        counts = np.zeros(nbins, dtype=np.int64) if counts is None else counts
        charge = np.zeros(nbins) if charge is None else charge
        rc = lib().or_radial_counts(self._h, nbins, r_lo, r_hi, counts.ctypes.data_as(_i64p),
                                    charge.ctypes.data_as(_dp))
        if rc:
            raise ValueError("or_radial_counts failed with status %d" % rc)
        return counts, charge

    def export_tree(self):
        """{(depth, key): (is_leaf, count, members-tuple or None)}"""
        cap = 8 * self.n_charges + 64
        mem = np.zeros(self.n_charges + 8, dtype=np.int64)
        while True:  # deep (fixed-level) trees hold more clusters than charges
            rows = np.zeros((cap, 4), dtype=np.int64)
            n = lib().or_export_tree(self._h, rows.ctypes.data_as(_i64p), cap,
                                     mem.ctypes.data_as(_i64p), len(mem))
            if n >= 0:
                break
            if cap > 64 * (self.n_charges + 64) * 21:
                raise RuntimeError("export buffer too small")
            cap *= 4
        out = {}
        off = 0
        for d, k, leaf, cnt in rows[:n]:
            members = None
            if leaf:
                members = tuple(int(v) for v in mem[off:off + cnt])
                off += cnt
            out[(int(d), int(k))] = (bool(leaf), int(cnt), members)
        return out

    def check(self) -> int:
        return lib().or_check(self._h)

    def node_moments(self, depth, key):
        M = np.zeros(nterms(self.params["p"]))
        st = lib().or_node_moments(self._h, depth, key, M.ctypes.data_as(_dp))
        return st, M

    def point_key(self, x) -> int:
        x, xp = _d(x)
        return int(lib().or_point_key(self._h, xp))


def radial_profiles(counts, charge, r_lo, r_hi, n_samples, q_fixed=0.0):
    """(bin centres, g, outer edges, Q) of Sec. 4 from accumulated counts (or_radial_profiles)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    charge = np.ascontiguousarray(charge, dtype=np.float64)
    n = len(counts)
    out = [np.zeros(n) for _ in range(4)]
    rc = lib().or_radial_profiles(n, r_lo, r_hi, counts.ctypes.data_as(_i64p), charge.ctypes.data_as(_dp),
                                  int(n_samples), q_fixed, *[o.ctypes.data_as(_dp) for o in out])
    if rc:
        raise ValueError("or_radial_profiles failed with status %d" % rc)
    return tuple(out)

