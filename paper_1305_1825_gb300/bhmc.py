"""ctypes binding of libbhmc.so (the C-ABI of include/bhmc.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The module-level functions carry the C names; ``Context`` and ``Batch`` are
thin owners of the handles.  Arrays may be numpy (host) or torch CUDA tensors
(device pointers, passed with BHMC_DEVICE_PTRS); the CUDA stream is torch's
current stream when torch is available.  If the library is missing this module
raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

OK, EINVAL, EDOMAIN, EOVERLAP, ENOMEM, ENOMEM_POOL, ECUDA, ETIMEOUT, ESTATE, ECAPACITY, ESTACK, ESCRATCH, ENONFINITE = range(13)
PREC_F32, PREC_F64 = 0, 1
LAYOUT_SOA, LAYOUT_AOS = 0, 1
HOST_PTRS, DEVICE_PTRS = 0, 1
ACCEPT, REJECT_ENERGY, REJECT_DOMAIN, REJECT_OVERLAP, REJECT_CAPACITY = range(5)


class BhmcError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, bhmc_status_string(status), status))


class Params(C.Structure):
    _fields_ = [
        ("lB", C.c_double), ("beta", C.c_double), ("theta", C.c_double),
        ("p", C.c_int32), ("N0", C.c_int32), ("C", C.c_int32), ("Dmax", C.c_int32),
        ("root_lo", C.c_double * 3), ("root_side", C.c_double),
        ("shell", C.c_int32), ("shell_rmin", C.c_double), ("shell_rmax", C.c_double),
        ("images", C.c_int32), ("image_R", C.c_double), ("image_alpha", C.c_double),
        ("precision", C.c_int32), ("warps", C.c_int32), ("layout", C.c_int32),
        ("node_factor", C.c_double), ("hard_core", C.c_double), ("fixed_depth", C.c_int32),
        ("fixed_direct", C.c_int32), ("round_limit", C.c_int32),
    ]


class Counters(C.Structure):
    _fields_ = [("visited", C.c_int64), ("accepted", C.c_int64), ("pairs", C.c_int64),
                ("mac_fp64", C.c_int64)]


class McStats(C.Structure):
    _fields_ = [("moves", C.c_int64), ("accepted", C.c_int64), ("rej_energy", C.c_int64),
                ("rej_domain", C.c_int64), ("rej_overlap", C.c_int64), ("rej_capacity", C.c_int64),
                ("flagged", C.c_int64), ("energy", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


RECORD_DTYPE = np.dtype([("i", "<i8"), ("r_new", "<f8", (3,)), ("dE", "<f8"), ("outcome", "<i4"),
                         ("flagged", "<i4")])

_lib = None
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


def lib():
    """Open libbhmc.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libbhmc.so is not built (run __graft_entry__.build()); "
                               "the CUDA library is required, there is no CPU fallback")
        L = C.CDLL(_build.LIB)
        st = C.c_int
        L.bhmc_status_string.argtypes = [st]
        L.bhmc_status_string.restype = C.c_char_p
        L.bhmc_create.argtypes = [C.POINTER(Params), C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                  C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]
        L.bhmc_destroy.argtypes = [C.c_void_p]
        L.bhmc_n_charges.argtypes = [C.c_void_p, _i64p]
        L.bhmc_get_charges.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
        L.bhmc_get_positions.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
        L.bhmc_get_counters.argtypes = [C.c_void_p, C.POINTER(Counters)]
        L.bhmc_delta_energy.argtypes = [C.c_void_p, C.c_int64, _dp, _dp, C.POINTER(Counters)]
        L.bhmc_commit_move.argtypes = [C.c_void_p, C.c_int64, _dp]
        L.bhmc_step_mc.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.c_uint64, C.c_uint64,
                                   C.POINTER(McStats), C.c_void_p]
        L.bhmc_step_mc_spec.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.c_uint64, C.c_uint64,
                                        C.c_int32, C.POINTER(McStats), C.c_void_p]
        L.bhmc_energy_counters.argtypes = [C.c_void_p, _dp, C.POINTER(Counters)]
        L.bhmc_radial_counts.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, _i64p, _dp]
        L.bhmc_batch_radial_counts.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, _i64p, _dp]
        L.bhmc_set_radial_sampling.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_int64]
        L.bhmc_get_radial_samples.argtypes = [C.c_void_p, _i64p, _dp, _i64p]
        L.bhmc_batch_set_radial_sampling.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_int64]
        L.bhmc_batch_get_radial_samples.argtypes = [C.c_void_p, _i64p, _dp, _i64p]
        L.bhmc_radial_profiles.argtypes = [C.c_int32, C.c_double, C.c_double, _i64p, _dp, C.c_int64, C.c_double,
                                           _dp, _dp, _dp, _dp]
        L.bhmc_step_mala.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.c_uint64, C.c_uint64,
                                     C.POINTER(McStats), C.c_void_p]
        L.bhmc_get_energy.argtypes = [C.c_void_p, _dp]
        L.bhmc_set_energy.argtypes = [C.c_void_p, C.c_double]
        L.bhmc_energy.argtypes = [C.c_void_p, _dp]
        L.bhmc_energy_direct.argtypes = [C.c_void_p, _dp]
        L.bhmc_potentials.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
        L.bhmc_forces.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
        L.bhmc_export_tree.argtypes = [C.c_void_p, _i64p, C.c_int64, _i64p, C.c_int64, _dp, _i64p]
        L.bhmc_batch_create.argtypes = [C.c_int32, C.POINTER(Params), _i64p, _i64p,
                                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int32,
                                        C.c_void_p, C.POINTER(C.c_void_p)]
        L.bhmc_batch_destroy.argtypes = [C.c_void_p]
        L.bhmc_batch_replica.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]
        L.bhmc_batch_step_mc.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(C.c_uint64),
                                         C.c_uint64, C.POINTER(McStats)]
        L.bhmc_batch_step_mc_records.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(C.c_uint64),
                                                 C.c_uint64, C.POINTER(McStats), C.c_void_p]
        L.bhmc_batch_step_mc_spec.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(C.c_uint64),
                                              C.c_uint64, C.c_int32, C.POINTER(McStats)]
        _lib = L
    return _lib


def bhmc_status_string(status: int) -> str:
    try:
        return lib().bhmc_status_string(status).decode()
    except Exception:  # library not loadable: still describe the code
        return "status %d" % status


def _check(rc, what):
    if rc != OK:
        raise BhmcError(rc, what)


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


def make_params(d: dict, precision=PREC_F32, warps=2, layout=LAYOUT_SOA, node_factor=0.0) -> Params:
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
    P.shell_rmin, P.shell_rmax = d["shell"] if d.get("shell") else (0.0, 0.0)
    P.images = 1 if d.get("image") else 0
    P.image_R, P.image_alpha = d["image"] if d.get("image") else (0.0, 0.0)
    P.precision = d.get("precision", precision)
    P.warps = d.get("warps", warps)
    P.layout = d.get("layout", layout)
    P.node_factor = d.get("node_factor", node_factor)
    P.hard_core = d.get("hard_core", 0.0) or 0.0
    P.fixed_depth = 1 if d.get("fixed_depth", False) else 0
    P.fixed_direct = 1 if d.get("fixed_direct", False) else 0
    P.round_limit = int(d.get("round_limit", 0))
    return P


def _ptr_and_flag(a):
    """(pointer, flags, keepalive) for a numpy array or a torch CUDA tensor of float64."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64:
                raise TypeError("float64 tensors required")
            a = a.contiguous()
            return C.c_void_p(a.data_ptr()), (DEVICE_PTRS if a.is_cuda else HOST_PTRS), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a, dtype=np.float64)
    return C.c_void_p(a.ctypes.data), HOST_PTRS, a


# ------------------------------------------------------------------ C-named wrappers
def bhmc_create(params: Params, n_mobile: int, n_fixed: int, q, xyz, stream=None):
    qp, f1, kq = _ptr_and_flag(q)
    xp, f2, kx = _ptr_and_flag(xyz)
    if f1 != f2:
        raise ValueError("q and xyz must both be host or both device arrays")
    h = C.c_void_p()
    _check(lib().bhmc_create(C.byref(params), n_mobile, n_fixed, qp, xp, f1, _stream(stream),
                             C.byref(h)), "bhmc_create")
    return h


def bhmc_destroy(h):
    _check(lib().bhmc_destroy(h), "bhmc_destroy")


def bhmc_delta_energy(h, i, r_new):
    b = (C.c_double * 3)(*[float(v) for v in r_new])
    dE = C.c_double()
    cnt = Counters()
    rc = lib().bhmc_delta_energy(h, int(i), b, C.byref(dE), C.byref(cnt))
    return rc, dE.value, cnt


def bhmc_commit_move(h, i, r_new):
    b = (C.c_double * 3)(*[float(v) for v in r_new])
    return lib().bhmc_commit_move(h, int(i), b)


def bhmc_step_mc(h, n_moves, step, seed, move0=0, records=False):
    st = McStats()
    rec = np.zeros(n_moves, dtype=RECORD_DTYPE) if records else None
    rp = C.c_void_p(rec.ctypes.data) if records and n_moves else C.c_void_p(0)
    _check(lib().bhmc_step_mc(h, n_moves, step, seed, move0, C.byref(st), rp), "bhmc_step_mc")
    return st, rec


def bhmc_step_mc_spec(h, n_moves, step, seed, move0=0, proposals=4, records=False):
    st = McStats()
    rec = np.zeros(n_moves, dtype=RECORD_DTYPE) if records else None
    rp = C.c_void_p(rec.ctypes.data) if records and n_moves else C.c_void_p(0)
    _check(lib().bhmc_step_mc_spec(h, n_moves, step, seed, move0, proposals, C.byref(st), rp),
           "bhmc_step_mc_spec")
    return st, rec


def bhmc_step_mala(h, n_moves, tau, seed, move0=0, records=False):
    st = McStats()
    rec = np.zeros(n_moves, dtype=RECORD_DTYPE) if records else None
    rp = C.c_void_p(rec.ctypes.data) if records and n_moves else C.c_void_p(0)
    _check(lib().bhmc_step_mala(h, n_moves, tau, seed, move0, C.byref(st), rp), "bhmc_step_mala")
    return st, rec


def bhmc_energy(h):
    e = C.c_double()
    _check(lib().bhmc_energy(h, C.byref(e)), "bhmc_energy")
    return e.value


def bhmc_energy_counters(h):
    e = C.c_double()
    c = Counters()
    _check(lib().bhmc_energy_counters(h, C.byref(e), C.byref(c)), "bhmc_energy_counters")
    return e.value, c


def bhmc_radial_counts(h, counts, charge, r_lo, r_hi, batch=False):
    """Adds the radial counts and charges of the mobile ions to the int64 and
    float64 numpy arrays counts and charge (one entry per bin)."""
    f = lib().bhmc_batch_radial_counts if batch else lib().bhmc_radial_counts
    _check(f(h, len(counts), r_lo, r_hi, counts.ctypes.data_as(_i64p), charge.ctypes.data_as(_dp)),
           "bhmc_radial_counts")


def radial_profiles(counts, charge, r_lo, r_hi, samples, q_fixed=0.0):
    """(bin centres, g, outer edges, Q) of Sec. 4 from accumulated radial counts
    (bhmc_radial_profiles)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    charge = np.ascontiguousarray(charge, dtype=np.float64)
    n = len(counts)
    out = [np.zeros(n) for _ in range(4)]
    _check(lib().bhmc_radial_profiles(n, r_lo, r_hi, counts.ctypes.data_as(_i64p), charge.ctypes.data_as(_dp),
                                      int(samples), q_fixed, *[o.ctypes.data_as(_dp) for o in out]),
           "bhmc_radial_profiles")
    return tuple(out)


def bhmc_set_radial_sampling(h, nbins, r_lo, r_hi, every, batch=False):
    f = lib().bhmc_batch_set_radial_sampling if batch else lib().bhmc_set_radial_sampling
    _check(f(h, nbins, r_lo, r_hi, every), "bhmc_set_radial_sampling")


def bhmc_get_radial_samples(h, nbins, n_rep=None):
    """(counts, charge, n_samples); with n_rep, per replica arrays [n_rep, nbins]."""
    shape = (nbins,) if n_rep is None else (n_rep, nbins)
    counts = np.zeros(shape, dtype=np.int64)
    charge = np.zeros(shape)
    ns = np.zeros(1 if n_rep is None else n_rep, dtype=np.int64)
    f = lib().bhmc_get_radial_samples if n_rep is None else lib().bhmc_batch_get_radial_samples
    _check(f(h, counts.ctypes.data_as(_i64p), charge.ctypes.data_as(_dp), ns.ctypes.data_as(_i64p)),
           "bhmc_get_radial_samples")
    return counts, charge, (int(ns[0]) if n_rep is None else ns)


def bhmc_energy_direct(h):
    e = C.c_double()
    _check(lib().bhmc_energy_direct(h, C.byref(e)), "bhmc_energy_direct")
    return e.value


def bhmc_potentials(h):
    phi = np.zeros(bhmc_n_charges(h))
    _check(lib().bhmc_potentials(h, C.c_void_p(phi.ctypes.data), HOST_PTRS), "bhmc_potentials")
    return phi


def bhmc_forces(h, dEdr=None, dEdq=None):
    """(dE/dr (n x 3), dE/dq (n)); torch CUDA tensors given as outputs are filled in place."""
    if dEdr is None:
        n = bhmc_n_charges(h)
        g = np.zeros((n, 3))
        dq = np.zeros(n)
        _check(lib().bhmc_forces(h, C.c_void_p(g.ctypes.data), C.c_void_p(dq.ctypes.data), HOST_PTRS),
               "bhmc_forces")
        return g, dq
    _check(lib().bhmc_forces(h, C.c_void_p(dEdr.data_ptr()), C.c_void_p(dEdq.data_ptr()), DEVICE_PTRS),
           "bhmc_forces")
    return dEdr, dEdq


def bhmc_get_energy(h):
    e = C.c_double()
    _check(lib().bhmc_get_energy(h, C.byref(e)), "bhmc_get_energy")
    return e.value


def bhmc_set_energy(h, E):
    _check(lib().bhmc_set_energy(h, float(E)), "bhmc_set_energy")


def bhmc_n_charges(h):
    n = C.c_int64()
    _check(lib().bhmc_n_charges(h, C.byref(n)), "bhmc_n_charges")
    return n.value


def bhmc_get_charges(h):
    n = bhmc_n_charges(h)
    q = np.zeros(n)
    x = np.zeros((n, 3))
    _check(lib().bhmc_get_charges(h, C.c_void_p(q.ctypes.data), C.c_void_p(x.ctypes.data), HOST_PTRS),
           "bhmc_get_charges")
    return q, x


def bhmc_get_positions(h):
    n = bhmc_n_charges(h)
    x = np.zeros((n, 3))
    _check(lib().bhmc_get_positions(h, C.c_void_p(x.ctypes.data), HOST_PTRS), "bhmc_get_positions")
    return x


def bhmc_get_counters(h):
    c = Counters()
    _check(lib().bhmc_get_counters(h, C.byref(c)), "bhmc_get_counters")
    return c


def bhmc_export_tree(h, K=None):
    """{(depth, key): (is_leaf, count, members or None)} and, if K is given, moments per key."""
    n = bhmc_n_charges(h)
    cap = 8 * n + 1024
    mem = np.zeros(n + 8, dtype=np.int64)
    nr = C.c_int64()
    for attempt in range(4):  # deep (fixed-level) trees hold more clusters than charges
        rows = np.zeros((cap, 4), dtype=np.int64)
        M = np.zeros((cap, K)) if K else None
        rc = lib().bhmc_export_tree(h, rows.ctypes.data_as(_i64p), cap, mem.ctypes.data_as(_i64p), len(mem),
                                    M.ctypes.data_as(_dp) if K else None, C.byref(nr))
        if rc != EINVAL or attempt == 3:
            break
        cap *= 8
    _check(rc, "bhmc_export_tree")
    tree, moms = {}, {}
    off = 0
    for r in range(nr.value):
        d, k, leaf, cnt = (int(v) for v in rows[r])
        members = None
        if leaf:
            members = tuple(int(v) for v in mem[off:off + cnt])
            off += cnt
        tree[(d, k)] = (bool(leaf), cnt, members)
        if K:
            moms[(d, k)] = M[r].copy()
    return (tree, moms) if K else tree


def bhmc_batch_create(params: Params, systems, stream=None):
    n = len(systems)
    nm = (C.c_int64 * n)(*[s["n_mobile"] for s in systems])
    nf = (C.c_int64 * n)(*[s["n_fixed"] for s in systems])
    keep = []
    qs = (C.c_void_p * n)()
    xs = (C.c_void_p * n)()
    flag = None
    for r, s in enumerate(systems):
        qp, f1, kq = _ptr_and_flag(s["q"])
        xp, f2, kx = _ptr_and_flag(s["xyz"])
        if flag is None:
            flag = f1
        if f1 != flag or f2 != flag:
            raise ValueError("all arrays must be host or all device")
        keep += [kq, kx]
        qs[r] = qp.value
        xs[r] = xp.value
    h = C.c_void_p()
    _check(lib().bhmc_batch_create(n, C.byref(params), nm, nf, qs, xs, flag, _stream(stream), C.byref(h)),
           "bhmc_batch_create")
    return h


def bhmc_batch_destroy(h):
    _check(lib().bhmc_batch_destroy(h), "bhmc_batch_destroy")


def bhmc_batch_replica(h, r):
    c = C.c_void_p()
    _check(lib().bhmc_batch_replica(h, r, C.byref(c)), "bhmc_batch_replica")
    return c


def bhmc_batch_step_mc(h, n_rep, n_moves, step, seeds, move0=0):
    sd = (C.c_uint64 * n_rep)(*[int(s) for s in seeds])
    st = (McStats * n_rep)()
    _check(lib().bhmc_batch_step_mc(h, n_moves, step, sd, move0, st), "bhmc_batch_step_mc")
    return [s.as_dict() for s in st]


def bhmc_batch_step_mc_records(h, n_rep, n_moves, step, seeds, move0=0):
    """(stats, records[n_rep, n_moves]) of one batched launch."""
    sd = (C.c_uint64 * n_rep)(*[int(s) for s in seeds])
    st = (McStats * n_rep)()
    rec = np.zeros((n_rep, n_moves), dtype=RECORD_DTYPE)
    _check(lib().bhmc_batch_step_mc_records(h, n_moves, step, sd, move0, st, C.c_void_p(rec.ctypes.data)),
           "bhmc_batch_step_mc_records")
    return [s.as_dict() for s in st], rec


def bhmc_batch_step_mc_spec(h, n_rep, n_moves, step, seeds, move0=0, proposals=4):
    sd = (C.c_uint64 * n_rep)(*[int(s) for s in seeds])
    st = (McStats * n_rep)()
    _check(lib().bhmc_batch_step_mc_spec(h, n_moves, step, sd, move0, proposals, st), "bhmc_batch_step_mc_spec")
    return [s.as_dict() for s in st]


# ------------------------------------------------------------------ owners
class Context:
    """One system and its device-resident octree."""

    def __init__(self, workload: dict, precision=PREC_F32, warps=2, layout=LAYOUT_SOA, node_factor=0.0,
                 stream=None, _handle=None):
        self.params = make_params(workload["params"], precision, warps, layout, node_factor)
        self.K = (self.params.p + 1) * (self.params.p + 2) * (self.params.p + 3) // 6
        self.n_mobile = workload["n_mobile"]
        self.n_fixed = workload["n_fixed"]
        self._owned = _handle is None
        self.h = _handle if _handle is not None else bhmc_create(
            self.params, self.n_mobile, self.n_fixed, workload["q"], workload["xyz"], stream)

    def close(self):
        if self._owned and self.h:
            bhmc_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def delta_energy(self, i, r_new):
        return bhmc_delta_energy(self.h, i, r_new)

    def commit_move(self, i, r_new):
        return bhmc_commit_move(self.h, i, r_new)

    def step_mc(self, n_moves, step, seed, move0=0, records=False):
        return bhmc_step_mc(self.h, n_moves, step, seed, move0, records)

    def step_mc_spec(self, n_moves, step, seed, move0=0, proposals=4, records=False):
        return bhmc_step_mc_spec(self.h, n_moves, step, seed, move0, proposals, records)

    def step_mala(self, n_moves, tau, seed, move0=0, records=False):
        return bhmc_step_mala(self.h, n_moves, tau, seed, move0, records)

    def energy(self):
        return bhmc_energy(self.h)

    def energy_counters(self):
        return bhmc_energy_counters(self.h)

    def radial_counts(self, counts, charge, r_lo, r_hi):
        bhmc_radial_counts(self.h, counts, charge, r_lo, r_hi)

    def set_radial_sampling(self, nbins, r_lo, r_hi, every):
        self._rdf_nbins = nbins
        bhmc_set_radial_sampling(self.h, nbins, r_lo, r_hi, every)

    def radial_samples(self):
        return bhmc_get_radial_samples(self.h, self._rdf_nbins)

    def energy_direct(self):
        return bhmc_energy_direct(self.h)

    def potentials(self):
        return bhmc_potentials(self.h)

    def forces(self, dEdr=None, dEdq=None):
        return bhmc_forces(self.h, dEdr, dEdq)

    def get_energy(self):
        return bhmc_get_energy(self.h)

    def set_energy(self, E):
        bhmc_set_energy(self.h, E)

    def charges(self):
        return bhmc_get_charges(self.h)

    def positions(self):
        return bhmc_get_positions(self.h)

    def counters(self):
        return bhmc_get_counters(self.h)

    def export_tree(self, moments=False):
        return bhmc_export_tree(self.h, self.K if moments else None)


class Batch:
    """Independent replicas, each with its own octree, stepped in one persistent launch."""

    def __init__(self, systems, precision=PREC_F32, warps=2, layout=LAYOUT_SOA, node_factor=0.0, stream=None):
        self.params = make_params(systems[0]["params"], precision, warps, layout, node_factor)
        self.n = len(systems)
        self.systems = systems
        self.h = bhmc_batch_create(self.params, systems, stream)

    def replica(self, r) -> Context:
        c = Context.__new__(Context)
        c.params = self.params
        c.K = (self.params.p + 1) * (self.params.p + 2) * (self.params.p + 3) // 6
        c.n_mobile = self.systems[r]["n_mobile"]
        c.n_fixed = self.systems[r]["n_fixed"]
        c._owned = False
        c.h = bhmc_batch_replica(self.h, r)
        return c

    def step_mc(self, n_moves, step, seeds, move0=0, records=False):
        if records:
            return bhmc_batch_step_mc_records(self.h, self.n, n_moves, step, seeds, move0)
        return bhmc_batch_step_mc(self.h, self.n, n_moves, step, seeds, move0)

    def step_mc_spec(self, n_moves, step, seeds, move0=0, proposals=4):
        return bhmc_batch_step_mc_spec(self.h, self.n, n_moves, step, seeds, move0, proposals)

    def radial_counts(self, counts, charge, r_lo, r_hi):
        bhmc_radial_counts(self.h, counts, charge, r_lo, r_hi, batch=True)

    def set_radial_sampling(self, nbins, r_lo, r_hi, every):
        self._rdf_nbins = nbins
        bhmc_set_radial_sampling(self.h, nbins, r_lo, r_hi, every, batch=True)

    def radial_samples(self):
        """(counts [n_rep, nbins], charge [n_rep, nbins], n_samples [n_rep])."""
        return bhmc_get_radial_samples(self.h, self._rdf_nbins, n_rep=self.n)

    def close(self):
        if self.h:
            bhmc_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
