"""ctypes wrapper around ``soma_oracle.cpp`` (test infrastructure only).

Argument marshalling only: every number comes from the C++ oracle.  See the
header of ``soma_oracle.cpp`` for the model and for what pins each function.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "soma_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")


def library_path():
    return _LIB


def build_oracle(force=False):
    """Compile the oracle with g++ (FP64, OpenMP over chains within a set)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC]
    subprocess.check_call(cmd)
    return _LIB


class OrcDesc(ctypes.Structure):
    _fields_ = [
        ("n_poly", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("n_A", ctypes.c_int32),
        ("sys_index", ctypes.c_int32),
        ("grid", ctypes.c_int32 * 3),
        ("move", ctypes.c_int32),
        ("box", ctypes.c_double * 3),
        ("chiN", ctypes.c_double),
        ("kappaN", ctypes.c_double),
        ("A", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("wall_z", ctypes.c_int32),
        ("pos64", ctypes.c_int32),
        ("conv", ctypes.c_int32),
        ("n_A_alt", ctypes.c_int32),
        ("zone_lo", ctypes.c_double),
        ("zone_hi", ctypes.c_double),
        ("thr", ctypes.c_uint64 * 4),
        ("mol", ctypes.POINTER(ctypes.c_uint8)),
    ]


class OrcObs(ctypes.Structure):
    _fields_ = [("Re2", ctypes.c_double), ("Rg2", ctypes.c_double),
                ("Ebond", ctypes.c_double), ("Enb", ctypes.c_double)]


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


class Oracle:
    """One system of the oracle: descriptor plus convenience wrappers."""

    _lib = None
    _path = None

    @classmethod
    def with_library(cls, path):
        """A subclass bound to another build of the oracle source (mutation tests)."""
        return type("OracleAt", (cls,), {"_lib": None, "_path": path})

    @classmethod
    def lib(cls):
        if cls._lib is None:
            path = cls._path or build_oracle()
            L = ctypes.CDLL(path)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            f64p = ctypes.POINTER(ctypes.c_double)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            dp = ctypes.POINTER(OrcDesc)
            L.orc_philox4x32_many.argtypes = [ctypes.c_int64, u32p, u32p, u32p]
            L.orc_params.argtypes = [dp, f64p, f64p, f64p]
            L.orc_cell_index.argtypes = [dp, f64p]
            L.orc_cell_index.restype = ctypes.c_int64
            L.orc_init.argtypes = [dp, f64p]
            L.orc_density.argtypes = [dp, f64p, u32p]
            L.orc_fields.argtypes = [dp, u32p, f64p]
            L.orc_normal_quantile.argtypes = [ctypes.c_double]
            L.orc_normal_quantile.restype = ctypes.c_double
            L.orc_energy_nb.argtypes = [dp, u32p]
            L.orc_energy_nb.restype = ctypes.c_double
            L.orc_fields_from_phi.argtypes = [dp, f64p, f64p]
            L.orc_mc_step.argtypes = [dp, f64p, f64p, ctypes.c_uint32, u8p, f64p, f64p, ctypes.c_int]
            L.orc_mc_step.restype = ctypes.c_int64
            L.orc_mc_step_chains.argtypes = [dp, f64p, u32p, ctypes.c_int64, f64p, ctypes.c_uint32, u8p, f64p,
                                             f64p, ctypes.c_int]
            L.orc_mc_step_chains.restype = ctypes.c_int64
            L.orc_observables.argtypes = [dp, f64p, ctypes.POINTER(OrcObs)]
            L.orc_structure_factor.argtypes = [dp, f64p, ctypes.c_int, i32p, f64p]
            L.orc_run.argtypes = [dp, f64p, ctypes.c_uint32, ctypes.c_int64, f64p, f64p, ctypes.c_double,
                                  ctypes.c_int, u64p, u64p, f64p, i64p]
            L.orc_energy_umbrella.argtypes = [dp, u32p, f64p, ctypes.c_double]
            L.orc_energy_umbrella.restype = ctypes.c_double
            L.orc_fields_umbrella.argtypes = [dp, u32p, f64p, ctypes.c_double, f64p]
            L.orc_place.argtypes = [dp, ctypes.POINTER(ctypes.c_float), f64p]
            L.orc_density_profile.argtypes = [dp, u32p, ctypes.c_int, f64p]
            L.orc_vertical_correlation.argtypes = [dp, u32p, ctypes.c_int, f64p]
            L.orc_place.restype = ctypes.c_int
            L.orc_run.restype = ctypes.c_int64
            L.orc_conversion_threshold.argtypes = [ctypes.c_double]
            L.orc_conversion_threshold.restype = ctypes.c_uint64
            L.orc_convert.argtypes = [dp, f64p, ctypes.c_uint32, i64p]
            cls._lib = L
        return cls._lib

    def __init__(self, n_poly, N, n_A, box, grid, chiN, kappaN, A=0.0, seed=1, sys_index=0, move=0, wall_z=0,
                 pos64=0):
        self.d = OrcDesc()
        self.d.n_poly, self.d.N, self.d.n_A, self.d.sys_index = n_poly, N, n_A, sys_index
        self.d.move = int(move)
        self.d.wall_z = int(wall_z)
        self.d.pos64 = int(pos64)
        for a in range(3):
            self.d.grid[a] = int(grid[a])
            self.d.box[a] = float(box[a])
        self.d.chiN, self.d.kappaN, self.d.A, self.d.seed = float(chiN), float(kappaN), float(A), int(seed)
        self.n_b = n_poly * N
        self.n_c = int(grid[0]) * int(grid[1]) * int(grid[2])
        self.types = None

    # -- molecule types and boundary-zone conversion ---------------------
    def set_conversion(self, n_A_alt, zone_lo, zone_hi, p):
        """Chains carry molecule types (all 0 at first) and convert in the
        zones; p = per-step probabilities (bottom 0->1, bottom 1->0, top 0->1,
        top 1->0), turned into thresholds by the oracle."""
        self.d.conv = 1
        self.d.n_A_alt = int(n_A_alt)
        self.d.zone_lo, self.d.zone_hi = float(zone_lo), float(zone_hi)
        for k in range(4):
            self.d.thr[k] = int(self.lib().orc_conversion_threshold(float(p[k])))
        if self.types is None:
            self.types = np.zeros(self.d.n_poly, np.uint8)
            self.d.mol = self.types.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))

    def set_types(self, types):
        """Molecule type of every logical chain (copied in; conversion must be on)."""
        assert self.types is not None
        self.types[:] = np.asarray(types, np.uint8)

    def convert(self, pos, t):
        """The boundary-zone conversions that open step t (types change in
        place); returns the counts (bottom 0->1, bottom 1->0, top 0->1, top 1->0)."""
        pos = np.ascontiguousarray(pos, np.float64)
        c4 = np.zeros(4, np.int64)
        self.lib().orc_convert(ctypes.byref(self.d), _p(pos, ctypes.c_double), ctypes.c_uint32(t & 0xFFFFFFFF),
                               _p(c4, ctypes.c_int64))
        return c4

    # -- constants -------------------------------------------------------
    def params(self):
        kb, A, rho = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self.lib().orc_params(ctypes.byref(self.d), ctypes.byref(kb), ctypes.byref(A), ctypes.byref(rho))
        return kb.value, A.value, rho.value

    # -- state -----------------------------------------------------------
    def init(self):
        pos = np.zeros((self.n_b, 3), np.float64)
        self.lib().orc_init(ctypes.byref(self.d), _p(pos, ctypes.c_double))
        return pos

    def density(self, pos):
        pos = np.ascontiguousarray(pos, np.float64)
        out = np.zeros((2, self.n_c), np.uint32)
        self.lib().orc_density(ctypes.byref(self.d), _p(pos, ctypes.c_double), _p(out, ctypes.c_uint32))
        return out

    def fields(self, counts):
        counts = np.ascontiguousarray(counts, np.uint32)
        w = np.zeros((2, self.n_c), np.float64)
        self.lib().orc_fields(ctypes.byref(self.d), _p(counts, ctypes.c_uint32), _p(w, ctypes.c_double))
        return w

    def energy_nb(self, counts):
        counts = np.ascontiguousarray(counts, np.uint32)
        return float(self.lib().orc_energy_nb(ctypes.byref(self.d), _p(counts, ctypes.c_uint32)))

    def fields_from_phi(self, phi):
        phi = np.ascontiguousarray(phi, np.float64)
        w = np.zeros((2, self.n_c), np.float64)
        self.lib().orc_fields_from_phi(ctypes.byref(self.d), _p(phi, ctypes.c_double), _p(w, ctypes.c_double))
        return w

    def energy_umbrella(self, counts, target, lambdaN):
        counts = np.ascontiguousarray(counts, np.uint32)
        target = np.ascontiguousarray(target, np.float64)
        return float(self.lib().orc_energy_umbrella(ctypes.byref(self.d), _p(counts, ctypes.c_uint32),
                                                    _p(target, ctypes.c_double), float(lambdaN)))

    def fields_umbrella(self, counts, target, lambdaN):
        counts = np.ascontiguousarray(counts, np.uint32)
        target = np.ascontiguousarray(target, np.float64)
        w = np.zeros((2, self.n_c), np.float64)
        self.lib().orc_fields_umbrella(ctypes.byref(self.d), _p(counts, ctypes.c_uint32),
                                       _p(target, ctypes.c_double), float(lambdaN), _p(w, ctypes.c_double))
        return w

    def density_profile(self, counts, axis):
        """Laterally averaged volume fractions [2, grid[axis]] along one axis."""
        counts = np.ascontiguousarray(counts, np.uint32)
        out = np.zeros((2, int(self.d.grid[axis])), np.float64)
        self.lib().orc_density_profile(ctypes.byref(self.d), _p(counts, ctypes.c_uint32), int(axis),
                                       _p(out, ctypes.c_double))
        return out

    def vertical_correlation(self, counts, type_):
        """C(dz) of the type counts, dz = 0 .. nz-1."""
        counts = np.ascontiguousarray(counts, np.uint32)
        out = np.zeros(int(self.d.grid[2]), np.float64)
        self.lib().orc_vertical_correlation(ctypes.byref(self.d), _p(counts, ctypes.c_uint32), int(type_),
                                            _p(out, ctypes.c_double))
        return out

    def place(self, target):
        """Positions [n_b, 3] of molecules placed from float32 target volume
        fractions [2, n_c]; raises ValueError when bead 0's type has no weight."""
        target = np.ascontiguousarray(target, np.float32)
        pos = np.zeros((self.n_b, 3), np.float64)
        if self.lib().orc_place(ctypes.byref(self.d), _p(target, ctypes.c_float), _p(pos, ctypes.c_double)):
            raise ValueError("target weights of bead 0's type sum to zero")
        return pos

    def cell_index(self, r):
        r = np.ascontiguousarray(r, np.float64)
        return int(self.lib().orc_cell_index(ctypes.byref(self.d), _p(r, ctypes.c_double)))

    def mc_step(self, pos, w, t, n_threads=1, record=True):
        """One step in place on ``pos``; returns (accepted, acc flags, margins, face distances)."""
        assert pos.dtype == np.float64 and pos.flags.c_contiguous
        w = np.ascontiguousarray(w, np.float64)
        acc = np.zeros(self.n_b, np.uint8) if record else None
        margin = np.zeros(self.n_b, np.float64) if record else None
        face = np.zeros(self.n_b, np.float64) if record else None
        n = self.lib().orc_mc_step(ctypes.byref(self.d), _p(pos, ctypes.c_double), _p(w, ctypes.c_double),
                                   ctypes.c_uint32(t & 0xFFFFFFFF), _p(acc, ctypes.c_uint8),
                                   _p(margin, ctypes.c_double), _p(face, ctypes.c_double), n_threads)
        return n, acc, margin, face

    def mc_step_chains(self, pos, ids, w, t, n_threads=1):
        """One step of the chains with logical ids ``ids`` (pos [len(ids)*N, 3], in place)."""
        assert pos.dtype == np.float64 and pos.flags.c_contiguous
        ids = np.ascontiguousarray(ids, np.uint32)
        w = np.ascontiguousarray(w, np.float64)
        nb = len(ids) * self.d.N
        acc = np.zeros(nb, np.uint8)
        margin = np.zeros(nb, np.float64)
        face = np.zeros(nb, np.float64)
        n = self.lib().orc_mc_step_chains(ctypes.byref(self.d), _p(pos, ctypes.c_double), _p(ids, ctypes.c_uint32),
                                          len(ids), _p(w, ctypes.c_double), ctypes.c_uint32(t & 0xFFFFFFFF),
                                          _p(acc, ctypes.c_uint8), _p(margin, ctypes.c_double),
                                          _p(face, ctypes.c_double), n_threads)
        return n, acc, margin, face

    def run(self, pos, t0, n_steps, w_frozen=None, n_threads=1, occ=False, pair_hist=False,
            re2_trace=False, acc_trace=False, target=None, lambdaN=0.0):
        assert pos.dtype == np.float64 and pos.flags.c_contiguous
        wf = np.ascontiguousarray(w_frozen, np.float64) if w_frozen is not None else None
        tg = np.ascontiguousarray(target, np.float64) if target is not None else None
        o = np.zeros(2 * self.n_c, np.uint64) if occ else None
        ph = np.zeros(self.n_c * self.n_c, np.uint64) if pair_hist else None
        rt = np.zeros(n_steps, np.float64) if re2_trace else None
        at = np.zeros(n_steps, np.int64) if acc_trace else None
        total = self.lib().orc_run(ctypes.byref(self.d), _p(pos, ctypes.c_double), ctypes.c_uint32(t0),
                                   n_steps, _p(wf, ctypes.c_double), _p(tg, ctypes.c_double),
                                   float(lambdaN), n_threads, _p(o, ctypes.c_uint64),
                                   _p(ph, ctypes.c_uint64), _p(rt, ctypes.c_double), _p(at, ctypes.c_int64))
        return dict(accepted=total, occ=o, pair_hist=ph, re2=rt, acc=at)

    def observables(self, pos):
        pos = np.ascontiguousarray(pos, np.float64)
        o = OrcObs()
        self.lib().orc_observables(ctypes.byref(self.d), _p(pos, ctypes.c_double), ctypes.byref(o))
        return dict(Re2=o.Re2, Rg2=o.Rg2, Ebond=o.Ebond, Enb=o.Enb)

    def structure_factor(self, pos, m):
        pos = np.ascontiguousarray(pos, np.float64)
        m = np.ascontiguousarray(m, np.int32).reshape(-1, 3)
        S = np.zeros(len(m), np.float64)
        self.lib().orc_structure_factor(ctypes.byref(self.d), _p(pos, ctypes.c_double), len(m),
                                        _p(m, ctypes.c_int32), _p(S, ctypes.c_double))
        return S

    @classmethod
    def normal_quantile(cls, p):
        return float(cls.lib().orc_normal_quantile(float(p)))

    @classmethod
    def philox(cls, ctr, key):
        """Philox4x32-10 of counters ``ctr`` [n,4] under keys ``key`` [n,2] (uint32)."""
        ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
        key = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
        out = np.zeros_like(ctr)
        cls.lib().orc_philox4x32_many(len(ctr), _p(ctr, ctypes.c_uint32), _p(key, ctypes.c_uint32),
                                      _p(out, ctypes.c_uint32))
        return out
