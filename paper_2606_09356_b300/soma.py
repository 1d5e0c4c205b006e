"""Thin ctypes binding of libsoma (include/soma.h), same names as the C ABI.

Argument marshalling only: every step of the Monte Carlo path runs in the
CUDA kernels of libsoma.so.  There is no CPU fallback; importing this module
without the built library raises.

Module-level functions mirror the C calls one to one (``soma_create``,
``soma_mc_steps`` ...).  ``System`` describes one melt and ``Handle`` wraps a
handle with numpy-returning convenience methods.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY = os.path.join(_HERE, "libsoma.so")
LIBRARY_DEBUG = os.path.join(_HERE, "libsoma_debug.so")  # checked build (device bounds checks)

SOMA_OK = 0
SOMA_EINVAL = -1
SOMA_ENOMEM = -2
SOMA_ECUDA = -3
SOMA_ETIMEOUT = -4
SOMA_EDEVICE_CHECK = -5
SOMA_ESTATE = -6
SOMA_ENOTSUP = -7
SOMA_HOST = 0
SOMA_DEVICE = 1
SOMA_PREC_FP32 = 0
SOMA_PREC_FP64 = 1
SOMA_MOVE_UNIFORM = 0
SOMA_MOVE_SMART = 1
SOMA_HIST_AUTO = 0
SOMA_HIST_FUSED = 1
SOMA_HIST_SEPARATE = 2

# every entry point declared in include/soma.h
EXPORTS = (
    "soma_options_default", "soma_create", "soma_destroy", "soma_strerror", "soma_last_error",
    "soma_mc_steps", "soma_sync", "soma_get_density", "soma_density_profile", "soma_vertical_correlation",
    "soma_get_fields",
    "soma_set_density",
    "soma_freeze_fields", "soma_set_umbrella", "soma_place", "soma_get_state", "soma_set_state",
    "soma_get_state64", "soma_set_state64", "soma_observables", "soma_get_accepted", "soma_copy_accepted",
    "soma_structure_factor", "soma_reorder", "soma_get_info", "soma_kernel_times", "soma_autotune",
    "soma_philox4x32", "soma_structure_factor_noalloc", "soma_selfcheck_timeout",
    "soma_normal_deviates", "soma_set_conversion", "soma_get_conversions", "soma_get_chain_types",
    "soma_set_chain_types", "soma_create_partition", "soma_exchange_counts", "soma_sort_pairs",
)


class SomaError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {soma_strerror(code)} ({code})")


class soma_system_desc(ctypes.Structure):
    _fields_ = [
        ("n_poly", ctypes.c_int32), ("N", ctypes.c_int32), ("n_A", ctypes.c_int32),
        ("system_id", ctypes.c_int32), ("grid", ctypes.c_int32 * 3), ("move", ctypes.c_int32),
        ("box", ctypes.c_double * 3), ("chiN", ctypes.c_double), ("kappaN", ctypes.c_double),
        ("A", ctypes.c_double), ("seed", ctypes.c_uint64), ("wall_z", ctypes.c_int32),
        ("reserved2", ctypes.c_int32),
    ]


_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class soma_options(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int32), ("sort_interval", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
        ("hist_mode", ctypes.c_int32), ("graph_steps", ctypes.c_int32), ("kernel_timing", ctypes.c_int32),
        ("autotune", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("alloc", _ALLOC), ("free", _FREE), ("alloc_ctx", ctypes.c_void_p),
        ("move_warps", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class soma_obs(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_uint64), ("accepted", ctypes.c_uint64), ("attempted", ctypes.c_uint64),
        ("acc", ctypes.c_double), ("Re2", ctypes.c_double), ("Rg2", ctypes.c_double),
        ("Ebond", ctypes.c_double), ("Enb", ctypes.c_double),
    ]


class soma_info(ctypes.Structure):
    _fields_ = [
        ("n_beads", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("k_b", ctypes.c_double),
        ("A", ctypes.c_double), ("rho_bar", ctypes.c_double), ("lanes_per_chain", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32), ("sort_interval", ctypes.c_int32), ("hist_mode", ctypes.c_int32),
        ("move_warps", ctypes.c_int32), ("reserved2", ctypes.c_int32),
    ]


_lib = None


def load_library(path=None):
    """Load libsoma.so (built in-tree by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIBRARY
    if not os.path.exists(path):
        raise ImportError(f"libsoma.so not built at {path}: run paper_2606_09356_b300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, sz, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_uint64
    L.soma_options_default.argtypes = [ctypes.POINTER(soma_options)]
    L.soma_create.argtypes = [ctypes.POINTER(soma_system_desc), i32, ctypes.POINTER(soma_options), ctypes.POINTER(vp)]
    L.soma_destroy.argtypes = [vp]
    L.soma_destroy.restype = None
    L.soma_strerror.argtypes = [i32]
    L.soma_strerror.restype = ctypes.c_char_p
    L.soma_last_error.argtypes = [vp]
    L.soma_mc_steps.argtypes = [vp, i64, vp]
    L.soma_sync.argtypes = [vp, vp]
    L.soma_get_density.argtypes = [vp, i32, vp, sz, i32]
    L.soma_get_fields.argtypes = [vp, i32, vp, sz, i32]
    L.soma_set_density.argtypes = [vp, i32, vp, sz, i32]
    L.soma_freeze_fields.argtypes = [vp, i32, vp, sz, i32]
    L.soma_set_umbrella.argtypes = [vp, i32, vp, sz, ctypes.c_double, i32]
    L.soma_selfcheck_timeout.argtypes = [i32, u64]
    L.soma_copy_accepted.argtypes = [vp, i32, vp, vp]
    L.soma_density_profile.argtypes = [vp, i32, i32, vp, sz]
    L.soma_vertical_correlation.argtypes = [vp, i32, i32, vp, sz]
    L.soma_normal_deviates.argtypes = [vp, vp, sz]
    L.soma_place.argtypes = [vp, i32, vp, sz, i32]
    L.soma_get_state.argtypes = [vp, i32, vp, vp, ctypes.POINTER(u64), i32]
    L.soma_set_state.argtypes = [vp, i32, vp, vp, u64, i32]
    L.soma_get_state64.argtypes = [vp, i32, vp, vp, ctypes.POINTER(u64), i32]
    L.soma_set_state64.argtypes = [vp, i32, vp, vp, u64, i32]
    L.soma_observables.argtypes = [vp, i32, ctypes.POINTER(soma_obs)]
    L.soma_get_accepted.argtypes = [vp, i32, ctypes.POINTER(u64)]
    L.soma_structure_factor.argtypes = [vp, i32, i32, vp, vp]
    L.soma_reorder.argtypes = [vp, vp]
    L.soma_get_info.argtypes = [vp, i32, ctypes.POINTER(soma_info)]
    L.soma_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32]
    L.soma_autotune.argtypes = [vp]
    L.soma_philox4x32.argtypes = [vp, vp, vp, sz]
    L.soma_structure_factor_noalloc.argtypes = [vp, i64, ctypes.c_int32, ctypes.c_int32, vp, i32, vp, vp, vp]
    L.soma_set_conversion.argtypes = [vp, i32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, vp]
    L.soma_get_conversions.argtypes = [vp, i32, vp]
    L.soma_get_chain_types.argtypes = [vp, i32, vp, sz]
    L.soma_set_chain_types.argtypes = [vp, i32, vp, sz]
    L.soma_create_partition.argtypes = [ctypes.POINTER(soma_system_desc), ctypes.POINTER(soma_options),
                                        ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vp)]
    L.soma_exchange_counts.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(sz)]
    L.soma_sort_pairs.argtypes = [vp, vp, sz, i32, vp, vp]
    for name in EXPORTS:
        if name not in ("soma_destroy", "soma_strerror"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor on the device
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _where(a):
    return SOMA_DEVICE if hasattr(a, "data_ptr") and a.is_cuda else SOMA_HOST


def _numel_f32(a, what):
    """Element count of a float32 buffer (numpy array or contiguous float32
    torch tensor, host or device)."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous float32 tensor")
        return a.numel()
    return a.size


def _check_words(a, n, itemsize, what):
    """A caller buffer of n contiguous elements of the given byte size
    (numpy array or torch tensor, host or device)."""
    if hasattr(a, "data_ptr"):
        ok = a.numel() == n and a.element_size() == itemsize and a.is_contiguous()
    else:
        ok = a.size == n and a.itemsize == itemsize and a.flags.c_contiguous
    if not ok:
        raise ValueError(f"{what}: expected {n} contiguous elements of {itemsize} bytes")


def _check_buffer(a, n, np_dtype, what):
    """A caller buffer the C call fills or reads in full: contiguous, of the
    right element type and exactly n elements (the C calls take no length)."""
    if hasattr(a, "data_ptr"):
        import torch
        tdt = {np.dtype(np.float32): torch.float32, np.dtype(np.int16): torch.int16,
               np.dtype(np.float64): torch.float64}[np.dtype(np_dtype)]
        ok = a.numel() == n and a.is_contiguous() and a.dtype == tdt
    else:
        ok = a.size == n and a.dtype == np_dtype and a.flags.c_contiguous
    if not ok:
        raise ValueError(f"{what}: expected a contiguous {np.dtype(np_dtype).name} buffer of {n} elements")


def _check(code, what):
    if code != SOMA_OK:
        raise SomaError(code, what)


# ---------------------------------------------------------------------------
# one-to-one C calls
# ---------------------------------------------------------------------------
def soma_strerror(code):
    return load_library().soma_strerror(code).decode()


def soma_options_default():
    o = soma_options()
    _check(load_library().soma_options_default(ctypes.byref(o)), "soma_options_default")
    return o


def soma_create(descs, options=None):
    L = load_library()
    arr = (soma_system_desc * len(descs))(*descs)
    h = ctypes.c_void_p()
    rc = L.soma_create(arr, len(descs), ctypes.byref(options) if options is not None else None, ctypes.byref(h))
    _check(rc, "soma_create")
    return h


def soma_create_partition(desc, chain_begin, chain_end, options=None):
    """A handle for the logical chains [chain_begin, chain_end) of one system."""
    L = load_library()
    h = ctypes.c_void_p()
    rc = L.soma_create_partition(ctypes.byref(desc), ctypes.byref(options) if options is not None else None,
                                 int(chain_begin), int(chain_end), ctypes.byref(h))
    _check(rc, "soma_create_partition")
    return h


def soma_exchange_counts(h):
    """(device pointer, number of uint32 words) of the counts the next step reads."""
    p, n = ctypes.c_void_p(), ctypes.c_size_t()
    _check(load_library().soma_exchange_counts(h, ctypes.byref(p), ctypes.byref(n)), "soma_exchange_counts")
    return p.value, n.value


def soma_destroy(h):
    load_library().soma_destroy(h)


def soma_mc_steps(h, n_steps, stream=None):
    _check(load_library().soma_mc_steps(h, int(n_steps), stream), "soma_mc_steps")


def soma_philox4x32(ctr, key):
    """Device Philox4x32-10 of counters [n,4] under keys [n,2] (uint32)."""
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    _check(load_library().soma_philox4x32(_ptr(ctr), _ptr(key), _ptr(out), len(ctr)), "soma_philox4x32")
    return out


def _check_current_device_tensor(a, what):
    """A torch tensor the C call reads or writes on the device: it must be a
    CUDA tensor on the current device, where the call runs."""
    import torch
    if not (isinstance(a, torch.Tensor) and a.is_cuda):
        raise ValueError(f"{what}: expected a CUDA tensor (or a raw device pointer as an int)")
    if a.device.index != torch.cuda.current_device():
        raise ValueError(f"{what}: tensor on cuda:{a.device.index}, but the current device is "
                         f"cuda:{torch.cuda.current_device()}")


def soma_structure_factor_noalloc(pos, n_beads, N, n_A, box, m, S, stream=None):
    """S(q) of device positions ``pos`` [n_beads, 3] FP32 into device ``S``
    [nq] FP64; the library allocates nothing.  pos and S are CUDA tensors on
    the current device (checked for type, size, contiguity and device) or
    raw device pointers given as ints (not checked: the caller vouches for
    them).  Every chain is taken as the base diblock (beads 0 .. n_A-1 A)."""
    box = np.ascontiguousarray(box, np.float64).reshape(-1)
    if box.size != 3:
        raise ValueError("box: expected 3 edges")
    m = np.ascontiguousarray(m, np.int32).reshape(-1, 3)
    tensors = [(a, n, dt, what) for a, n, dt, what in ((pos, 3 * int(n_beads), np.float32, "pos"),
                                                       (S, len(m), np.float64, "S")) if not isinstance(a, int)]
    for a, n, dt, what in tensors:
        _check_buffer(a, n, dt, what)
    for a, _, _, what in tensors:
        _check_current_device_tensor(a, what)
    p = pos if isinstance(pos, int) else pos.data_ptr()
    q = S if isinstance(S, int) else S.data_ptr()
    _check(load_library().soma_structure_factor_noalloc(ctypes.c_void_p(p), int(n_beads), int(N), int(n_A),
                                                         _ptr(box), len(m), _ptr(m), ctypes.c_void_p(q), stream),
           "soma_structure_factor_noalloc")


def soma_sort_pairs(keys, vals, end_bit=64):
    """The library's stable radix sort of (uint64 key, uint32 value) pairs by
    the key bits [0, end_bit) (verification aid)."""
    keys = np.ascontiguousarray(keys, np.uint64)
    vals = np.ascontiguousarray(vals, np.uint32)
    if keys.shape != vals.shape or keys.ndim != 1:
        raise ValueError("keys and vals: two 1-D arrays of the same length")
    ko, vo = np.empty_like(keys), np.empty_like(vals)
    _check(load_library().soma_sort_pairs(_ptr(keys), _ptr(vals), keys.size, int(end_bit), _ptr(ko), _ptr(vo)),
           "soma_sort_pairs")
    return ko, vo


def soma_normal_deviates(words):
    """The smart move's normal deviates of uint32 words (as the kernel computes them)."""
    words = np.ascontiguousarray(words, np.uint32)
    out = np.zeros(words.shape, np.float32)
    _check(load_library().soma_normal_deviates(_ptr(words), _ptr(out), words.size), "soma_normal_deviates")
    return out


def soma_selfcheck_timeout(device=-1, cycles=200_000_000):
    """Return code of the bounded-wait self-check (SOMA_ETIMEOUT when the
    failure path works as designed)."""
    return int(load_library().soma_selfcheck_timeout(device, cycles))


def soma_sync(h, stream=None):
    _check(load_library().soma_sync(h, stream), "soma_sync")


# ---------------------------------------------------------------------------
class System:
    """One AB diblock melt (the fields of soma_system_desc)."""

    def __init__(self, n_poly, N, n_A, box, grid, chiN, kappaN, A=0.0, seed=1, system_id=0,
                 move=SOMA_MOVE_UNIFORM, wall_z=0):
        self.n_poly, self.N, self.n_A = int(n_poly), int(N), int(n_A)
        self.system_id = int(system_id)
        self.move = int(move)
        self.wall_z = int(wall_z)
        self.box = tuple(float(b) for b in box)
        self.grid = tuple(int(g) for g in grid)
        self.chiN, self.kappaN, self.A, self.seed = float(chiN), float(kappaN), float(A), int(seed)

    @property
    def n_beads(self):
        return self.n_poly * self.N

    @property
    def n_cells(self):
        return self.grid[0] * self.grid[1] * self.grid[2]

    def desc(self):
        d = soma_system_desc()
        d.n_poly, d.N, d.n_A, d.system_id = self.n_poly, self.N, self.n_A, self.system_id
        d.move = self.move
        d.wall_z = self.wall_z
        for a in range(3):
            d.grid[a] = self.grid[a]
            d.box[a] = self.box[a]
        d.chiN, d.kappaN, d.A, d.seed = self.chiN, self.kappaN, self.A, self.seed
        return d


class PartitionOf(System):
    """The logical chains [begin, end) of a system: sizes are the partition's
    (n_poly = end - begin), the descriptor the whole system's."""

    def __init__(self, system, begin, end):
        super().__init__(system.n_poly, system.N, system.n_A, system.box, system.grid, system.chiN,
                         system.kappaN, system.A, system.seed, system.system_id, system.move, system.wall_z)
        self.whole, self.begin, self.end = system, int(begin), int(end)
        self.n_poly = self.end - self.begin

    def desc(self):
        return self.whole.desc()


class Handle:
    """Owns a soma_handle for a list of systems that step together, or, with
    partition=(begin, end), for the logical chains [begin, end) of one system
    (soma_create_partition)."""

    def __init__(self, systems, partition=None, **options):
        if isinstance(systems, System):
            systems = [systems]
        self.systems = list(systems)
        self.lib = load_library()
        o = soma_options_default()
        for k, v in options.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown soma option {k}")
            setattr(o, k, v)
        self.precision = o.precision
        self.device = int(o.device)
        if self.device < 0:
            try:
                import torch
                self.device = torch.cuda.current_device() if torch.cuda.is_available() else 0
            except ImportError:
                self.device = 0
        if partition is not None:
            if len(self.systems) != 1:
                raise ValueError("a partition holds chains of one system")
            self.systems = [PartitionOf(self.systems[0], *partition)]
            self.h = soma_create_partition(self.systems[0].desc(), partition[0], partition[1], o)
        else:
            self.h = soma_create([s.desc() for s in self.systems], o)

    def close(self):
        if self.h:
            soma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- stepping --------------------------------------------------------
    def mc_steps(self, n, stream=None):
        soma_mc_steps(self.h, n, stream)

    def exchange_counts(self):
        """(device pointer, uint32 words) of the counts the next step reads
        (a partition: to be summed over all partitions before that step)."""
        return soma_exchange_counts(self.h)

    def sync(self, stream=None):
        soma_sync(self.h, stream)

    def reorder(self, stream=None):
        _check(self.lib.soma_reorder(self.h, stream), "soma_reorder")

    def autotune(self):
        _check(self.lib.soma_autotune(self.h), "soma_autotune")

    # -- grids -----------------------------------------------------------
    def get_density(self, sys=0, out=None):
        nc = self.systems[sys].n_cells
        out = np.zeros((2, nc), np.uint32) if out is None else out
        _check_words(out, 2 * nc, 4, "out")
        _check(self.lib.soma_get_density(self.h, sys, _ptr(out), 2 * nc, _where(out)), "soma_get_density")
        return out

    def density_profile(self, axis, sys=0):
        """Laterally averaged volume fractions [2, grid[axis]] along one axis."""
        out = np.zeros((2, self.systems[sys].grid[axis]), np.float64)
        _check(self.lib.soma_density_profile(self.h, sys, int(axis), _ptr(out), out.size), "soma_density_profile")
        return out

    def vertical_correlation(self, type_, sys=0):
        """C(dz) of the type counts (0 = A, 1 = B), dz = 0 .. grid[2]-1."""
        out = np.zeros(self.systems[sys].grid[2], np.float64)
        _check(self.lib.soma_vertical_correlation(self.h, sys, int(type_), _ptr(out), out.size),
               "soma_vertical_correlation")
        return out

    def get_fields(self, sys=0):
        nc = self.systems[sys].n_cells
        out = np.zeros((2, nc), np.float32)
        _check(self.lib.soma_get_fields(self.h, sys, _ptr(out), 2 * nc, SOMA_HOST), "soma_get_fields")
        return out

    def set_density(self, phi, sys=0):
        phi = np.ascontiguousarray(phi, np.float32)
        _check(self.lib.soma_set_density(self.h, sys, _ptr(phi), phi.size, SOMA_HOST), "soma_set_density")

    def freeze_fields(self, w, sys=0):
        if w is None:
            _check(self.lib.soma_freeze_fields(self.h, sys, None, 0, SOMA_HOST), "soma_freeze_fields")
            return
        w = np.ascontiguousarray(w, np.float32)
        _check(self.lib.soma_freeze_fields(self.h, sys, _ptr(w), w.size, SOMA_HOST), "soma_freeze_fields")

    # -- state -----------------------------------------------------------
    def set_conversion(self, n_A_alt, zone_lo=0.0, zone_hi=0.0, p=(0.0, 0.0, 0.0, 0.0), sys=0):
        """Boundary-zone conversion: converted molecules have n_A_alt A beads;
        zone widths in z; p = per-step probabilities (bottom 0->1, bottom
        1->0, top 0->1, top 1->0).  n_A_alt < 0 switches it off."""
        pv = np.ascontiguousarray(p, np.float64).reshape(-1)
        if pv.size != 4:
            raise ValueError("p holds four per-step probabilities")
        _check(self.lib.soma_set_conversion(self.h, sys, int(n_A_alt), float(zone_lo), float(zone_hi), _ptr(pv)),
               "soma_set_conversion")

    def conversions(self, sys=0):
        """Conversions since the rates were last set, in the order of p."""
        out = np.zeros(4, np.uint64)
        _check(self.lib.soma_get_conversions(self.h, sys, _ptr(out)), "soma_get_conversions")
        return out

    def chain_types(self, sys=0):
        """Molecule type (0 own, 1 converted) of every chain, logical order."""
        out = np.zeros(self.systems[sys].n_poly, np.uint8)
        _check(self.lib.soma_get_chain_types(self.h, sys, _ptr(out), out.size), "soma_get_chain_types")
        return out

    def set_chain_types(self, types, sys=0):
        """Set every chain's molecule type (conversion must be on); the counts
        and fields are rebuilt with the new types."""
        t = np.ascontiguousarray(types, np.uint8)
        _check(self.lib.soma_set_chain_types(self.h, sys, _ptr(t), t.size), "soma_set_chain_types")

    def set_umbrella(self, phi_target, lambdaN, sys=0):
        """Restraint toward target volume fractions [2, n_c]; None or 0 turns it off."""
        if phi_target is None or lambdaN == 0:
            _check(self.lib.soma_set_umbrella(self.h, sys, None, 0, 0.0, SOMA_HOST), "soma_set_umbrella")
            return
        if not hasattr(phi_target, "data_ptr"):
            phi_target = np.ascontiguousarray(phi_target, np.float32)
        _check(self.lib.soma_set_umbrella(self.h, sys, _ptr(phi_target), _numel_f32(phi_target, "phi_target"),
                                          float(lambdaN),
                                          _where(phi_target)), "soma_set_umbrella")

    def place(self, phi_target, sys=0):
        """New configuration of molecules placed from target volume fractions [2, n_c]."""
        if not hasattr(phi_target, "data_ptr"):
            phi_target = np.ascontiguousarray(phi_target, np.float32)
        _check(self.lib.soma_place(self.h, sys, _ptr(phi_target), _numel_f32(phi_target, "phi_target"),
                                   _where(phi_target)),
               "soma_place")

    def get_state(self, sys=0, pos=None, img=None):
        nb = self.systems[sys].n_beads
        pos = np.zeros((nb, 3), np.float32) if pos is None else pos
        img = np.zeros((nb, 3), np.int16) if img is None else img
        _check_buffer(pos, 3 * nb, np.float32, "pos")
        _check_buffer(img, 3 * nb, np.int16, "img")
        if _where(pos) != _where(img):
            raise ValueError("pos and img must both be host or both be device buffers")
        step = ctypes.c_uint64()
        _check(self.lib.soma_get_state(self.h, sys, _ptr(pos), _ptr(img), ctypes.byref(step), _where(pos)),
               "soma_get_state")
        return pos, img, step.value

    def set_state(self, pos, img, step, sys=0):
        where = _where(pos)
        if where == SOMA_HOST:
            pos = np.ascontiguousarray(pos, np.float32)
            img = np.ascontiguousarray(img, np.int16)
        nb = self.systems[sys].n_beads
        _check_buffer(pos, 3 * nb, np.float32, "pos")
        _check_buffer(img, 3 * nb, np.int16, "img")
        if _where(img) != where:
            raise ValueError("pos and img must both be host or both be device buffers")
        _check(self.lib.soma_set_state(self.h, sys, _ptr(pos), _ptr(img), int(step), where), "soma_set_state")

    def get_state64(self, sys=0):
        nb = self.systems[sys].n_beads
        pos = np.zeros((nb, 3), np.float64)
        img = np.zeros((nb, 3), np.int16)
        step = ctypes.c_uint64()
        _check(self.lib.soma_get_state64(self.h, sys, _ptr(pos), _ptr(img), ctypes.byref(step), SOMA_HOST),
               "soma_get_state64")
        return pos, img, step.value

    def set_state64(self, pos, img, step, sys=0):
        pos = np.ascontiguousarray(pos, np.float64)
        img = np.ascontiguousarray(img, np.int16)
        nb = self.systems[sys].n_beads
        _check_buffer(pos, 3 * nb, np.float64, "pos")
        _check_buffer(img, 3 * nb, np.int16, "img")
        _check(self.lib.soma_set_state64(self.h, sys, _ptr(pos), _ptr(img), int(step), SOMA_HOST),
               "soma_set_state64")

    def unwrapped(self, sys=0):
        """FP64 unwrapped positions x + image * L in logical order."""
        if getattr(self, "precision", 0) == SOMA_PREC_FP64:
            pos, img, _ = self.get_state64(sys)
        else:
            pos, img, _ = self.get_state(sys)
        return pos.astype(np.float64) + img.astype(np.float64) * np.array(self.systems[sys].box)

    # -- measurements ----------------------------------------------------
    def observables(self, sys=0):
        o = soma_obs()
        _check(self.lib.soma_observables(self.h, sys, ctypes.byref(o)), "soma_observables")
        nb = self.systems[sys].n_beads
        return dict(step=o.step, accepted=o.accepted, attempted=o.attempted, acc=o.acc, Re2=o.Re2, Rg2=o.Rg2,
                    Ebond=o.Ebond, Enb=o.Enb, n_beads=nb)

    def accepted(self, sys=0):
        a = ctypes.c_uint64()
        _check(self.lib.soma_get_accepted(self.h, sys, ctypes.byref(a)), "soma_get_accepted")
        return a.value

    def copy_accepted(self, dst, sys=0, stream=None):
        """Enqueue the accepted count into dst (a 1-element uint64 host array;
        pinned and 8-byte aligned, the reduction kernel writes it directly,
        otherwise it is copied); valid after the stream synchronises."""
        _check_words(dst, 1, 8, "dst")
        _check(self.lib.soma_copy_accepted(self.h, sys, _ptr(dst), stream), "soma_copy_accepted")

    def structure_factor(self, m, sys=0):
        m = np.ascontiguousarray(m, np.int32).reshape(-1, 3)
        S = np.zeros(len(m), np.float64)
        _check(self.lib.soma_structure_factor(self.h, sys, len(m), _ptr(m), _ptr(S)), "soma_structure_factor")
        return S

    def info(self, sys=0):
        i = soma_info()
        _check(self.lib.soma_get_info(self.h, sys, ctypes.byref(i)), "soma_get_info")
        return {f: getattr(i, f) for f, _ in soma_info._fields_}

    def kernel_times(self, reset=False):
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        _check(self.lib.soma_kernel_times(self.h, ms, n, int(reset)), "soma_kernel_times")
        names = ("move", "bin", "field", "reorder")
        return {k: (ms[i], n[i]) for i, k in enumerate(names)}
