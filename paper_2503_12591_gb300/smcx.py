"""Thin Python binding of the smcx C ABI (include/smcx.h).

Argument marshalling only: every computation runs in the CUDA library
``_build/libsmcx.so``.  There is no CPU fallback; if the library has not been
built, loading fails with an error that says so.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SMCX_DEBUG=1 loads the debug build (in-kernel bounds checks, see
# smcx_debug_status); otherwise the normal library.
LIB_PATH = os.path.join(HERE, "_build", "libsmcx_debug.so" if os.environ.get("SMCX_DEBUG") == "1" else "libsmcx.so")

BCC, FCC = 0, 1
INT8, PACKED4 = 0, 1
KERNEL_AUTO, KERNEL_GENERIC = 0, 1
PROPOSAL_SITE, PROPOSAL_TILE, PROPOSAL_BLOCK = 0, 1, 2
NA_MAX, NB = 4096, 1024

OK = 0
E_INVALID_ARG, E_NO_EPI, E_SCHEDULE, E_CUDA, E_OOM, E_TIMEOUT, E_RANGE, E_UNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7, -8)


class SmcxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"smcx error {code}: {msg}")
        self.code = code


class Sched(C.Structure):
    _fields_ = [("L", C.c_int32), ("nt", C.c_int32 * 3)]


_lib = None

# name -> (restype, argtypes); every entry point returns an int status
_SIGS = {
    "smcx_last_error": (C.c_char_p, []),
    "smcx_version": (C.c_int, []),
    "smcx_lattice_wrap": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p]),
    "smcx_local_energy": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_clusters": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "smcx_cluster_summary": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]),
    "smcx_set_qsro": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_autotune": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_void_p, C.c_void_p]),
    "smcx_store_bytes": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_get_config_store": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "smcx_set_config_store": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "smcx_sweep_energies": (C.c_int, [C.c_void_p, C.c_double, C.c_int64, C.c_uint64, C.c_void_p]),
    "smcx_sweep_cv": (C.c_int, [C.c_void_p, C.c_double, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p]),
    "smcx_debug_status": (C.c_int, [C.c_void_p]),
    "smcx_probe_lds_rate": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_lattice_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]),
    "smcx_lattice_destroy": (C.c_int, [C.c_void_p]),
    "smcx_set_epi": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "smcx_set_kernel": (C.c_int, [C.c_void_p, C.c_int]),
    "smcx_set_replica": (C.c_int, [C.c_void_p, C.c_int]),
    "smcx_set_block": (C.c_int, [C.c_void_p, C.c_int]),
    "smcx_set_proposal": (C.c_int, [C.c_void_p, C.c_int]),
    "smcx_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_void_p]),
    "smcx_batch_destroy": (C.c_int, [C.c_void_p]),
    "smcx_batch_sweep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64]),
    "smcx_batch_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "smcx_batch_exchange": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_uint64,
                                      C.c_void_p, C.c_void_p]),
    "smcx_batch_fluct_accumulate": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "smcx_batch_energy": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_batch_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smcx_batch_set_fault": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "smcx_batch_set_block": (C.c_int, [C.c_void_p, C.c_int]),
    "smcx_set_schedule": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_get_schedule": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_sweep": (C.c_int, [C.c_void_p, C.c_double, C.c_int64, C.c_uint64]),
    "smcx_sweep_partial": (C.c_int, [C.c_void_p, C.c_double, C.c_uint64, C.c_int]),
    "smcx_energy": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_pair_counts": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_sro": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_get_config": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_set_config": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smcx_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "smcx_set_sweep_counter": (C.c_int, [C.c_void_p, C.c_uint64]),
    "smcx_device_buffer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "smcx_synchronize": (C.c_int, [C.c_void_p]),
    "smcx_lattice_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "smcx_threshold_tables": (C.c_int, [C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smcx_pair_counts_batch": (C.c_int, [C.c_int] * 6 + [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "smcx_epi_energy_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "smcx_epi_grad_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "smcx_fluct_accumulate": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_int64, C.c_void_p, C.c_void_p]),
    "smcx_lattice_fluct_accumulate": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "smcx_fluct_gradient": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    "smcx_energy_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}


def lib():
    """Load libsmcx.so (built by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def debug_status():
    """(tag, index) of the first out-of-bounds access the debug build recorded
    since the last call, (0, 0) if none; SmcxError(E_UNSUPPORTED) in the
    normal build."""
    info = np.zeros(2, np.uint64)
    _check(lib().smcx_debug_status(_p(info)))
    return int(info[0]), int(info[1])


def probe_lds_rate(stream=None):
    """Measured shared-memory byte-load rate of the device (lane-loads/s)."""
    v = np.zeros(1, np.float64)
    _check(lib().smcx_probe_lds_rate(_p(v), _stream_ptr(stream)))
    return float(v[0])


def exported_symbols():
    return sorted(_SIGS)


def _check(rc):
    if rc != OK:
        raise SmcxError(rc, lib().smcx_last_error().decode())


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)  # torch.cuda.Stream


def threshold_tables(T):
    A = np.zeros(NA_MAX, np.uint32)
    B = np.zeros(NB, np.uint32)
    nA = np.zeros(1, np.int32)
    _check(lib().smcx_threshold_tables(float(T), _p(A), _p(nA), _p(B)))
    return A, int(nA[0]), B


def energy_noalloc(kind, dims, M, storage, V, d_sites, stream=None):
    """Energy of the configuration at device pointer d_sites (see
    smcx_energy_noalloc: no device allocation, one shared fixed scratch)."""
    V = np.ascontiguousarray(V, np.int32)
    e = np.zeros(1, np.int64)
    _check(lib().smcx_energy_noalloc(int(kind), *[int(d) for d in dims], int(M), int(storage), int(V.shape[0]),
                                     _p(V), C.c_void_p(int(d_sites)), _p(e), _stream_ptr(stream)))
    return int(e[0])


class Lattice:
    """A lattice handle (smcx_lattice)."""

    def __init__(self, kind, dims, M, comp, init_seed=1, storage=INT8, sched=None, stream=None):
        self.kind, self.dims, self.M, self.storage = kind, tuple(int(d) for d in dims), int(M), storage
        self.m = 2 if kind == BCC else 4
        self.N = self.dims[0] * self.dims[1] * self.dims[2] * self.m
        self.K = 0
        h = C.c_void_p()
        c = np.ascontiguousarray(comp, np.float64)
        sp = None
        if sched is not None:
            s = Sched(int(sched[0]), (C.c_int32 * 3)(*[int(t) for t in sched[1]]))
            sp = C.byref(s)
        _check(lib().smcx_lattice_create(C.byref(h), kind, *self.dims, self.M, _p(c), int(init_seed), storage,
                                         sp, _stream_ptr(stream)))
        self._h = h

    # -- local energies and clusters (device outputs) -----------------------
    def local_energy(self, d_e2):
        """2 E_i of every site into the device int32 buffer at d_e2 ([N])."""
        _check(lib().smcx_local_energy(self._h, C.c_void_p(int(d_e2))))

    def clusters(self, thr2, d_labels):
        """Cluster labels into the device int32 buffer at d_labels ([N]);
        returns the number of clusters."""
        n = np.zeros(1, np.int64)
        _check(lib().smcx_clusters(self._h, int(thr2), C.c_void_p(int(d_labels)), _p(n)))
        return int(n[0])

    def cluster_summary(self, d_labels, min_size, max_out):
        """(roots, sizes, species counts [n][M]) of the largest clusters."""
        roots = np.zeros(max(1, max_out), np.int64)
        sizes = np.zeros(max(1, max_out), np.int64)
        counts = np.zeros((max(1, max_out), self.M), np.int64)
        n = np.zeros(1, np.int32)
        _check(lib().smcx_cluster_summary(self._h, C.c_void_p(int(d_labels)), int(min_size), int(max_out),
                                          _p(roots), _p(sizes), _p(counts), _p(n)))
        k = int(n[0])
        return roots[:k], sizes[:k], counts[:k]

    @classmethod
    def wrap(cls, kind, dims, M, ptr, nbytes, storage=INT8, sched=None, stream=None, owner=None):
        """Handle over a caller-held device lattice store (smcx_lattice_wrap);
        `owner` (e.g. the torch tensor behind ptr) is kept alive with it."""
        self = cls.__new__(cls)
        self.kind, self.dims, self.M, self.storage = kind, tuple(int(d) for d in dims), int(M), storage
        self.m = 2 if kind == BCC else 4
        self.N = self.dims[0] * self.dims[1] * self.dims[2] * self.m
        self.K = 0
        self._owner = owner
        h = C.c_void_p()
        sp = None
        if sched is not None:
            s = Sched(int(sched[0]), (C.c_int32 * 3)(*[int(t) for t in sched[1]]))
            sp = C.byref(s)
        _check(lib().smcx_lattice_wrap(C.byref(h), kind, *self.dims, self.M, C.c_void_p(int(ptr)), int(nbytes),
                                       storage, sp, _stream_ptr(stream)))
        self._h = h
        return self

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _check(lib().smcx_lattice_destroy(self._h))
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

    # -- model and schedule ---------------------------------------------
    def set_epi(self, V):
        V = np.ascontiguousarray(V, np.int32)
        K = V.shape[0]
        assert V.shape == (K, self.M, self.M)
        _check(lib().smcx_set_epi(self._h, K, _p(V)))
        self.K = K

    def set_qsro(self, W):
        """qSRO weights W [K][M] (0.01 meV), or None for the pair model."""
        if W is None:
            _check(lib().smcx_set_qsro(self._h, None))
        else:
            W = np.ascontiguousarray(W, np.int32)
            if self.K and W.shape != (self.K, self.M):
                raise ValueError(f"W must have shape ({self.K}, {self.M})")
            _check(lib().smcx_set_qsro(self._h, _p(W)))

    def autotune(self, T, trial_sweeps=2):
        """Measure candidate schedules and install the fastest (smcx_autotune);
        returns ((L, tiles), threads)."""
        sc = Sched()
        th = np.zeros(1, np.int32)
        _check(lib().smcx_autotune(self._h, float(T), int(trial_sweeps), C.byref(sc), _p(th)))
        return (int(sc.L), tuple(int(t) for t in sc.nt)), int(th[0])

    def store_bytes(self):
        n = np.zeros(1, np.uint64)
        _check(lib().smcx_store_bytes(self._h, _p(n)))
        return int(n[0])

    def get_config_store(self):
        """The lattice store as stored (int8 ids or packed nibbles)."""
        out = np.empty(self.store_bytes(), np.uint8)
        _check(lib().smcx_get_config_store(self._h, _p(out), out.size))
        return out

    def get_config_store_ptr(self, ptr, nbytes):
        _check(lib().smcx_get_config_store(self._h, C.c_void_p(int(ptr)), int(nbytes)))

    def set_config_store(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        _check(lib().smcx_set_config_store(self._h, _p(buf), buf.size))

    def set_config_store_ptr(self, ptr, nbytes):
        _check(lib().smcx_set_config_store(self._h, C.c_void_p(int(ptr)), int(nbytes)))

    def sweep_energies(self, T, n_sweeps, seed):
        """n_sweeps sweeps; the exact energy after each (int64 [n_sweeps])."""
        E = np.zeros(max(1, int(n_sweeps)), np.int64)
        _check(lib().smcx_sweep_energies(self._h, float(T), int(n_sweeps), int(seed), _p(E)))
        return E[:int(n_sweeps)]

    def sweep_cv(self, T, n_sweeps, seed, want_trace=True):
        """n_sweeps sweeps; (trace or None, mean E, Var E, C_V / (N k_B)),
        the moments reduced on the device (smcx_sweep_cv)."""
        m = np.zeros(3, np.float64)
        E = np.zeros(max(1, int(n_sweeps)), np.int64) if want_trace else None
        _check(lib().smcx_sweep_cv(self._h, float(T), int(n_sweeps), int(seed), None if E is None else _p(E),
                                   _p(m)))
        return (None if E is None else E[:int(n_sweeps)]), float(m[0]), float(m[1]), float(m[2])

    def set_kernel(self, which):
        _check(lib().smcx_set_kernel(self._h, int(which)))

    def set_replica(self, r):
        _check(lib().smcx_set_replica(self._h, int(r)))

    def set_proposal(self, mode):
        _check(lib().smcx_set_proposal(self._h, int(mode)))

    def set_block(self, threads):
        _check(lib().smcx_set_block(self._h, int(threads)))

    def set_schedule(self, sched):
        if sched is None:
            _check(lib().smcx_set_schedule(self._h, None))
        else:
            s = Sched(int(sched[0]), (C.c_int32 * 3)(*[int(t) for t in sched[1]]))
            _check(lib().smcx_set_schedule(self._h, C.byref(s)))

    def schedule(self):
        s = Sched()
        _check(lib().smcx_get_schedule(self._h, C.byref(s)))
        return int(s.L), tuple(int(t) for t in s.nt)

    # -- compute ----------------------------------------------------------
    def sweep(self, T, n_sweeps, seed):
        _check(lib().smcx_sweep(self._h, float(T), int(n_sweeps), int(seed)))

    def sweep_partial(self, T, seed, n_colours):
        _check(lib().smcx_sweep_partial(self._h, float(T), int(seed), int(n_colours)))

    def energy(self):
        e = np.zeros(1, np.int64)
        _check(lib().smcx_energy(self._h, _p(e)))
        return int(e[0])

    def pair_counts(self):
        out = np.zeros((self.K, self.M, self.M), np.int64)
        _check(lib().smcx_pair_counts(self._h, _p(out)))
        return out

    def sro(self):
        out = np.zeros((self.K, self.M, self.M), np.float64)
        _check(lib().smcx_sro(self._h, _p(out)))
        return out

    # -- configuration and state -----------------------------------------
    def get_config(self, out=None):
        if out is None:
            out = np.empty(self.N, np.int8)
        assert out.dtype == np.int8 and out.size == self.N and out.flags.c_contiguous
        _check(lib().smcx_get_config(self._h, _p(out)))
        return out

    def set_config(self, cfg):
        cfg = np.ascontiguousarray(cfg, np.int8)
        assert cfg.size == self.N
        _check(lib().smcx_set_config(self._h, _p(cfg)))

    def get_config_ptr(self, host_ptr):
        _check(lib().smcx_get_config(self._h, C.c_void_p(host_ptr)))

    def set_config_ptr(self, host_ptr):
        _check(lib().smcx_set_config(self._h, C.c_void_p(host_ptr)))

    def state(self):
        sw = np.zeros(1, np.uint64)
        st = np.zeros(4, np.int64)
        _check(lib().smcx_get_state(self._h, _p(sw), _p(st)))
        return int(sw[0]), st

    def set_sweep_counter(self, n):
        _check(lib().smcx_set_sweep_counter(self._h, int(n)))

    def device_buffer(self):
        p = C.c_void_p()
        n = C.c_size_t()
        _check(lib().smcx_device_buffer(self._h, C.byref(p), C.byref(n)))
        return int(p.value or 0), int(n.value)

    def synchronize(self):
        _check(lib().smcx_synchronize(self._h))

    def fluct_accumulate(self, shell, d_acc_ptr):
        _check(lib().smcx_lattice_fluct_accumulate(self._h, int(shell), C.c_void_p(int(d_acc_ptr))))


class Batch:
    """Replicas swept together in one persistent launch (smcx_batch).  Holds
    references to the Lattice objects so they outlive the batch."""

    def __init__(self, lattices, stream=None):
        self.lattices = list(lattices)
        arr = (C.c_void_p * len(self.lattices))(*[l._h.value for l in self.lattices])
        h = C.c_void_p()
        _check(lib().smcx_batch_create(C.byref(h), len(self.lattices), arr, _stream_ptr(stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().smcx_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, T, n_sweeps, seed):
        T = np.ascontiguousarray(T, np.float64)
        assert T.size == len(self.lattices)
        _check(lib().smcx_batch_sweep(self._h, _p(T), int(n_sweeps), int(seed)))

    def autotune(self, T, trial_sweeps=2):
        T = np.ascontiguousarray(T, np.float64)
        th = np.zeros(1, np.int32)
        _check(lib().smcx_batch_autotune(self._h, _p(T), int(trial_sweeps), _p(th)))
        return int(th[0])

    def exchange(self, T_slot, slot_rep, n_rounds, sweeps_per_round, seed, round_ctr=0, accepts=None):
        """Replica exchange (smcx_batch_exchange).  Returns (slot_rep, round
        counter, accepts), the arrays updated copies of the inputs."""
        T = np.ascontiguousarray(T_slot, np.float64)
        R = len(self.lattices)
        assert T.size == R
        rep = np.ascontiguousarray(slot_rep, np.int32).copy()
        ctr = np.array([round_ctr], np.uint64)
        acc = (np.zeros(max(R - 1, 1), np.int64) if accepts is None
               else np.ascontiguousarray(accepts, np.int64).copy())
        _check(lib().smcx_batch_exchange(self._h, _p(T), _p(rep), int(n_rounds), int(sweeps_per_round), int(seed),
                                         _p(ctr), _p(acc)))
        return rep, int(ctr[0]), acc

    def fluct_accumulate(self, shell, d_acc):
        """Per-replica fluctuation sums into the device FP64 array at d_acc
        ([R][1 + MM + KMM + MM*KMM])."""
        _check(lib().smcx_batch_fluct_accumulate(self._h, int(shell), C.c_void_p(int(d_acc))))

    def energy(self):
        e = np.zeros(len(self.lattices), np.int64)
        _check(lib().smcx_batch_energy(self._h, _p(e)))
        return e

    def info(self):
        v = np.zeros(3, np.int32)
        _check(lib().smcx_batch_info(self._h, _p(v[0:]), _p(v[1:]), _p(v[2:])))
        return {"grid": int(v[0]), "threads": int(v[1]), "graph": bool(v[2])}

    def set_block(self, threads):
        _check(lib().smcx_batch_set_block(self._h, int(threads)))

    def set_fault(self, skip_cta, timeout_ms):
        _check(lib().smcx_batch_set_fault(self._h, int(skip_cta), int(timeout_ms)))


# ---- differentiation (device pointers; enqueued on `stream`) -------------
def pair_counts_batch(kind, dims, M, K, d_configs, B, d_counts, stream=None):
    _check(lib().smcx_pair_counts_batch(int(kind), *[int(d) for d in dims], int(M), int(K),
                                        C.c_void_p(int(d_configs)), int(B), C.c_void_p(int(d_counts)),
                                        _stream_ptr(stream)))


def epi_energy_batch(d_V, d_counts, B, KMM, d_E, stream=None):
    _check(lib().smcx_epi_energy_batch(C.c_void_p(int(d_V)), C.c_void_p(int(d_counts)), int(B), int(KMM),
                                       C.c_void_p(int(d_E)), _stream_ptr(stream)))


def epi_grad_batch(d_g, d_counts, B, KMM, d_grad, stream=None):
    _check(lib().smcx_epi_grad_batch(C.c_void_p(int(d_g)), C.c_void_p(int(d_counts)), int(B), int(KMM),
                                     C.c_void_p(int(d_grad)), _stream_ptr(stream)))


def fluct_accumulate(d_counts, B, d_weights, kind, K, M, shell, n_sites, d_acc, stream=None):
    _check(lib().smcx_fluct_accumulate(C.c_void_p(int(d_counts)), int(B),
                                       C.c_void_p(int(d_weights)) if d_weights else None, int(kind), int(K),
                                       int(M), int(shell), int(n_sites), C.c_void_p(int(d_acc)),
                                       _stream_ptr(stream)))


def fluct_gradient(d_acc, K, M, T, d_grad, stream=None):
    _check(lib().smcx_fluct_gradient(C.c_void_p(int(d_acc)), int(K), int(M), float(T), C.c_void_p(int(d_grad)),
                                     _stream_ptr(stream)))
