"""ctypes binding of libqaa.so (include/qaa.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  Device buffers are passed
as raw pointers; ``torch`` tensors (complex64 for states, int16/uint16 for the
energy diagonal) are accepted for convenience and only their ``data_ptr()`` is
used.  If the shared library is missing this module raises ImportError: there
is no fallback.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqaa.so")

QAA_OK = 0
QAA_PENDING = 1
STATUS_NAMES = {0: "QAA_OK", 1: "QAA_PENDING", -1: "QAA_E_ARG", -2: "QAA_E_NOMEM", -3: "QAA_E_CUDA",
                -4: "QAA_E_TIMEOUT", -5: "QAA_E_UNSAT", -6: "QAA_E_STATE"}
MAX_QUBITS = 34
MAX_CLAUSES = 1023


class QaaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Obs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("expect_hp", ctypes.c_double), ("expect_hb", ctypes.c_double),
                ("ground_prob", ctypes.c_double), ("ground_count", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("success_prob", ctypes.c_double), ("energy", ctypes.c_double), ("norm", ctypes.c_double),
                ("expect_hb", ctypes.c_double), ("ground_count", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("t_dev_start", ctypes.c_double),
                ("t_dev_end", ctypes.c_double), ("n", ctypes.c_int),
                ("steps", ctypes.c_int64), ("status", ctypes.c_int)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("peak_used_bytes", ctypes.c_size_t), ("batches", ctypes.c_int64),
                ("batched_requests", ctypes.c_int64), ("streamed_requests", ctypes.c_int64)]


_c_int, _vp, _dbl, _i64 = ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_int64

# name -> (restype, argtypes); the exported surface of include/qaa.h
SIGNATURES = {
    "qaa_version": (_c_int, []),
    "qaa_last_error": (ctypes.c_char_p, []),
    "qaa_create": (_c_int, [_c_int, _vp, _c_int, ctypes.POINTER(_vp)]),
    "qaa_destroy": (_c_int, [_vp]),
    "qaa_set_stream": (_c_int, [_vp, _vp]),
    "qaa_set_variant": (_c_int, [_vp, _c_int, _c_int]),
    "qaa_set_launch_mode": (_c_int, [_vp, _c_int]),
    "qaa_evolve_substeps": (_c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.c_int64]),
    "qaa_evolve_order4": (_c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int64]),
    "qaa_lowest_eigenvalues": (_c_int, [_vp, ctypes.c_double, _c_int, _c_int, _c_int, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "qaa_autotune": (_c_int, [_vp, _vp, _c_int, ctypes.c_double, ctypes.c_char_p, ctypes.c_size_t]),
    "qaa_tune_candidates": (_c_int, [_c_int, ctypes.c_char_p, ctypes.c_size_t]),
    "qaa_forget_tuned_plans": (_c_int, []),
    "qaa_init_uniform": (_c_int, [_vp, _vp]),
    "qaa_evolve": (_c_int, [_vp, _vp, _dbl, _i64]),
    "qaa_evolve_range": (_c_int, [_vp, _vp, _dbl, _i64, _i64, _i64]),
    "qaa_evolve_schedule": (_c_int, [_vp, _vp, _dbl, ctypes.POINTER(_dbl), _i64]),
    "qaa_observables": (_c_int, [_vp, _vp, ctypes.POINTER(Obs)]),
    "qaa_energy": (_c_int, [_vp, _vp, _dbl, ctypes.POINTER(_dbl)]),
    "qaa_success_prob": (_c_int, [_vp, _vp, ctypes.POINTER(_dbl)]),
    "qaa_norm": (_c_int, [_vp, _vp, ctypes.POINTER(_dbl)]),
    "qaa_hp_diagonal": (_c_int, [_vp, _vp]),
    "qaa_observables_noalloc": (_c_int, [_c_int, _vp, _c_int, _vp, _vp, ctypes.POINTER(Obs)]),
    "qaa_describe_plan": (_c_int, [_vp, ctypes.c_char_p, ctypes.c_size_t]),
    "qaa_server_create": (_c_int, [ctypes.c_size_t, _c_int, ctypes.POINTER(_vp)]),
    "qaa_submit": (_c_int, [_vp, _c_int, _vp, _c_int, _dbl, _i64, ctypes.POINTER(ctypes.c_uint64)]),
    "qaa_poll": (_c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "qaa_cancel": (_c_int, [_vp, ctypes.c_uint64]),
    "qaa_server_stats": (_c_int, [_vp, ctypes.POINTER(ServerInfo)]),
    "qaa_server_inject": (_c_int, [_vp, _c_int, _c_int]),
    "qaa_server_destroy": (_c_int, [_vp]),
    "qaa_profile_enable": (_c_int, [_vp, _c_int]),
    "qaa_profile_reset": (_c_int, [_vp]),
    "qaa_profile_read": (_c_int, [_vp, _c_int, ctypes.POINTER(_i64), ctypes.POINTER(_dbl)]),
}

KERNEL_KINDS = ["low_first", "low_merge", "low_last", "strided", "strided_phase", "tables", "onchip",
                "observe", "diag", "init", "graph"]
LAUNCH_PASSES, LAUNCH_GRAPH = 0, 1


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1103_1399_gb300.build.build() "
                          "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check(status):
    if status != QAA_OK:
        raise QaaError(status, lib.qaa_last_error().decode(errors="replace"))
    return status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("expected a device pointer (int) or an object with data_ptr()")


def tune_candidates(n):
    """Stage-1 autotune candidates for n, as plan descriptions (qaa_tune_candidates; no GPU needed)."""
    buf = ctypes.create_string_buffer(1 << 20)
    count = lib.qaa_tune_candidates(int(n), buf, len(buf))
    if count < 0:
        _check(count)
    return [line for line in buf.value.decode().split("\n") if line][:count]


def forget_tuned_plans():
    """Drop every plan recorded by autotune in this process (qaa_forget_tuned_plans)."""
    _check(lib.qaa_forget_tuned_plans())


def _check_state(inst, psi):
    if hasattr(psi, "dtype"):
        import torch
        if psi.dtype != torch.complex64 or not psi.is_cuda or not psi.is_contiguous():
            raise TypeError("psi must be a contiguous CUDA complex64 tensor")
        if psi.numel() != (1 << inst.n):
            raise ValueError(f"psi must have 2^{inst.n} elements")


def flatten_clauses(clauses):
    """List of clauses (each 1..3 signed literals) -> flat int32 buffer of m*3 (0-padded)."""
    flat = []
    for c in clauses:
        c = [int(l) for l in c]
        if not 1 <= len(c) <= 3:
            raise ValueError("clauses must have 1..3 literals")
        flat.extend(c + [0] * (3 - len(c)))
    buf = (ctypes.c_int32 * max(len(flat), 1))(*flat) if flat else (ctypes.c_int32 * 1)(0)
    return buf, len(clauses)


class Instance:
    """One 3-SAT instance on the current CUDA device (a qaa_handle)."""

    def __init__(self, n, clauses, stream=None):
        buf, m = flatten_clauses(clauses)
        h = ctypes.c_void_p()
        _check(lib.qaa_create(int(n), ctypes.cast(buf, ctypes.c_void_p), m, ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        self.m = m
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_h", None):
            lib.qaa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        """stream: an int cudaStream_t, or a torch.cuda.Stream."""
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        _check(lib.qaa_set_stream(self._h, s))

    def set_variant(self, wht_kind=0, q=0):
        _check(lib.qaa_set_variant(self._h, int(wht_kind), int(q)))

    def autotune(self, psi, steps=3, budget_ms=60000.0):
        """Time candidate pass plans on psi (overwritten); keep the fastest for this
        handle and for later handles / server requests with the same n.  Returns the
        report text (qaa_autotune)."""
        _check_state(self, psi)
        buf = ctypes.create_string_buffer(1 << 16)
        _check(lib.qaa_autotune(self._h, _ptr(psi), int(steps), float(budget_ms), buf, len(buf)))
        return buf.value.decode()

    def set_launch_mode(self, mode):
        """0: one launch per pass; 1: one CUDA graph per evolve range (qaa_set_launch_mode)."""
        _check(lib.qaa_set_launch_mode(self._h, int(mode)))

    def init_uniform(self, psi):
        _check_state(self, psi)
        _check(lib.qaa_init_uniform(self._h, _ptr(psi)))

    def evolve(self, psi, T, steps):
        _check_state(self, psi)
        _check(lib.qaa_evolve(self._h, _ptr(psi), float(T), int(steps)))

    def evolve_range(self, psi, T, steps, k0, k1):
        _check_state(self, psi)
        _check(lib.qaa_evolve_range(self._h, _ptr(psi), float(T), int(steps), int(k0), int(k1)))

    def evolve_schedule(self, psi, dt, s_values):
        _check_state(self, psi)
        s = [float(v) for v in s_values]
        arr = (ctypes.c_double * len(s))(*s)
        _check(lib.qaa_evolve_schedule(self._h, _ptr(psi), float(dt), arr, len(s)))

    def evolve_substeps(self, psi, dt_values, s_values):
        """Strang sub-steps of individual lengths dt_values[j], frozen at s_values[j] (qaa_evolve_substeps)."""
        _check_state(self, psi)
        d = [float(v) for v in dt_values]
        s = [float(v) for v in s_values]
        if len(d) != len(s):
            raise ValueError("dt_values and s_values must have the same length")
        da = (ctypes.c_double * len(d))(*d)
        sa = (ctypes.c_double * len(s))(*s)
        _check(lib.qaa_evolve_substeps(self._h, _ptr(psi), da, sa, len(d)))

    def evolve_order4(self, psi, T, steps):
        """The linear schedule in fourth-order (Yoshida triple-jump) steps (qaa_evolve_order4)."""
        _check_state(self, psi)
        _check(lib.qaa_evolve_order4(self._h, _ptr(psi), float(T), int(steps)))

    def lowest_eigenvalues(self, s, k=2, max_iter=200, start=0, seed=0):
        """Lowest k levels of H(s) by Lanczos (qaa_lowest_eigenvalues): (levels, iterations)."""
        ev = (ctypes.c_double * k)()
        found, its = _c_int(), _c_int()
        _check(lib.qaa_lowest_eigenvalues(self._h, float(s), int(k), int(max_iter), int(start), int(seed), ev,
                                          ctypes.byref(found), ctypes.byref(its)))
        return [ev[i] for i in range(found.value)], its.value

    def observables(self, psi):
        _check_state(self, psi)
        o = Obs()
        _check(lib.qaa_observables(self._h, _ptr(psi), ctypes.byref(o)))
        return {"norm": o.norm, "expect_hp": o.expect_hp, "expect_hb": o.expect_hb,
                "ground_prob": o.ground_prob, "ground_count": int(o.ground_count)}

    def energy(self, psi, s):
        _check_state(self, psi)
        out = ctypes.c_double()
        _check(lib.qaa_energy(self._h, _ptr(psi), float(s), ctypes.byref(out)))
        return out.value

    def success_prob(self, psi):
        _check_state(self, psi)
        out = ctypes.c_double()
        _check(lib.qaa_success_prob(self._h, _ptr(psi), ctypes.byref(out)))
        return out.value

    def norm(self, psi):
        _check_state(self, psi)
        out = ctypes.c_double()
        _check(lib.qaa_norm(self._h, _ptr(psi), ctypes.byref(out)))
        return out.value

    def describe_plan(self):
        buf = ctypes.create_string_buffer(512)
        _check(lib.qaa_describe_plan(self._h, buf, 512))
        return buf.value.decode()

    def profile(self, on=True):
        _check(lib.qaa_profile_enable(self._h, 1 if on else 0))

    def profile_reset(self):
        _check(lib.qaa_profile_reset(self._h))

    def profile_read(self):
        """{kind name: (launches, total_ms)} since the last reset (synchronises)."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            n = ctypes.c_int64()
            ms = ctypes.c_double()
            _check(lib.qaa_profile_read(self._h, k, ctypes.byref(n), ctypes.byref(ms)))
            out[name] = (int(n.value), float(ms.value))
        return out

    def hp_diagonal(self, out):
        """Write E(x) (uint16) for all x into a device buffer of 2^n 16-bit values."""
        if hasattr(out, "numel") and out.numel() != (1 << self.n):
            raise ValueError("out must have 2^n elements")
        _check(lib.qaa_hp_diagonal(self._h, _ptr(out)))


class Server:
    """Continuous-batching evolve server on the current device (qaa_server_*)."""

    def __init__(self, hbm_budget_bytes=0, max_slots=256):
        h = ctypes.c_void_p()
        _check(lib.qaa_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
        self._s = h

    def submit(self, n, clauses, T, steps):
        buf, m = flatten_clauses(clauses)
        t = ctypes.c_uint64()
        _check(lib.qaa_submit(self._s, int(n), ctypes.cast(buf, ctypes.c_void_p), m, float(T), int(steps),
                              ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        """None while pending, else a dict of the result (status 0 = QAA_OK)."""
        r = Result()
        st = lib.qaa_poll(self._s, ctypes.c_uint64(ticket), ctypes.byref(r))
        if st == QAA_PENDING:
            return None
        _check(st)
        return {f: getattr(r, f) for f, _ in Result._fields_}

    def cancel(self, ticket):
        _check(lib.qaa_cancel(self._s, ctypes.c_uint64(ticket)))

    def stats(self):
        i = ServerInfo()
        _check(lib.qaa_server_stats(self._s, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in ServerInfo._fields_}

    def inject(self, fault, param=0):
        _check(lib.qaa_server_inject(self._s, int(fault), int(param)))

    def close(self):
        if getattr(self, "_s", None):
            lib.qaa_server_destroy(self._s)
            self._s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
